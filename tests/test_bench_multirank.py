"""bench.py under torchrun with two ranks (CPU, gloo): only rank 0 prints one
JSON line, and the run ends cleanly on every rank.  Uses the oracle arm on the
small workload so it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_two_ranks_print_one_line(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29531",
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--case", "1",
           "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=str(tmp_path), env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def _max_rank_worker(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # each rank's timed region; the slowest one sets the whole job's time
        v = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, torch.device("cpu"))
        out.put((rank, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_takes_the_slowest_rank():
    # the reduction the GPU arm applies to its timed region and its end-to-end
    # time, run over two gloo ranks on CPU
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_max_rank_worker, args=(r, 2, 29533, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = dict(out.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}
