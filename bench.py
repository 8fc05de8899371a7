"""Benchmark: HSMA3D energy+force evaluations per second on one GB300.

Workload (one "step" = one full evaluation of the hot path: prep, near field,
check-point sums, fit + surface map, far field, assembly), the largest
single-GPU configuration:
  N = 262,144 ions (87,381 at +2, 174,762 at -1, one at 0: neutral; uniform,
  number density 0.1, so L = 137.9), p = 10, M = 4,000 Fibonacci surface
  charges, lambda = 1.3 (27-cell shell), FP32 pair arithmetic with compensated
  FP64 accumulation and an FP64 fit.
Seeded synthetic input (the paper's electrolytes are MD states that are not
available).  ``value`` is evaluations/s with inputs resident in HBM; ``e2e``
is the same through the C ABI with pinned host buffers, copies included.
The N = 100,000, p = 8, M = 2,000 workload is reported beside it (``case2``),
and the served request stream last (``serve``, ``serve_precision2``).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank evaluates its own independent replica (no data-path
collective); timing is the max over ranks.
"""
import argparse
import json
import math
import os
import platform
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "HSMA energy+force evals/s & pair-ints/s at stated rel. error; serve p50/p99 ms"
FP32_INSTR_PER_PAIR = 13      # 3 FADD, 3 FMUL/FFMA for r^2, 4 FMUL, 1 FADD, 3 FFMA
FLOP_PER_PAIR = 20            # FMA = 2, rsqrt = 2
FP32_LANES = 128              # FP32 lanes per SM


def sm_count():
    """Streaming multiprocessors of the current CUDA device."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def peaks():
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(mp.get("sm_max_mhz", 2070.0)), "measured sm_max_mhz"
    except Exception:
        return 2070.0, "fallback 2070 MHz"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index, path=None):
        import tempfile
        self.index = index
        self.proc = None
        self.keep = path is not None
        self.path = path or os.path.join(tempfile.gettempdir(), f"hsma_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
            if not self.keep:
                os.remove(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
            except Exception:
                continue
            for k, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(k)
        if sm:
            out.update(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(mx)),
                       reasons=sorted(reasons), samples=len(sm))
        return out


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        return dist, int(os.environ["RANK"]), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def max_over_ranks(dist, v, device):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _pairs_parallel(O, tgt, src, qs, exclude, threads):
    """The oracle's direct sum, its targets split over a thread pool (NumPy
    releases the interpreter lock inside its array operations)."""
    from concurrent.futures import ThreadPoolExecutor
    n = len(tgt)
    parts = [p for p in np.array_split(np.arange(n), max(1, min(n, 4 * threads))) if len(p)]
    phi = np.zeros(n)
    grad = np.zeros((n, 3))

    def one(ix):
        ex = None if exclude is None else exclude[ix]
        return ix, O.pair_field(tgt[ix], src, qs, exclude=ex)

    with ThreadPoolExecutor(threads) as pool:
        for ix, (p, g) in pool.map(one, parts):
            phi[ix] = p
            grad[ix] = g
    return phi, grad


def oracle_sample(c, x, q, n_targets, seed=99, n_check=None, st=None, threads=None):
    """Time the oracle on a bounded sample; return (s per full eval, details).

    The near set, fit and surface map run in full; the near + far sums run on
    n_targets sampled ions and are scaled by N / n_targets.  With n_check, the
    check-point sums also run on a sample (timing only) and are scaled.  The
    pair sums are split over ``threads`` host threads by target.
    """
    from oracle import hsma as O
    threads = threads or host_cores()
    t0 = time.perf_counter()
    if st is None:
        st = O.make_setup(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], lam=c.lam,
                          dtn_grid=c.dtn_grid)
    t_setup = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(c.N, n_targets, replace=False))
    t1 = time.perf_counter()
    xc, qc = O.prepare_inputs(st, x, q)
    ipos, iq, isrc, isid = O.near_set(st, xc, qc)
    nc = len(st.check_pts)
    if n_check is None or n_check >= nc:
        cphi, cgrad = _pairs_parallel(O, st.check_pts, ipos, iq, None, threads)
        t_chk = 0.0
    else:
        ci = np.sort(rng.choice(nc, n_check, replace=False))
        tc = time.perf_counter()
        sphi, sgrad = _pairs_parallel(O, st.check_pts[ci], ipos, iq, None, threads)
        t_chk = (time.perf_counter() - tc) * (nc / n_check - 1.0)
        cphi = np.zeros(nc); cgrad = np.zeros((nc, 3))
        cphi[ci] = sphi; cgrad[ci] = sgrad
    A = st.P @ O.check_raw(st, cphi, cgrad)
    Q = st.W @ A
    t2 = time.perf_counter()
    s0 = O.self_shift(st)
    self_idx = np.full(c.N, -1)
    m0 = isid == s0
    self_idx[isrc[m0]] = np.nonzero(m0)[0]
    nphi, ngrad = _pairs_parallel(O, xc[idx], ipos, iq, self_idx[idx], threads)
    fphi, fgrad = _pairs_parallel(O, xc[idx], st.ysurf, Q, None, threads)
    t3 = time.perf_counter()
    t_full = (t2 - t1 + t_chk) + (t3 - t2) * c.N / n_targets
    F = -qc[idx, None] * (ngrad + fgrad)
    return t_full, dict(idx=idx, F=F, phi=nphi + fphi, t_setup=t_setup, t_fixed=t2 - t1,
                        t_targets=t3 - t2, t_wall=t3 - t1, Ns=len(iq), threads=threads)


def serve_bench(P, n_req=512, slots=16, budget=40e9, seed=4, n_sample=32, log=None, precision=1, **server_opts):
    """Served workload: independent HSMA3D requests, Poisson arrivals.

    Requests: neutral +-1 electrolytes at density 0.1, N log-uniform in
    [1000, 50000] (even), p in {6, 8, 10}, M = 4 p^2 + 400.  The arrival rate
    is 0.8 x the one-at-a-time FP32 capacity measured here on a sample of the
    same requests.  Reports served evals/s, p50/p99 latency (completion -
    arrival, host clock; after one untimed pass over the stream, so that the
    slot buffers are at their steady sizes) and the one-at-a-time FP64 and FP32 forms on a
    stratified sample, extrapolated to the whole stream; then the served
    capacity, with all requests submitted at once (the median of three such
    passes, after one that lets the slot buffers grow to their steady sizes).
    """
    shapes = workloads.serving_stream(n_req, seed=seed)
    reqs = []
    for r in shapes:
        c = workloads.small_case(r["N"], dims=3, box=r["box"], p=r["p"], M=r["M"], seed=r["seed"])
        x, q = workloads.electrolyte(c)
        reqs.append((c, x, q))
    order = np.argsort([c.N for c, _, _ in reqs])
    sample = order[np.linspace(0, n_req - 1, n_sample).astype(int)]

    geo = {}    # sampled request -> (images in B, check points)

    def one_at_a_time(prec, idx):
        res = {}
        for i in idx:
            c, x, q = reqs[i]
            h = P.HSMA(c.box, 3, c.p, c.M, precision=prec)
            h.eval(x, q)                       # set-up + warm-up, untimed
            t0 = time.perf_counter()
            E, F, _ = h.eval(x, q)
            res[i] = (time.perf_counter() - t0, E, F)
            geo[i] = (P.hsma_get_info(h.h, "Ns"), P.hsma_get_info(h.h, "n_check"))
            h.close()
        return res

    r32 = one_at_a_time(precision, sample)
    r64 = one_at_a_time(0, sample)
    # the stream's pair work: every request has the same density and sphere
    # scale, so its images in B are N times the sampled ratio N_s / N; its
    # check points depend on p only
    ns_ratio = float(np.mean([geo[i][0] / reqs[i][0].N for i in sample]))
    n_check = {reqs[i][0].p: geo[i][1] for i in sample}
    stream_pairs = sum((c.N + n_check[c.p]) * ns_ratio * c.N + c.M * c.N for c, _, _ in reqs)
    # the sample is stratified by N: scale its mean to the whole stream
    t32 = np.mean([r32[i][0] for i in sample])
    t64 = np.mean([r64[i][0] for i in sample])
    rate = 0.8 / t32
    arrivals = workloads.poisson_arrivals(n_req, rate, seed=seed)

    server = P.hsma_server_create(slots, budget, precision)
    for k, v in server_opts.items():
        P.hsma_set_option(server, k, v)
    for p in (6, 8, 10):                       # build the three unit geometries, untimed
        c, x, q = next(r for r in reqs if r[0].p == p)
        t = P.hsma_submit(server, x, q, c.box, c.p, c.M)
        while P.hsma_poll(server, t, c.N) is None:
            pass
    tickets = [None] * n_req
    done_t = np.zeros(n_req)
    out = [None] * n_req
    fbuf = [np.empty((c.N, 3)) for c, _, _ in reqs]      # result buffers, allocated once
    # one untimed pass over the stream first, so that the slots' device and
    # pinned buffers have grown to their steady sizes (a server that has been
    # running), as for the saturated measurement below
    warm = [P.hsma_submit(server, x, q, c.box, c.p, c.M) for c, x, q in reqs]
    for i in range(n_req):
        while P.hsma_poll(server, warm[i], reqs[i][0].N, out=fbuf[i]) is None:
            pass
    nxt = 0
    pending = set()
    t_start = time.perf_counter()
    while nxt < n_req or pending:
        now = time.perf_counter() - t_start
        while nxt < n_req and arrivals[nxt] <= now:
            c, x, q = reqs[nxt]
            tickets[nxt] = P.hsma_submit(server, x, q, c.box, c.p, c.M)
            pending.add(nxt)
            nxt += 1
        for i in list(pending):
            r = P.hsma_poll(server, tickets[i], reqs[i][0].N, out=fbuf[i])
            if r is not None:
                done_t[i] = time.perf_counter() - t_start
                out[i] = r
                pending.discard(i)
        if not pending and nxt < n_req:
            time.sleep(max(0.0, min(0.001, arrivals[nxt] - (time.perf_counter() - t_start))))
    P.hsma_destroy(server)
    lat = (done_t - arrivals) * 1e3
    span = done_t.max() - arrivals[0]

    # served capacity: the same requests all submitted at once (saturated queue)
    server = P.hsma_server_create(slots, budget, precision)
    for k, v in server_opts.items():
        P.hsma_set_option(server, k, v)
    for p in (6, 8, 10):                       # unit geometries, untimed
        c, x, q = next(r for r in reqs if r[0].p == p)
        t = P.hsma_submit(server, x, q, c.box, c.p, c.M)
        while P.hsma_poll(server, t, c.N) is None:
            pass
    # four passes over the stream: the first lets the slots' buffers grow to
    # their steady-state sizes (as the one-at-a-time handles are warmed up),
    # the other three are timed and the median pass is reported (one pass is
    # under a second); results are collected in submission order, and each
    # poll also advances the server
    passes = []
    for rep in range(4):
        g0 = P.hsma_get_info(server, "gpu_ms")
        t_sat = time.perf_counter()
        sat_tickets = [P.hsma_submit(server, x, q, c.box, c.p, c.M) for c, x, q in reqs]
        for i in range(n_req):
            while P.hsma_poll(server, sat_tickets[i], reqs[i][0].N, out=fbuf[i]) is None:
                pass
        if rep > 0:
            passes.append((time.perf_counter() - t_sat, (P.hsma_get_info(server, "gpu_ms") - g0) / 1e3))
    P.hsma_destroy(server)
    sat_span, sat_gpu_s = sorted(passes)[len(passes) // 2]
    de = [abs(out[i][0] - r64[i][1]) / abs(r64[i][1]) for i in sample]
    # the same error against the energy scale 1/2 sum |q_i Phi_i| (|E| itself can
    # nearly cancel in a random neutral configuration)
    des = []
    for i in sample:
        c, x, q = reqs[i]
        h = P.HSMA(c.box, 3, c.p, c.M, precision=0)
        _, _, pot = h.eval(x, q, forces=False, potential=True)
        h.close()
        des.append(abs(out[i][0] - r64[i][1]) / (0.5 * float(np.sum(np.abs(q * pot)))))
    df = [math.sqrt(np.mean(np.sum((out[i][1] - r64[i][2]) ** 2, 1)) / np.mean(np.sum(r64[i][2] ** 2, 1)))
          for i in sample]
    return {"workload": f"{n_req} requests, N log-uniform [1e3, 5e4], p in {{6,8,10}}, M = 4p^2+400, "
                        f"rho = 0.1, Poisson arrivals at {rate:.1f}/s (0.8 x the one-at-a-time capacity "
                        f"at precision {precision})",
            "precision": precision, "slots": slots, "budget_bytes": budget, "server_options": server_opts,
            "evals_per_s": n_req / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_N": float(np.mean([c.N for c, _, _ in reqs])),
            "one_at_a_time_fp64_evals_per_s": 1.0 / t64, "one_at_a_time_evals_per_s": 1.0 / t32,
            "served_vs_fp64": (n_req / span) * t64,
            "saturated_evals_per_s": n_req / sat_span,
            "saturated_batch_device_s": sat_gpu_s, "saturated_wall_s": sat_span,
            "stream_pairs": stream_pairs,
            "saturated_pair_ints_per_s": stream_pairs / sat_span,
            "saturated_vs_one_at_a_time": (n_req / sat_span) * t32,
            "saturated_vs_fp64": (n_req / sat_span) * t64,
            "sample": f"{n_sample} requests stratified by N, timed one at a time",
            "max_rel_energy_err_vs_fp64": float(max(de)),
            "median_rel_energy_err_vs_fp64": float(np.median(de)),
            "max_energy_err_over_energy_scale": float(max(des)),
            "max_rel_force_rms_vs_fp64": float(max(df))}


def other_cases(P, torch, dev, stream, peak_instr):
    """Evaluations/s of the other workload shapes (inputs resident in HBM),
    FP32 and FP64 paths, with the FP32 energy error against the FP64 path."""
    out = {}
    cases = [(workloads.case(1), 20, 5), (workloads.case(3, -0.95), 20, 3),
             (workloads.case(3, 0.0), 20, 3), (workloads.case(3, 0.95), 20, 3),
             (workloads.case(2), 5, 1), (workloads.case(5), 3, 0)]
    for c, n32, n64 in cases:
        x, q = workloads.electrolyte(c)
        xd = torch.from_numpy(x).to(dev)
        qd = torch.from_numpy(q).to(dev)
        fd = torch.empty((c.N, 3), dtype=torch.float64, device=dev)
        rec = {"N": c.N, "p": c.p, "M": c.M}
        energies = {}
        for prec, n in ((1, n32), (0, n64)):
            if n == 0:
                continue
            h = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=prec,
                       dtn_grid=c.dtn_grid)
            P.hsma_set_stream(h.h, stream.cuda_stream)
            e = np.zeros(1)
            for _ in range(2):
                P.hsma_eval_into(h.h, xd, qd, c.N, e, fd)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(n):
                P.hsma_eval_into(h.h, xd, qd, c.N, e, fd)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / n
            key = "fp32" if prec else "fp64"
            rec[key + "_evals_per_s"] = 1e3 / ms
            if prec:
                Ns = int(P.hsma_get_info(h.h, "Ns"))
                nck = int(P.hsma_get_info(h.h, "n_check"))
                rec["N_s"] = Ns
                rec["pairs_per_eval"] = (c.N + nck) * Ns + c.N * c.M
                rec["fp32_pair_ints_per_s"] = rec["pairs_per_eval"] * 1e3 / ms
            energies[prec] = float(e[0])
            h.close()
        if 0 in energies:
            rec["fp32_vs_fp64_rel_energy"] = abs(energies[1] - energies[0]) / abs(energies[0])
        if c.dims == 2 or c.N >= 100000:
            # the tree evaluation of the near field (option near_tree) beside it
            h = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=1, near_tree=1,
                       dtn_grid=c.dtn_grid)
            P.hsma_set_stream(h.h, stream.cuda_stream)
            e = np.zeros(1)
            ft = torch.empty_like(fd)
            P.hsma_eval_into(h.h, xd, qd, c.N, e, ft)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(max(3, n32)):
                P.hsma_eval_into(h.h, xd, qd, c.N, e, ft)
            b.record(stream)
            torch.cuda.synchronize()
            rec["tree_fp32_evals_per_s"] = 1e3 * max(3, n32) / a.elapsed_time(b)
            # the tree's own near stage, timed per phase, and its roofline
            ht = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=1, near_tree=1,
                        timing=1, dtn_grid=c.dtn_grid)
            P.hsma_set_stream(ht.h, stream.cuda_stream)
            et = np.zeros(1)
            f2 = torch.empty_like(fd)
            tn = []
            for _ in range(4):
                P.hsma_eval_into(ht.h, xd, qd, c.N, et, f2)
                torch.cuda.synchronize()
                tn.append(P.hsma_get_info(ht.h, "t_near_ms"))
            rec["tree_roofline"] = tree_roofline(P, ht, xd, qd, c.N, et, f2, float(np.median(tn[1:])), 10,
                                                 peak_instr)
            ht.close()
            rec["tree_levels"] = int(P.hsma_get_info(h.h, "tree_levels"))
            rec["tree_direct_leaf"] = int(P.hsma_get_info(h.h, "tree_direct_leaf"))
            rec["tree_vs_dense_rel_energy"] = abs(float(e[0]) - energies[1]) / abs(energies[1])
            # fd holds the forces of the last dense run (FP64 where it ran, else FP32)
            ref = "fp64" if 0 in energies else "fp32"
            rec["tree_vs_" + ref + "_rel_force_rms"] = float(
                torch.sqrt(((ft - fd) ** 2).sum(1).mean() / (fd ** 2).sum(1).mean()).item())
            h.close()
        out[c.name] = rec
    return out


def far_series_compare(P, torch, stream, c, xd, qd, fd, h_surface, n=10):
    """The main workload with the far field taken from the fitted series
    (far_field = 1) instead of the M surface charges: evaluations/s, the far
    stage's time in both forms and their energy / force difference."""
    N = c.N
    h = P.HSMA(c.box, c.dims, c.p, c.M, precision=1, timing=1, far_field=1)
    P.hsma_set_stream(h.h, stream.cuda_stream)
    e = np.zeros(1)
    f = torch.empty_like(fd)
    for _ in range(2):
        P.hsma_eval_into(h.h, xd, qd, N, e, f)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    far_ms = []
    a.record(stream)
    for _ in range(n):
        P.hsma_eval_into(h.h, xd, qd, N, e, f)
        far_ms.append(P.hsma_get_info(h.h, "t_far_ms"))
    b.record(stream)
    torch.cuda.synchronize()
    e0 = np.zeros(1)
    P.hsma_eval_into(h_surface.h, xd, qd, N, e0, fd)
    torch.cuda.synchronize()
    rec = {"evals_per_s": 1e3 * n / a.elapsed_time(b), "far_ms_series": float(np.mean(far_ms)),
           "far_ms_surface": P.hsma_get_info(h_surface.h, "t_far_ms"),
           "rel_energy_vs_surface": abs(float(e[0]) - float(e0[0])) / abs(float(e0[0])),
           "rel_force_rms_vs_surface": float(torch.sqrt(((f - fd) ** 2).sum() / (fd ** 2).sum()))}
    h.close()
    return rec


def pair_sources_sha1():
    """Hash of the pair kernels' sources: pair.cu and the two structs of
    internal.hpp they read (PairArgs, DevScalars).  A stored DRAM-traffic
    figure is used only while this matches the one it was captured with."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2104_05260_gb300", "csrc")
    hdr = open(os.path.join(csrc, "internal.hpp")).read()
    blocks = [m.group(0) for m in re.finditer(r"struct (PairArgs|DevScalars) \{.*?\n\};", hdr, re.S)]
    src = open(os.path.join(csrc, "pair.cu"), "rb").read() + "".join(blocks).encode()
    return hashlib.sha1(src).hexdigest()


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")


def traffic_records(tr=TRAFFIC_JSON):
    """The DRAM-traffic records of profiles/traffic.json, one per captured
    (kernel, source chunks) launch plan."""
    if not os.path.exists(tr):
        return []
    d = json.load(open(tr))
    return d.get("records", [d] if "bytes_per_launch" in d else [])


def record_traffic(csv_path, kernel, workload, chunks, command, tr=TRAFFIC_JSON):
    """Add to profiles/traffic.json the DRAM bytes of the near-field launch in
    an ncu CSV (--csv --log-file) holding gpu__time_duration.sum,
    dram__bytes_read.sum and dram__bytes_write.sum: of the captured launches
    the longest one, which is the near-field and check-point sum (the far
    field's launch of the same kernel takes about 1/200 of its time)."""
    import csv
    rows = [r for r in csv.reader(open(csv_path)) if len(r) > 10]
    h = rows[0]
    launches = {}
    for r in rows[1:]:
        name, unit, v = r[h.index("Metric Name")], r[h.index("Metric Unit")], r[h.index("Metric Value")]
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9,
                 "ns": 1e-9, "us": 1e-6, "ms": 1e-3, "s": 1,
                 "nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "second": 1}.get(unit)
        if scale is not None:
            launches.setdefault(r[h.index("ID")], {})[name] = float(v.replace(",", "")) * scale
    vals = max(launches.values(), key=lambda m: m.get("gpu__time_duration.sum", 0.0))
    rd, wr = vals["dram__bytes_read.sum"], vals["dram__bytes_write.sum"]
    rec = {"kernel": kernel, "workload": workload, "pair_sources_sha1": pair_sources_sha1(), "chunks": chunks,
           "bytes_per_launch": int(rd + wr), "read_bytes": int(rd), "write_bytes": int(wr),
           "command": command}
    recs = [r for r in traffic_records(tr) if not (r.get("kernel") == kernel and r.get("chunks") == chunks)]
    recs.append(rec)
    recs.sort(key=lambda r: (r.get("kernel", ""), r.get("chunks", 0)))
    out = {"hash_covers": "paper_2104_05260_gb300/csrc/pair.cu and the PairArgs and DevScalars structs of "
                          "internal.hpp; a record whose pair_sources_sha1 differs is not used by bench.py",
           "records": recs}
    with open(tr, "w") as f:
        json.dump(out, f, indent=1)
    return rec


def option_variant(P, torch, stream, c, xd, qd, fd, e_default, n=3, **opt):
    """The main workload with one option changed: evaluations/s, N_s and the
    energy / force difference from the default configuration (fd, e_default)."""
    h = P.HSMA(c.box, c.dims, c.p, c.M, precision=1, **opt)
    P.hsma_set_stream(h.h, stream.cuda_stream)
    e = np.zeros(1)
    f = torch.empty_like(fd)
    P.hsma_eval_into(h.h, xd, qd, c.N, e, f)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n):
        P.hsma_eval_into(h.h, xd, qd, c.N, e, f)
    b.record(stream)
    torch.cuda.synchronize()
    rec = {"options": opt, "evals_per_s": 1e3 * n / a.elapsed_time(b), "N_s": int(P.hsma_get_info(h.h, "Ns")),
           "rel_energy_vs_default": abs(float(e[0]) - e_default) / abs(e_default),
           "rel_force_rms_vs_default": float(torch.sqrt(((f - fd) ** 2).sum() / (fd ** 2).sum()))}
    h.close()
    return rec


def paper_like(P, torch, dev, stream, n32=5):
    """The main workload shape with ions kept >= 0.8 apart (the soft cores of
    the paper's LJ electrolytes): FP32 evaluations/s and the FP32-vs-FP64
    energy and force errors, which close pairs dominate in the uniform case."""
    c = workloads.case(2)
    x, q = workloads.electrolyte(c, min_dist=0.8)
    xd = torch.from_numpy(x).to(dev)
    qd = torch.from_numpy(q).to(dev)
    out = {"workload": c.name + "_mindist0.8", "N": c.N}
    res = {}
    for prec, n in ((1, n32), (0, 1)):
        h = P.HSMA(c.box, 3, c.p, c.M, precision=prec, autotune=1 if prec else 0)
        P.hsma_set_stream(h.h, stream.cuda_stream)
        e = np.zeros(1)
        f = torch.empty((c.N, 3), dtype=torch.float64, device=dev)
        P.hsma_eval_into(h.h, xd, qd, c.N, e, f)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            P.hsma_eval_into(h.h, xd, qd, c.N, e, f)
        b.record(stream)
        torch.cuda.synchronize()
        out[("fp32" if prec else "fp64") + "_evals_per_s"] = 1e3 * n / a.elapsed_time(b)
        res[prec] = (float(e[0]), f)
        h.close()
    (e32, f32), (e64, f64) = res[1], res[0]
    out["fp32_vs_fp64_rel_energy"] = abs(e32 - e64) / abs(e64)
    out["fp32_vs_fp64_rel_force_rms"] = float(torch.sqrt(((f32 - f64) ** 2).sum() / (f64 ** 2).sum()))
    return out


PAPER_E1 = {"monovalent": (0.3561, 1.2132e-3), "divalent": (-1.4840, 2.3875e-3),
            "trivalent": (-3.2741, 3.8337e-3)}     # Sec. 4.1, table: HSMA3D mean, variance


def md_e1(P, valence=1, steps_eq=20000, steps_prod=200000, rdf_every=100, seed=11, tdamp=0.01):
    """The primitive electrolyte of Sec. 4.1 under the library's MD loop:
    L = 25 sigma, 3000 ions (valence z:1, so 1500/1000/750 cations), WCA
    soft spheres with eps = kT, Bjerrum length 3.5 sigma, dt = 0.01 tau,
    Nose-Hoover with damping time 0.01 tau.  Electrostatics: HSMA3D with
    p = 10, N_m = 200 (the paper's parameter line), M = 2000, the unmasked
    near set (force error 3e-6 against Ewald at p = 10), FP32 pairs.
    Start: hard-core random positions 1.0 sigma apart, Maxwell velocities.
    Reports the total energy per ion (mean, variance; block standard error
    of the mean over 20 blocks) beside the paper's, the cation-anion g(r)
    peak and steps/s."""
    L, N = 25.0, 3000
    n_cat = {1: 1500, 2: 1000, 3: 750}[valence]
    c = workloads.Case(f"e1_z{valence}", 3, (L, L, L), {valence: n_cat, -1: N - n_cat}, p=10, M=2000,
                       lam=1.3, seed=seed)
    x, q = workloads.electrolyte(c, min_dist=1.0)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    v = rng.normal(0.0, 1.0, (N, 3))
    v -= v.mean(axis=0)
    h = P.HSMA(c.box, 3, 10, 2000, precision=1, coulomb_prefactor=3.5, n_monitor=200, sphere_mask=0)
    md = P.MD(h, x, v, q, mass=1.0, dt=0.01, kT=1.0, tdamp=tdamp, lj_sigma=1.0, lj_eps=1.0)
    t0 = time.perf_counter()
    md.run(steps_eq)
    t_eq = time.perf_counter() - t0
    bins, rmax = 100, 5.0
    md.set_option("rdf_bins", bins)
    md.set_option("rdf_rmax", rmax)
    md.set_option("rdf_every", rdf_every)
    t0 = time.perf_counter()
    th = md.run(steps_prod)
    t_prod = time.perf_counter() - t0
    e = (th[:, 0] + th[:, 1] + th[:, 2]) / N
    blocks = np.array_split(e, 20)
    sem = float(np.std([b.mean() for b in blocks], ddof=1) / math.sqrt(len(blocks)))
    counts = md.get("rdf").reshape(3, bins)
    samples = md.get("state")[4]
    r = (np.arange(bins) + 0.5) * (rmax / bins)
    shell = 4.0 / 3.0 * math.pi * ((r + rmax / bins / 2) ** 3 - (r - rmax / bins / 2) ** 3)
    n_a = int(np.sum(q < 0))
    g_ca = counts[0] / (samples * n_cat * n_a / L ** 3 * shell)
    k = int(np.argmax(g_ca))
    T = 2 * th[:, 0] / (3 * N - 3)
    name = {1: "monovalent", 2: "divalent", 3: "trivalent"}[valence]
    # mean-spherical approximation of the primitive model with equal diameters
    # sigma = 1: 2 Gamma (1 + Gamma) = kappa, U / N = -l_B Gamma / (1 + Gamma) <z^2>
    z2 = float(np.mean(q * q))
    kappa = math.sqrt(4.0 * math.pi * 3.5 * z2 * N / L ** 3)
    gam = (-1.0 + math.sqrt(1.0 + 2.0 * kappa)) / 2.0
    msa = -3.5 * gam / (1.0 + gam) * z2
    md.close()
    h.close()
    return {"system": f"Sec. 4.1 {name} electrolyte, N = {N}, L = {L}, l_B = 3.5, dt = 0.01, "
                      f"tdamp = {tdamp}, {steps_eq} + {steps_prod} steps",
            "steps_per_s": (steps_eq + steps_prod) / (t_eq + t_prod),
            # the production run alone (set-up, tuning and graph capture fall
            # in the equilibration run)
            "production_steps_per_s": steps_prod / t_prod,
            "energy_per_ion_mean": float(e.mean()), "energy_per_ion_var": float(e.var()),
            "energy_per_ion_sem": sem, "paper_hsma3d_mean_var": PAPER_E1[name],
            "temperature_mean": float(T.mean()),
            "kinetic_per_ion_var": float(np.var(th[:, 0] / N)),
            "potential_per_ion_var": float(np.var((th[:, 1] + th[:, 2]) / N)),
            "kinetic_potential_cov": float(np.cov(th[:, 0] / N, (th[:, 1] + th[:, 2]) / N)[0, 1]),
            "canonical_kinetic_per_ion_var": 0.5 * (3 * N - 3) / N ** 2,
            "coulomb_per_ion_mean": float(th[:, 2].mean() / N), "coulomb_per_ion_msa": msa,
            "lj_per_ion_mean": float(th[:, 1].mean() / N),
            "g_ca_peak": [float(r[k]), float(g_ca[k])], "rdf_samples": int(samples),
            "g_ca": [round(float(v), 4) for v in g_ca]}


def md_e3(P, valence=1, steps_eq=20000, steps_prod=200000, every=100, seed=13, bins=50):
    """The confined electrolyte of Sec. 4.3 under the library's MD loop:
    Lx = Ly = 100 sigma, Lz = 50 sigma, 218 anions and 218 (1:1) or 109 (2:1)
    cations, WCA ions, LJ walls (eps kT, sigma 0.5) at the two interfaces,
    gamma = 0.939 on both sides, Bjerrum length 3.5 sigma, dt = 0.005 tau,
    Nose-Hoover with damping time 0.05 tau.  HSMA2D with lambda 1.6, p = 6
    (the paper's parameter line), M = 600, G = 80, FP32 pairs.  Reports the
    ion density across the slab (cations, anions, relative to the mean) and
    the depletion next to the walls that the repulsive images cause."""
    Lx, Lz = 100.0, 50.0
    n_cat = {1: 218, 2: 109}[valence]
    c = workloads.Case(f"e3_z{valence}", 2, (Lx, Lx, Lz), {valence: n_cat, -1: 218}, p=6, M=600, lam=1.6,
                       gammas=(0.939, 0.939), dtn_grid=80, seed=seed)
    x, q = workloads.electrolyte(c, min_dist=1.0, margin=1.0)
    N = len(q)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    v = rng.normal(0.0, 1.0, (N, 3))
    v -= v.mean(axis=0)
    h = P.HSMA(c.box, 2, 6, 600, 0.939, 0.939, precision=1, coulomb_prefactor=3.5, dtn_grid=80)
    md = P.MD(h, x, v, q, mass=1.0, dt=0.005, kT=1.0, tdamp=0.05, lj_sigma=1.0, lj_eps=1.0)
    t0 = time.perf_counter()
    md.run(steps_eq)
    md.set_option("zhist_bins", bins)
    md.set_option("rdf_every", every)
    th = md.run(steps_prod)
    dt_run = time.perf_counter() - t0
    zh = md.get("zhist").reshape(2, bins)
    samples = md.get("state")[4]
    prof = zh / (samples * np.array([[n_cat], [218]]) / bins)    # density relative to the mean
    edge = max(1, bins // 25)                                     # the outer 2 sigma on each side
    mid = slice(bins // 2 - 5, bins // 2 + 5)
    md.close()
    h.close()
    return {"system": f"Sec. 4.3 {'1:1' if valence == 1 else '2:1'} electrolyte between interfaces, gamma 0.939, "
                      f"{Lx:g} x {Lx:g} x {Lz:g}, N = {N}, {steps_eq} + {steps_prod} steps",
            "steps_per_s": (steps_eq + steps_prod) / dt_run,
            "temperature_mean": float(np.mean(2 * th[:, 0] / (3 * N - 3))),
            "cation_near_wall_over_middle": float(np.concatenate([prof[0, :edge], prof[0, -edge:]]).mean()
                                                  / prof[0, mid].mean()),
            "anion_near_wall_over_middle": float(np.concatenate([prof[1, :edge], prof[1, -edge:]]).mean()
                                                 / prof[1, mid].mean()),
            "z_bin_width": Lz / bins, "samples": int(samples),
            "cation_profile": [round(float(v), 3) for v in prof[0]],
            "anion_profile": [round(float(v), 3) for v in prof[1]]}


def workload_config(c, ws=1):
    """The workload's config, the same for both arms."""
    return {"workload": c.name, "N": c.N, "p": c.p, "M": c.M, "lambda": c.lam,
            "box": [round(v, 6) for v in c.box], "parallelism": f"replicas x{ws}"}


def run_reference(args, c, rank, dist, ws):
    if rank != 0:
        return
    from oracle import hsma as O
    x, q = workloads.electrolyte(c)
    st = O.make_setup(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], lam=c.lam,
                      dtn_grid=c.dtn_grid)
    threads = host_cores()
    n_t, n_c = min(128, c.N), 64
    for _ in range(args.warmup):
        oracle_sample(c, x, q, n_t, n_check=n_c, st=st, threads=threads)
    t_eval, t_wall = [], []
    for k in range(args.steps):
        t, d = oracle_sample(c, x, q, n_t, seed=100 + k, n_check=n_c, st=st, threads=threads)
        t_eval.append(t)
        t_wall.append(d["t_wall"])
    # each step computes part of an evaluation: the near set, the fit and the
    # surface map in full, the pair sums of a sample; evals_per_step is that
    # part's share of one evaluation's (scaled) time
    v = 1.0 / float(np.mean(t_eval))
    ms_step = 1e3 * float(np.mean(t_wall))
    sample = (f"per step: near set, fit and surface map in full; check-point sums on {n_c} "
              f"sampled check points and near+far sums on {n_t} sampled ions, each scaled to "
              f"the full count; pair sums split by target over {threads} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "evals_per_step": v * ms_step / 1e3,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(c, ws),
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "cpu": platform.processor() or platform.machine()},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


KERNEL_NAMES = {12: "k_pair_f32x2<1>", 14: "k_pair_f32x2<2>", 24: "k_pair_f32x2s<2>", 1: "k_pair_f32<1>",
                2: "k_pair_f32<2>", 4: "k_pair_f32<4>", 32: "k_pair_f32x2x<1>", 34: "k_pair_f32x2x<2>",
                44: "k_pair_f32x2xs<2>"}


def pair_roofline(P, h, c, pairs_near, near_ms, peak_instr, mhz_src, sms, lib_total_ms=None):
    """FP32 issue-rate roofline of the near-field + check-point launch."""
    plan = {"kernel": KERNEL_NAMES.get(int(P.hsma_get_info(h.h, "kernel")), "k_pair_f32"),
            "chunks": int(P.hsma_get_info(h.h, "chunks")), "grid": int(P.hsma_get_info(h.h, "grid")),
            "tile_targets": int(P.hsma_get_info(h.h, "tile_targets"))}
    t_near = near_ms / 1e3
    achieved = pairs_near * FP32_INSTR_PER_PAIR / t_near / 1e12
    roof = {"bound": "alu", "kernel": plan["kernel"] + " (near field + check points)",
            "achieved": achieved, "peak": peak_instr, "unit": "T FP32-pipe instr/s",
            "frac": achieved / peak_instr, "traffic": None,
            "algorithmic": f"{FP32_INSTR_PER_PAIR} FP32-pipe instructions per pair x {pairs_near} pairs "
                           f"(targets x images in B) per launch",
            "flops_view": {"achieved_tflops": pairs_near * FLOP_PER_PAIR / t_near / 1e12,
                           "peak_tflops": 2 * peak_instr,
                           "frac": (pairs_near * FLOP_PER_PAIR / t_near / 1e12) / (2 * peak_instr)},
            "peak_source": f"{sms} SMs x {FP32_LANES} FP32 lanes x {mhz_src}",
            "near_ms": near_ms}
    if lib_total_ms is not None:
        roof["lib_total_ms"] = lib_total_ms
    try:
        sha = pair_sources_sha1()
        for rec in traffic_records():
            if (rec.get("pair_sources_sha1") == sha and rec.get("chunks") == plan["chunks"]
                    and rec.get("workload") == c.name and rec.get("kernel", "").startswith(plan["kernel"])):
                roof["traffic"] = rec.get("bytes_per_launch")
                roof["traffic_workload"] = rec.get("workload")
    except Exception:
        pass
    return roof, plan


M2P_OPS_PER_TERM = 17     # FP32 operations per (n, m >= 0) term of a multipole evaluation (M2P)


def tree_roofline(P, h, xd, qd, N, e, f, near_ms, order, peak_instr):
    """FP32 issue-rate roofline of the tree evaluation of the near field and
    check points: one extra evaluation with the counting kernel gives the
    multipole evaluations (M2P) at each order and the FP32 direct pairs it
    performs; the algorithmic work is (M2P x (P+1)(P+2)/2 + far-cell M2P x
    (P-3)(P-2)/2) terms x 17 + pairs x 13 FP32 operations (far cells are
    evaluated to order P - 4), over the evaluation kernel's CUDA-event time (h must have
    option timing = 1); the whole near stage (binning and multipoles too) is
    given beside it."""
    import torch
    # the evaluation kernel alone (CUDA events around it; option timing = 1)
    t_eval = []
    for _ in range(3):
        P.hsma_eval_into(h.h, xd, qd, N, e, f)
        torch.cuda.synchronize()
        t_eval.append(P.hsma_get_info(h.h, "t_tree_eval_ms"))
    eval_ms = float(np.median(t_eval))
    P.hsma_set_option(h.h, "tree_count", 1)
    P.hsma_eval_into(h.h, xd, qd, N, e, f)
    torch.cuda.synchronize()
    m2p = P.hsma_get_info(h.h, "tree_m2p")
    m2p_low = P.hsma_get_info(h.h, "tree_m2p_low")
    direct = P.hsma_get_info(h.h, "tree_direct_pairs")
    P.hsma_set_option(h.h, "tree_count", 0)
    terms = (order + 1) * (order + 2) // 2
    low = order - 4 if order >= 8 else order
    terms_low = (low + 1) * (low + 2) // 2
    ops = (m2p * terms + m2p_low * terms_low) * M2P_OPS_PER_TERM + direct * FP32_INSTR_PER_PAIR
    achieved = ops / (eval_ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": f"k_tree_eval<{order}> (near field + check points)",
            "achieved": achieved, "peak": peak_instr, "unit": "T FP32-pipe instr/s", "frac": achieved / peak_instr,
            "traffic": None, "m2p_per_eval": m2p, "m2p_low_order_per_eval": m2p_low,
            "direct_pairs_per_eval": direct,
            "algorithmic": f"(M2P x {terms} + far-cell M2P x {terms_low}) terms x {M2P_OPS_PER_TERM} + direct "
                           f"pairs x {FP32_INSTR_PER_PAIR} FP32 operations = {ops:.4g} per evaluation",
            "eval_kernel_ms": eval_ms, "near_stage_ms": near_ms,
            "near_stage_frac": ops / (near_ms / 1e3) / 1e12 / peak_instr}


def timed_evals(P, torch, stream, h, xd, qd, N, e, f, n):
    """Mean device time (ms) of n evaluations on the stream, inputs resident."""
    P.hsma_eval_into(h.h, xd, qd, N, e, f)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n):
        P.hsma_eval_into(h.h, xd, qd, N, e, f)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n


def secondary_case(P, torch, dev, stream, c, peak_instr, mhz_src, sms, steps=10):
    """Another dense workload at full size, inputs resident, L2 flushed between
    evaluations: evaluations/s, pair interactions/s and the near-field launch's
    FP32 roofline."""
    x, q = workloads.electrolyte(c)
    xd = torch.from_numpy(x).to(dev)
    qd = torch.from_numpy(q).to(dev)
    fd = torch.empty((c.N, 3), dtype=torch.float64, device=dev)
    e = np.zeros(1)
    h = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=1, timing=1, dtn_grid=c.dtn_grid)
    P.hsma_set_stream(h.h, stream.cuda_stream)
    for _ in range(3):
        P.hsma_eval_into(h.h, xd, qd, c.N, e, fd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    ms, near = [], []
    for i in range(steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        P.hsma_eval_into(h.h, xd, qd, c.N, e, fd)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        near.append(P.hsma_get_info(h.h, "t_near_ms"))
    Ns = int(P.hsma_get_info(h.h, "Ns"))
    nck = int(P.hsma_get_info(h.h, "n_check"))
    pairs_near = (c.N + nck) * Ns
    pairs = pairs_near + c.N * c.M
    roof, plan = pair_roofline(P, h, c, pairs_near, float(np.mean(near)), peak_instr, mhz_src, sms)
    h.close()
    t = float(np.mean(ms)) / 1e3
    return {"workload": c.name, "N": c.N, "p": c.p, "M": c.M, "evals_per_s": 1.0 / t, "ms_per_eval": 1e3 * t,
            "N_s": Ns, "n_check": nck, "pairs_per_eval": pairs, "pair_ints_per_s": pairs / t,
            "plan": plan, "roofline": roof}


def paper_accuracy(P, torch, dev, stream):
    """Throughput at the accuracy the paper times at (relative force error
    about 1e-5 against the exact sum, Sec. 3.2 and Sec. 5): the unmasked
    27-cell near set at p = 10 (reading R12), dense and tree, at N = 100,000.
    The method's error at the same parameters is measured here against Ewald
    on the N = 1000 system (FP32 pairs, through the library)."""
    from oracle.ewald import ewald3d
    opts = dict(sphere_mask=0, n_monitor=242)
    p, M = 10, 2000
    small = workloads.case(1)
    xs, qs = workloads.electrolyte(small)
    L = small.box[0]
    xc = (xs - L * np.floor(xs / L)) - 0.5 * L
    Ee, _, ge = ewald3d(xc, qs, small.box)
    Fe = -qs[:, None] * ge
    out = {"parameters": f"p = {p}, M = {M}, N_m = 242, lambda = 1.3, unmasked 27-cell near set (R12), FP32 pairs"}
    errs = {}
    for tree in (0, 1):
        h = P.HSMA(small.box, 3, p, M, precision=1, near_tree=tree, **opts)
        E, F, _ = h.eval(xs, qs)
        h.close()
        errs[tree] = (float(math.sqrt(np.mean(np.sum((F - Fe) ** 2, 1)) / np.mean(np.sum(Fe ** 2, 1)))),
                      abs(E - Ee) / abs(Ee))
    c = workloads.case(2)
    x, q = workloads.electrolyte(c)
    xd = torch.from_numpy(x).to(dev)
    qd = torch.from_numpy(q).to(dev)
    f = torch.empty((c.N, 3), dtype=torch.float64, device=dev)
    e = np.zeros(1)
    for tree, n in ((0, 3), (1, 10)):
        h = P.HSMA(c.box, 3, p, M, precision=1, near_tree=tree, **opts)
        P.hsma_set_stream(h.h, stream.cuda_stream)
        ms = timed_evals(P, torch, stream, h, xd, qd, c.N, e, f, n)
        key = "tree" if tree else "dense"
        out[key] = {"workload": f"hsma3d_n100000_rho0.1_p{p}_M{M}_unmasked", "evals_per_s": 1e3 / ms,
                    "N_s": int(P.hsma_get_info(h.h, "Ns")),
                    "rel_force_err_vs_ewald_n1000": errs[tree][0], "rel_energy_err_vs_ewald_n1000": errs[tree][1]}
        h.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-other-cases", action="store_true")
    ap.add_argument("--case", type=int, default=5,
                    help="workload case (default 5: N = 262,144, p = 10, M = 4000; 2: N = 100,000)")
    ap.add_argument("--clocks-log", default=None,
                    help="keep the nvidia-smi samples of the timed region in this CSV file")
    ap.add_argument("--record-traffic", default=None,
                    help="add to profiles/traffic.json the near-field launch of this ncu CSV, captured "
                         "with --targets-per-thread T --chunks K on --case C, and exit")
    ap.add_argument("--chunks", type=int, default=0,
                    help="source chunks of the near-field launch (0: the library's autotuner)")
    ap.add_argument("--targets-per-thread", type=int, default=0,
                    help="pair-kernel variant of the main handle (0: the autotuner; 24: k_pair_f32x2s<2>)")
    ap.add_argument("--md", type=int, default=0, choices=[0, 1, 2, 3],
                    help="run the Sec. 4.1 electrolyte MD validation with this valence and exit")
    ap.add_argument("--md-steps", type=int, default=200000, help="production steps of --md")
    ap.add_argument("--md-tdamp", type=float, default=0.01, help="thermostat damping time of --md")
    ap.add_argument("--md-eq", type=int, default=20000, help="equilibration steps of --md")
    ap.add_argument("--md-slab", type=int, default=0, choices=[0, 1, 2],
                    help="run the Sec. 4.3 confined-electrolyte MD with this cation valence and exit")
    ap.add_argument("--serve-only", type=int, default=0, metavar="N_REQ",
                    help="run only the served stream (precision 1) with this many requests and exit")
    ap.add_argument("--near-tree", type=int, default=0, choices=[0, 1],
                    help="1: tree evaluation of the near-field sums (option near_tree, order 10)")
    ap.add_argument("--far-field", type=int, default=0, choices=[0, 1],
                    help="0: surface charges (Eq. 8, default); 1: the fitted series (Eq. 5)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    c = workloads.case(args.case)
    if args.record_traffic:
        if not args.targets_per_thread or args.chunks < 1:
            raise SystemExit("--record-traffic needs --targets-per-thread T and --chunks K")
        k, tpt = args.chunks, args.targets_per_thread
        kname = KERNEL_NAMES[tpt]
        regex = kname.split("<")[0]
        print(json.dumps(record_traffic(
            args.record_traffic, kname + " near field + check points", c.name,
            k, "ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum "
               f"--clock-control none -k regex:{regex} -s 4 -c 2 --csv --log-file near_traffic.csv "
               f"python bench.py --case {args.case} --steps 2 --warmup 3 --no-cpu-baseline --fp64-steps 0 "
               f"--no-serve --no-other-cases --targets-per-thread {tpt} --chunks {k}")))
        return
    dist, rank, ws, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, c, rank, dist, ws)
        if dist:
            dist.barrier()
        return

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_05260_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    import paper_2104_05260_gb300 as P

    if args.md_slab:
        if rank == 0:
            print(json.dumps({"md_slab": md_e3(P, valence=args.md_slab, steps_eq=args.md_eq,
                                               steps_prod=args.md_steps)}), flush=True)
        if dist:
            dist.barrier()
        return
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"serve": serve_bench(P, n_req=args.serve_only)}), flush=True)
        if dist:
            dist.barrier()
        return
    if args.md:
        if rank == 0:
            print(json.dumps({"md_validation": md_e1(P, valence=args.md, steps_eq=args.md_eq,
                                                     steps_prod=args.md_steps, tdamp=args.md_tdamp)}),
                  flush=True)
        if dist:
            dist.barrier()
        return

    x, q = workloads.electrolyte(c, seed=c.seed + 1000 * rank)
    N = c.N
    h = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=1, timing=1,
               far_field=args.far_field, near_tree=args.near_tree, dtn_grid=c.dtn_grid)
    if args.targets_per_thread:
        h.set_option("targets_per_thread", args.targets_per_thread)
    if args.chunks:
        h.set_option("chunks", args.chunks)
    stream = torch.cuda.current_stream(dev)
    P.hsma_set_stream(h.h, stream.cuda_stream)
    xd = torch.from_numpy(x).to(dev)
    qd = torch.from_numpy(q).to(dev)
    fd = torch.empty((N, 3), dtype=torch.float64, device=dev)
    ebuf = np.zeros(1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        P.hsma_eval_into(h.h, xd, qd, N, ebuf, fd)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    near_ms, total_lib_ms = [], []
    with Clocks(local, args.clocks_log) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))              # evict L2 between steps (outside the events)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            near_ms.append(P.hsma_get_info(h.h, "t_near_ms"))
            total_lib_ms.append(P.hsma_get_info(h.h, "t_total_ms"))
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = float(np.sum([a.elapsed_time(b) for a, b in ev]))
    ms = max_over_ranks(dist, ms, dev)
    ms_step = ms / args.steps
    energy = float(ebuf[0])
    Ns = int(P.hsma_get_info(h.h, "Ns"))
    n_check = int(P.hsma_get_info(h.h, "n_check"))
    pairs_near = (N + n_check) * Ns
    pairs_far = 0 if args.far_field else N * c.M     # the series has no pair sum
    pairs = pairs_near + pairs_far
    value = ws / (ms_step / 1e3)

    # e2e through the C ABI with pinned host buffers (H2D + D2H inside)
    xh = torch.from_numpy(x).pin_memory()
    qh = torch.from_numpy(q).pin_memory()
    fh = torch.empty((N, 3), dtype=torch.float64).pin_memory()
    eh = torch.empty(1, dtype=torch.float64).pin_memory()
    for _ in range(2):
        P.hsma_eval_into(h.h, xh, qh, N, eh, fh)
    torch.cuda.synchronize()
    # median of >= 20 calls, each a full hsma_eval with its copies (host clock)
    e2e_t = []
    for _ in range(max(20, args.steps)):
        t0 = time.perf_counter()
        P.hsma_eval_into(h.h, xh, qh, N, eh, fh)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t))
    e2e_s = max_over_ranks(dist, e2e_s, dev)

    # the plain FP64 GPU form, for the record (one GPU only: with several,
    # every rank would repeat the same single-GPU figure)
    fp64 = None
    if args.fp64_steps > 0 and ws == 1:
        h64 = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=0, timing=1,
                     dtn_grid=c.dtn_grid)
        P.hsma_set_stream(h64.h, stream.cuda_stream)
        e64 = np.zeros(1)
        f64 = torch.empty((N, 3), dtype=torch.float64, device=dev)
        t64 = timed_evals(P, torch, stream, h64, xd, qd, N, e64, f64, args.fp64_steps)
        dF = (fd - f64).double()
        fp64 = {"evals_per_s": 1e3 / t64, "ms_per_eval": t64,
                "near_ms": P.hsma_get_info(h64.h, "t_near_ms"),
                "fp32_vs_fp64_rel_energy": abs(energy - float(e64[0])) / abs(float(e64[0])),
                "fp32_vs_fp64_rel_force_rms": float(torch.sqrt((dF ** 2).sum() / (f64 ** 2).sum())),
                "fp32_vs_fp64_max_ion_force_err": float(
                    (torch.sqrt((dF ** 2).sum(1)).max() / torch.sqrt((f64 ** 2).sum(1).mean())).item())}
        h64.close()
        # precision 2 (exact source-target differences) against the same FP64 result
        h2 = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=2, dtn_grid=c.dtn_grid)
        P.hsma_set_stream(h2.h, stream.cuda_stream)
        e2 = np.zeros(1)
        f2 = torch.empty((N, 3), dtype=torch.float64, device=dev)
        t2 = timed_evals(P, torch, stream, h2, xd, qd, N, e2, f2, 5)
        dF2 = (f2 - f64).double()
        fp64["precision2"] = {"evals_per_s": 1e3 / t2,
                              "kernel": KERNEL_NAMES.get(int(P.hsma_get_info(h2.h, "kernel"))),
                              "rel_energy_vs_fp64": abs(float(e2[0]) - float(e64[0])) / abs(float(e64[0])),
                              "rel_force_rms_vs_fp64": float(torch.sqrt((dF2 ** 2).sum() / (f64 ** 2).sum()))}
        h2.close()

    if rank != 0:
        if dist:
            dist.barrier()
        return

    mhz, mhz_src = peaks()
    sms = sm_count()
    peak_instr = sms * FP32_LANES * mhz * 1e6 / 1e12          # T lane-instr/s
    mhz_txt = f"{mhz:.0f} MHz ({mhz_src})"
    roof, plan = pair_roofline(P, h, c, pairs_near, float(np.mean(near_ms)), peak_instr, mhz_txt, sms,
                               lib_total_ms=float(np.mean(total_lib_ms)))
    if args.near_tree:
        roof = tree_roofline(P, h, xd, qd, N, ebuf, fd, float(np.mean(near_ms)), 10, peak_instr)
        roof["lib_total_ms"] = float(np.mean(total_lib_ms))

    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 pairs, f64 accumulation/fit",
            "data": "synthetic",
            "config": workload_config(c, ws),
            "run": {"N_s": Ns, "n_check": n_check, "precision": "fp32-compute/fp64-accumulate",
                    "l2": "flushed between steps (256 MB write)",
                    "far_field": "series (Eq. 5)" if args.far_field else "surface charges (Eq. 8)",
                    "near_field": "tree, order 10" if args.near_tree else "direct sums", "plan": plan},
            "pair_ints_per_s": pairs * ws / (ms_step / 1e3), "pairs_per_eval": pairs,
            "energy": energy, "roofline": roof,
            "e2e": {"value": ws / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": N * 32,
                    "d2h_bytes_per_step": N * 24 + 8},
            "gpu_launches": int(P.hsma_get_info(h.h, "kernels_per_eval")) * args.steps, "clocks": clk.summary(),
            "fp64_path": fp64}
    # the oracle baseline, the other workloads and the served stream are
    # single-GPU figures: taken at N = 1 only, so that a run on several GPUs
    # holds them no longer than its timed region needs
    single = ws == 1
    # the served stream first among the single-GPU extras, while the process
    # holds only the main handle (its host-driven loop is sensitive to what
    # ran before it on the host); reported at the end of the line
    serve_res = None
    h.close()     # the large system's buffers are not needed beyond this point
    if not args.no_serve and single:
        serve_res = (serve_bench(P), serve_bench(P, precision=2))
    if not args.no_cpu_baseline and single:
        n_s = 512
        t_full, d = oracle_sample(c, x, q, n_s)
        Fg = fd.cpu().numpy()[d["idx"]]
        Fo = d["F"]
        line["cpu_baseline"] = {
            "value": 1.0 / t_full, "unit": "evals/s", "cores": d["threads"], "kind": "oracle",
            "sample": (f"full check-point sums + fit, near+far on {n_s} of {N} ions, scaled by N/{n_s}; "
                       f"pair sums split by target over {d['threads']} host threads; "
                       f"measured {d['t_wall']:.1f} s wall"),
            "cpu": platform.processor() or platform.machine()}
        line["accuracy_vs_oracle"] = {
            "sampled_ions": n_s,
            "rel_force_rms": float(math.sqrt(np.mean(np.sum((Fg - Fo) ** 2, 1)) / np.mean(np.sum(Fo ** 2, 1)))),
            "max_ion_force_err_over_rms": float(np.sqrt(np.sum((Fg - Fo) ** 2, 1)).max()
                                                / math.sqrt(np.mean(np.sum(Fo ** 2, 1)))),
            "rel_energy_vs_fp64_gpu": fp64["fp32_vs_fp64_rel_energy"] if fp64 else None}
    if not args.no_other_cases and single:
        if args.case != 2:
            line["case2"] = secondary_case(P, torch, dev, stream, workloads.case(2), peak_instr, mhz_txt, sms)
        line["case3_2d"] = secondary_case(P, torch, dev, stream, workloads.case(3, 0.95), peak_instr, mhz_txt,
                                          sms)
        line["paper_accuracy"] = paper_accuracy(P, torch, dev, stream)
        if not args.far_field and not args.near_tree:
            c2 = workloads.case(2)
            x2, q2 = workloads.electrolyte(c2)
            xd2 = torch.from_numpy(x2).to(dev)
            qd2 = torch.from_numpy(q2).to(dev)
            fd2 = torch.empty((c2.N, 3), dtype=torch.float64, device=dev)
            h2b = P.HSMA(c2.box, 3, c2.p, c2.M, precision=1, timing=1)
            P.hsma_set_stream(h2b.h, stream.cuda_stream)
            e0 = np.zeros(1)
            P.hsma_eval_into(h2b.h, xd2, qd2, c2.N, e0, fd2)
            torch.cuda.synchronize()
            line["far_field_series"] = far_series_compare(P, torch, stream, c2, xd2, qd2, fd2, h2b)
            P.hsma_eval_into(h2b.h, xd2, qd2, c2.N, e0, fd2)
            torch.cuda.synchronize()
            line["option_variants"] = [
                option_variant(P, torch, stream, c2, xd2, qd2, fd2, float(e0[0]), sphere_mask=0),
                option_variant(P, torch, stream, c2, xd2, qd2, fd2, float(e0[0]), grad_rows=1),
                option_variant(P, torch, stream, c2, xd2, qd2, fd2, float(e0[0]), n=10, near_tree=1),
                option_variant(P, torch, stream, c2, xd2, qd2, fd2, float(e0[0]), n=10, near_tree=1, far_field=1)]
            h2b.close()
        line["other_cases"] = other_cases(P, torch, dev, stream, peak_instr)
        line["paper_like"] = paper_like(P, torch, dev, stream)
    if serve_res:
        # last, so that the end of the line (what a log tail keeps) shows them
        line["serve"], line["serve_precision2"] = serve_res
        line["serve_summary"] = {
            f"precision{k}": {key: round(float(line[name][key]), 4) for key in
                              ("evals_per_s", "p50_ms", "p99_ms", "one_at_a_time_evals_per_s",
                               "saturated_evals_per_s", "saturated_vs_one_at_a_time", "served_vs_fp64",
                               "saturated_pair_ints_per_s", "max_rel_force_rms_vs_fp64")}
            for k, name in ((1, "serve"), (2, "serve_precision2"))}
        if not args.near_tree and not args.far_field:
            # the served pair rate against the single large system's direct sums
            line["serve_summary"]["precision1"]["saturated_pair_rate_vs_bench"] = round(
                line["serve"]["saturated_pair_ints_per_s"] / line["pair_ints_per_s"], 4)
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
    h.close()


if __name__ == "__main__":
    main()
