"""Host logic of bench.py: the DRAM-traffic records (parsing an ncu CSV of
several launches, picking the near-field launch, keeping one record per
kernel and chunk count), the pair roofline's arithmetic, and the timed oracle
sample behind the CPU baseline.  No GPU: the CSV is written here in ncu's
layout and the binding is faked."""
import csv
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def write_csv(path, launches):
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(HDR)
        for i, metrics in enumerate(launches):
            for name, unit, v in metrics:
                w.writerow([str(i), "1", "python", "h", "void k_pair_f32x2s<2>(PairArgs)", "1", "7", "(256, 1, 1)",
                            "(456, 1, 1)", "0", "10.3", "Command line profiler metrics", name, unit, v])


def launch(ns, rd, wr, unit="byte", tunit="ns"):
    return [("dram__bytes_read.sum", unit, rd), ("dram__bytes_write.sum", unit, wr),
            ("gpu__time_duration.sum", tunit, ns)]


def test_longest_launch_is_recorded_and_records_merge(tmp_path):
    tr = str(tmp_path / "traffic.json")
    c1 = str(tmp_path / "a.csv")
    # far field first (short), then the near field (long); thousands separators as ncu prints them
    write_csv(c1, [launch("106,656", "1,680,640", "45,056"), launch("25,096,992", "23,778,048", "246,297,344")])
    rec = bench.record_traffic(c1, "k_pair_f32x2s<2> near field", "w", 92, "cmd", tr=tr)
    assert rec["bytes_per_launch"] == 23778048 + 246297344 and rec["chunks"] == 92
    assert rec["pair_sources_sha1"] == bench.pair_sources_sha1()
    # another chunk count is added beside it; MB units and msecond are scaled
    c2 = str(tmp_path / "b.csv")
    write_csv(c2, [launch("26.1", "12.6", "24.3", unit="Mbyte", tunit="msecond"),
                   launch("0.1", "1.0", "0.1", unit="Mbyte", tunit="msecond")])
    bench.record_traffic(c2, "k_pair_f32x2s<2> near field", "w", 23, "cmd", tr=tr)
    recs = bench.traffic_records(tr)
    assert [r["chunks"] for r in recs] == [23, 92]
    assert recs[0]["bytes_per_launch"] == int(12.6e6) + int(24.3e6)
    # re-recording a chunk count replaces its record
    bench.record_traffic(c1, "k_pair_f32x2s<2> near field", "w", 23, "cmd", tr=tr)
    recs = bench.traffic_records(tr)
    assert len(recs) == 2 and recs[0]["bytes_per_launch"] == 23778048 + 246297344


def test_single_record_files_still_read(tmp_path):
    tr = str(tmp_path / "traffic.json")
    with open(tr, "w") as f:
        json.dump({"kernel": "k", "chunks": 46, "bytes_per_launch": 1}, f)
    assert bench.traffic_records(tr) == [{"kernel": "k", "chunks": 46, "bytes_per_launch": 1}]
    assert bench.traffic_records(str(tmp_path / "missing.json")) == []


def test_committed_records_are_well_formed():
    # one record per (kernel, chunks), each with its bytes and the command
    # that captured it; a record whose source hash no longer matches is
    # simply not used by the bench
    recs = bench.traffic_records()
    keys = [(r["kernel"], r["chunks"]) for r in recs]
    assert recs and len(set(keys)) == len(keys)
    for r in recs:
        assert r["bytes_per_launch"] == r["read_bytes"] + r["write_bytes"] > 0
        assert r["command"].startswith("ncu ") and "--clock-control none" in r["command"]


class _FakeLib:
    """Stands in for the binding: the plan's info keys of one handle."""

    def __init__(self, info):
        self.info = info

    def hsma_get_info(self, h, key):
        return self.info[key]


class _FakeHandle:
    h = object()


def test_pair_roofline_arithmetic_and_traffic_record():
    # 13 FP32-pipe operations per pair over the launch time, against the
    # issue peak; the traffic record of the same (workload, kernel, chunks)
    # and kernel source is attached, any other plan reports null
    import workloads
    c = workloads.case(5)
    rec = next(r for r in bench.traffic_records() if r["workload"] == c.name
               and r["kernel"].startswith("k_pair_f32x2s<2>"))
    P = _FakeLib({"kernel": 24, "chunks": rec["chunks"], "grid": 456, "tile_targets": 1024})
    pairs, near_ms, peak = 4.115e11, 167.0, 40.27392
    roof, plan = bench.pair_roofline(P, _FakeHandle(), c, pairs, near_ms, peak, "2070 MHz", 152)
    assert plan["kernel"] == "k_pair_f32x2s<2>" and plan["chunks"] == rec["chunks"]
    assert abs(roof["achieved"] - pairs * 13 / (near_ms / 1e3) / 1e12) < 1e-9
    assert abs(roof["frac"] - roof["achieved"] / peak) < 1e-12
    if rec.get("pair_sources_sha1") == bench.pair_sources_sha1():
        assert roof["traffic"] == rec["bytes_per_launch"]
    P2 = _FakeLib({"kernel": 24, "chunks": 9999, "grid": 456, "tile_targets": 1024})
    roof2, _ = bench.pair_roofline(P2, _FakeHandle(), c, pairs, near_ms, peak, "2070 MHz", 152)
    assert roof2["traffic"] is None


def test_oracle_sample_reproduces_the_oracle():
    # the bench's timed oracle sample (pair sums split over host threads) gives
    # the oracle's own forces and potentials on its sampled ions: the
    # reference of the bench's accuracy_vs_oracle figure
    import numpy as np
    import workloads
    from oracle import hsma as O
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    _, d = bench.oracle_sample(c, x, q, 48, threads=3)
    st = O.make_setup(c.box, c.dims, c.p, c.M, lam=c.lam)
    ref = O.evaluate(st, x, q, targets=d["idx"])
    scale = np.sqrt(np.mean(np.sum(ref["forces"] ** 2, 1)))
    assert np.abs(d["F"] - ref["forces"]).max() <= 1e-12 * scale
    dphi = d["phi"] - ref["phi"]
    assert np.abs(dphi - dphi.mean()).max() <= 1e-12 * np.abs(ref["phi"]).max()
    assert d["Ns"] == ref["Ns"] and d["threads"] == 3
