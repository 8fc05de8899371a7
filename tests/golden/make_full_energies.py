"""Write full oracle energies of the large workload cases (run once, offline).

The CPU HSMA oracle evaluated in full (every ion, every image in B) on the
seeded workloads of ``workloads.py``: case 2 (N = 100,000) and case 3
(N = 20,000, three values of gamma).  The near-field and far-field sums over
all ions are split over a pool of worker processes (``spawn``); each worker
calls the oracle's own pair sum on a contiguous block of ions, and the
energies are summed in block order.  Only ``oracle/`` and ``workloads.py``
are used.

    python tests/golden/make_full_energies.py [--workers 8]

Output: tests/golden/full_energies.json.
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def _setup(case_args):
    import workloads
    from oracle import hsma as O
    c = workloads.case(*case_args)
    x, q = workloads.electrolyte(c)
    st = O.make_setup(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], lam=c.lam,
                      dtn_grid=c.dtn_grid)
    return c, x, q, st


def _block(args):
    case_args, i0, i1, Q = args
    from oracle import hsma as O
    c, x, q, st = _setup(case_args)
    out = O.evaluate(st, x, q, targets=np.arange(i0, i1), Q=Q)
    return i0, float(np.dot(out["q"][i0:i1], out["phi"])), out["Ns"]


def full_energy(case_args, workers):
    from oracle import hsma as O
    t0 = time.time()
    c, x, q, st = _setup(case_args)
    # the fit once (check-point sums over every image in B), then the ions in blocks
    Q = O.evaluate(st, x, q, targets=np.arange(1))["Q"]
    blocks = np.linspace(0, c.N, 8 * workers + 1).astype(int)
    jobs = [(case_args, int(a), int(b), Q) for a, b in zip(blocks[:-1], blocks[1:]) if b > a]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = sorted(pool.map(_block, jobs), key=lambda t: t[0])
    e = sum(p[1] for p in parts)
    return {"name": c.name, "N": c.N, "energy": 0.5 * e, "N_s": parts[0][2],
            "seconds": time.time() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 4)
    a = ap.parse_args()
    res = {}
    for case_args in ((3, -0.95), (3, 0.0), (3, 0.95), (2,)):
        r = full_energy(case_args, a.workers)
        print(json.dumps(r), flush=True)
        res[r["name"]] = r
    with open(os.path.join(HERE, "full_energies.json"), "w") as f:
        json.dump({"source": "oracle.hsma (CPU FP64), written by tests/golden/make_full_energies.py",
                   "cases": res}, f, indent=1)


if __name__ == "__main__":
    main()
