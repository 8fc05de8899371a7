"""HSMA-vs-Ewald method error for the workload shapes (TEST INFRASTRUCTURE).

The HSMA result is an approximation of the plain sums of Sec. 2.1, Eq. 3 and
Eq. 4; this script measures how far the CPU HSMA (``oracle.hsma``) lands from
the Ewald ground truth (``oracle.ewald``) for the workload shapes, so the
method's own error can be stated beside the GPU-vs-oracle parity.

    python -m oracle.method_error [--quick]

Large systems are measured on sampled ions (forces) because the Ewald sums
here are plain O(N^2) NumPy.
"""
import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import hsma as O  # noqa: E402
from oracle.ewald import ewald3d, ewald2d_field, image_factor, image_z, slab_lmax  # noqa: E402


def rel_rms(F, Fe):
    return math.sqrt(np.mean(np.sum((F - Fe) ** 2, 1)) / np.mean(np.sum(Fe ** 2, 1)))


def case1():
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    L = c.box[0]
    xc = (x - L * np.floor(x / L)) - 0.5 * L
    Ee, _, ge = ewald3d(xc, q, c.box)
    out = O.evaluate(O.make_setup(c.box, 3, c.p, c.M), x, q)
    return {"case": c.name, "rel_energy": abs(out["energy"] - Ee) / abs(Ee),
            "rel_force_rms": rel_rms(out["forces"], -q[:, None] * ge)}


def ewald3d_at(xc, q, box, idx, rcut):
    """Ewald potential gradient at the ions idx only (same formulas as ewald3d)."""
    from scipy.special import erfc
    L = np.asarray(box)
    s = math.sqrt(-math.log(1e-16))
    a = s / rcut
    kmax = 2 * a * s
    n = [int(math.ceil(rcut / L[d])) + 1 for d in range(3)]
    g = np.stack(np.meshgrid(*[np.arange(-k, k + 1) for k in n], indexing="ij"), -1).reshape(-1, 3) * L
    grad = np.zeros((len(idx), 3))
    for t, i in enumerate(idx):
        d = xc[None, :, :] + g[:, None, :] - xc[i]
        r = np.sqrt((d * d).sum(-1))
        keep = (r < rcut) & (r > 0)
        rr = np.where(keep, r, 1.0)
        f = np.where(keep, (erfc(a * rr) / rr ** 2 + a * 2 / math.sqrt(math.pi) * np.exp(-(a * rr) ** 2) / rr) / rr, 0.0)
        grad[t] = np.einsum("sj,sjc,j->c", f, d, q)
    m = [int(math.floor(kmax * L[d] / (2 * math.pi))) + 1 for d in range(3)]
    mm = np.stack(np.meshgrid(*[np.arange(-k, k + 1) for k in m], indexing="ij"), -1).reshape(-1, 3)
    mm = mm[np.any(mm != 0, axis=1)]
    kv = 2 * math.pi * mm / L
    k2 = (kv * kv).sum(1)
    sel = k2 <= kmax * kmax
    kv, k2 = kv[sel], k2[sel]
    fk = np.exp(-k2 / (4 * a * a)) / k2
    V = L.prod()
    for c0 in range(0, len(kv), 4000):
        kc = kv[c0:c0 + 4000]
        kr = xc @ kc.T
        Sre = q @ np.cos(kr)
        Sim = q @ np.sin(kr)
        kt = xc[idx] @ kc.T
        grad += (4 * math.pi / V) * (((np.sin(kt) * -Sre + np.cos(kt) * Sim) * fk[c0:c0 + 4000]) @ kc)
    return grad


def case2_shape(N=8000, n_samp=48):
    L = (N / 0.1) ** (1 / 3)
    c = workloads.small_case(N, dims=3, box=(L, L, L), p=8, M=2000, seed=2)
    x, q = workloads.electrolyte(c)
    xc = (x - L * np.floor(x / L)) - 0.5 * L
    idx = np.sort(np.random.default_rng(0).choice(N, n_samp, replace=False))
    ge = ewald3d_at(xc, q, c.box, idx, rcut=0.5 * L)
    out = O.evaluate(O.make_setup(c.box, 3, 8, 2000), x, q, targets=idx)
    return {"case": f"density 0.1, N = {N}, p = 8, M = 2000 (case-2 parameters)",
            "rel_force_rms_sampled": rel_rms(out["forces"], -q[idx, None] * ge), "sampled_ions": n_samp}


def case3_shape(gam, margin, N=2000, n_samp=32, gam_bot=None):
    """Slab of the case-3 shape; gam_bot (default gam) gives unequal
    interfaces (image factors per Sec. 2.1, Eq. 4 with reading R7)."""
    gb = gam if gam_bot is None else gam_bot
    c = workloads.small_case(N, dims=2, box=(20.0, 20.0, 10.0), p=8, M=1500, gammas=(gam, gb),
                             G=80, seed=3)
    x, q = workloads.electrolyte(c, margin=margin)
    Lx, Ly, Lz = c.box
    xc = x - np.array([Lx / 2, Ly / 2, Lz / 2])
    idx = np.sort(np.random.default_rng(1).choice(N, n_samp, replace=False))
    rc = 0.5 * Lx + 0.5 * Lz
    ex = -np.ones(N, dtype=int)
    _, g = ewald2d_field(xc[idx], xc, q, Lx, Ly, rc, tol=1e-12,
                         exclude=np.arange(N)[idx])
    for l in range(1, slab_lmax(gam, gb, Lx, Ly, Lz, eps=1e-12) + 1):
        for sign in (+1, -1):
            f = image_factor(l, sign, gam, gb)
            if f == 0.0:
                continue
            img = xc.copy()
            img[:, 2] = image_z(xc[:, 2], l, sign, Lz)
            _, gl = ewald2d_field(xc[idx], img, f * q, Lx, Ly, rc, tol=1e-12)
            g += gl
    out = O.evaluate(O.make_setup(c.box, 2, 8, 1500, gam, gb, dtn_grid=80), x, q, targets=idx)
    return {"case": f"2D 20x20x10, N = {N}, gamma_top = {gam}, gamma_bot = {gb}, wall margin {margin}, "
                    f"p = 8, M = 1500, G = 80",
            "rel_force_rms_sampled": rel_rms(out["forces"], -q[idx, None] * g), "sampled_ions": n_samp}


def case1_variants():
    """Case 1 under the options of the build: the unmasked near set, the
    gradient-periodicity rows and the series far field, each against Ewald."""
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    L = c.box[0]
    xc = (x - L * np.floor(x / L)) - 0.5 * L
    Ee, _, ge = ewald3d(xc, q, c.box)
    out = []
    for label, kw, far in (("unmasked near set", dict(sphere_mask=False), "surface"),
                           ("gradient rows", dict(grad_rows=True), "surface"),
                           ("series far field", {}, "series")):
        r = O.evaluate(O.make_setup(c.box, 3, c.p, c.M, **kw), x, q, far=far)
        out.append({"case": f"{c.name}, {label}", "rel_energy": abs(r["energy"] - Ee) / abs(Ee),
                    "rel_force_rms": rel_rms(r["forces"], -q[:, None] * ge)})
    return out


def surface_rules():
    """Case 1 positions at p = 10 under the two surface rules (R3, R18), at
    the default sphere (lambda = 1.3) and the literal one (lambda = 2.6)."""
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    L = c.box[0]
    xc = (x - L * np.floor(x / L)) - 0.5 * L
    Ee, _, ge = ewald3d(xc, q, c.box)
    out = []
    for lam, runs in ((1.3, ((0, 800), (1, 987))), (2.6, ((0, 800), (0, 2584), (1, 610), (1, 2584)))):
        for rule, M in runs:
            r = O.evaluate(O.make_setup(c.box, 3, 10, M, lam=lam, surface_rule=rule), x, q)
            name = "golden spiral" if rule == 0 else "Fibonacci lattice"
            out.append({"case": f"{c.name} positions, p = 10, lambda = {lam}, {name}, M = {M}",
                        "rel_energy": abs(r["energy"] - Ee) / abs(Ee),
                        "rel_force_rms": rel_rms(r["forces"], -q[:, None] * ge)})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    a = ap.parse_args()
    res = [case1(), *case1_variants(), *surface_rules(), case2_shape(N=4000 if a.quick else 8000)]
    for gam in (-0.95, 0.0, 0.95):
        for margin in (0.0, 0.5):
            res.append(case3_shape(gam, margin, N=800 if a.quick else 2000))
    for gt, gb in ((0.95, -0.95), (-0.5, 0.8), (0.95, 0.0)):
        res.append(case3_shape(gt, 0.5, N=800 if a.quick else 2000, gam_bot=gb))
    for r in res:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
