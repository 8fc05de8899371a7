"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: relative energy error <= 1e-6 for the FP64 path and <= 1e-5 for
the FP32-compute path; forces are compared by their relative RMS error, with
the bound written next to each check, and each ion's force error by itself
(at most FMAX times the RMS bound, relative to the reference's RMS force).  Integer work (the set of images in the
sphere B) must match exactly.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import hsma as O

pytestmark = pytest.mark.gpu

# precision 2 is an FP32-compute path (exact differences): the FP32 bounds;
# its gain at large coordinates is checked at the bench size below
E_TOL = {0: 1e-6, 1: 1e-5, 2: 1e-5}
F_TOL = {0: 1e-6, 1: 2e-5, 2: 2e-5}      # relative RMS of the per-ion forces


@pytest.fixture(scope="module")
def P():
    from paper_2104_05260_gb300 import build
    build.build()
    import paper_2104_05260_gb300 as P
    P.lib()
    return P


def rel(a, b):
    return abs(a - b) / abs(b)


def frms(F, Fr):
    return math.sqrt(np.mean(np.sum((F - Fr) ** 2, 1)) / np.mean(np.sum(Fr ** 2, 1)))


def pot_err(pot, ref):
    d = pot - ref
    return math.sqrt(np.mean((d - d.mean()) ** 2) / np.mean(ref ** 2))

# Per-ion bound beside the relative RMS: the largest single-ion force error
# (and, after removing the mean offset, potential error) relative to the RMS of
# the reference, at most FMAX times the RMS bound.  A local mistake (one ion's
# own images, an ion next to a wall) can hide inside an RMS over all ions.
FMAX = 20


def fmax(F, Fr):
    return float(np.sqrt(np.sum((F - Fr) ** 2, 1)).max() / math.sqrt(np.mean(np.sum(Fr ** 2, 1))))


def pmax(pot, ref):
    d = pot - ref
    return float(np.abs(d - d.mean()).max() / math.sqrt(np.mean(ref ** 2)))



def run(P, c, x, q, prec, **opt):
    h = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=prec, **opt)
    E, F, pot = h.eval(x, q, potential=True)
    return h, E, F, pot


def check_full(P, c, x, q, prec, st=None, **opt):
    st = st or O.make_setup(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], lam=c.lam,
                            dtn_grid=c.dtn_grid, **{k: v for k, v in opt.items() if k == "n_monitor"})
    ref = O.evaluate(st, x, q)
    h, E, F, pot = run(P, c, x, q, prec, **opt)
    assert int(h.info("Ns")) == ref["Ns"]                      # same images in B, exactly
    assert rel(E, ref["energy"]) <= E_TOL[prec], (E, ref["energy"])
    assert frms(F, ref["forces"]) <= F_TOL[prec]
    assert fmax(F, ref["forces"]) <= FMAX * F_TOL[prec], fmax(F, ref["forces"])
    # the per-ion potential is fixed only up to an additive constant (A_0^0 is
    # dropped; for a neutral system energy and forces do not see it), so it is
    # compared after removing the mean offset
    assert pot_err(pot, ref["phi"]) <= F_TOL[prec]
    assert pmax(pot, ref["phi"]) <= FMAX * F_TOL[prec], pmax(pot, ref["phi"])
    # each step on its own: check-point sums, surface charges
    nc = int(h.info("n_check"))
    cphi = h.array("check_phi", nc)
    assert np.abs(cphi - ref["check_phi"]).max() <= 10 * E_TOL[prec] * np.abs(ref["check_phi"]).max()
    # surface charges, judged by the far field they produce at the ions (their
    # high-order parts are amplified by lambda^n in the map but decay as
    # (r/R_s)^n inside the box)
    Q = h.array("surface_q", c.M)
    fphi, _ = O.pair_field(ref["xc"], st.ysurf, Q)
    d = fphi - ref["far_phi"]
    assert math.sqrt(np.mean((d - d.mean()) ** 2) / np.mean(ref["phi"] ** 2)) <= F_TOL[prec]
    if prec == 0:
        assert np.abs(Q - ref["Q"]).max() <= 100 * E_TOL[prec] * np.abs(ref["Q"]).max()
    h.close()
    return E, ref


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cfg1_full(P, prec):
    c = workloads.case(1)                          # N = 1000, L = 10, p = 6, M = 800
    x, q = workloads.electrolyte(c)
    check_full(P, c, x, q, prec)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("N,val", [(2, (1, -1)), (3, (2, -1)), (258, (1, -1)), (1001, (2, -1)),
                                   (2050, (3, -1))])
def test_ragged_and_tiny_sizes(P, prec, N, val):
    L = 10.0 * (N / 1000) ** (1 / 3)
    c = workloads.small_case(N, dims=3, box=(L, L, L), p=4, M=200, valences=val, seed=N)
    x, q = workloads.electrolyte(c)
    check_full(P, c, x, q, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_positions_on_boundaries_and_outside(P, prec):
    L = 6.0
    c = workloads.small_case(40, dims=3, box=(L, L, L), p=4, M=200, seed=3)
    x, q = workloads.electrolyte(c)
    # exact box edges, exact wrap ties, and far-away periodic copies
    x[0] = [0.0, 0.0, 0.0]
    x[1] = [L, L / 2, -L]
    x[2] = [-1e-300, 2.5 * L, 7 * L + 0.25]
    x[3] = [L / 2, L / 2, L / 2]
    x[4] = [-3 * L + 1.0, 1e3 * L + 2.0, L - 1e-12]
    check_full(P, c, x, q, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_literal_sphere_radius_125_cells(P, prec):
    L = 5.0
    c = workloads.small_case(200, dims=3, box=(L, L, L), p=10, M=2000, lam=2.6, seed=5)
    x, q = workloads.electrolyte(c)
    st = O.make_setup(c.box, 3, 10, 2000, lam=2.6, n_monitor=200)
    assert len(st.shifts) == 125
    check_full(P, c, x, q, prec, st=st, **{"lambda": 2.6, "n_monitor": 200})


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("gam", [(-0.95, -0.95), (0.0, 0.0), (0.95, 0.95), (0.6, 0.0)])
def test_2d_small(P, prec, gam):
    c = workloads.small_case(300, dims=2, box=(20.0, 20.0, 10.0), p=6, M=600, gammas=gam,
                             G=24, seed=13)
    # ions uniform in the slab, two of them right next to a wall.  An ion at
    # distance d from a dielectric wall meets its own reflection at 2d; the
    # FP32 path sums every ion's own images in FP64, so only FP32 pairs of two
    # different ions that are both that close limit it.
    x, q = workloads.electrolyte(c)
    d = 1e-3 if prec == 1 else 1e-6
    x[0, 2] = d                          # bottom wall
    x[1, 2] = 10.0 - d                   # top wall
    check_full(P, c, x, q, prec, dtn_grid=24)


@pytest.mark.parametrize("prec", [0, 1])
def test_unmasked_near_set_3d(P, prec):
    # every image of the 27 cells is near (option sphere_mask = 0)
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    st = O.make_setup(c.box, 3, c.p, c.M, lam=c.lam, sphere_mask=False)
    assert len(st.shifts) == 27
    check_full(P, c, x, q, prec, st=st, sphere_mask=0)


@pytest.mark.parametrize("prec", [0, 1])
def test_unmasked_near_set_2d(P, prec):
    c = workloads.small_case(300, dims=2, box=(20.0, 20.0, 10.0), p=6, M=600, gammas=(0.5, -0.3),
                             G=24, seed=17)
    x, q = workloads.electrolyte(c, margin=1e-3)
    st = O.make_setup(c.box, 2, c.p, c.M, 0.5, -0.3, lam=c.lam, dtn_grid=24, sphere_mask=False)
    check_full(P, c, x, q, prec, st=st, dtn_grid=24, sphere_mask=0)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [3, 2])
def test_fibonacci_lattice_surface_rule(P, prec, dims):
    # option surface_rule = 1: the F_w/F lattice rule of Sec. 3.2 (M = F)
    import dataclasses
    if dims == 3:
        c = dataclasses.replace(workloads.case(1), M=987)
        x, q = workloads.electrolyte(c)
        st = O.make_setup(c.box, 3, c.p, c.M, lam=c.lam, surface_rule=1)
        check_full(P, c, x, q, prec, st=st, surface_rule=1)
    else:
        c = workloads.small_case(300, dims=2, box=(20.0, 20.0, 10.0), p=6, M=610, gammas=(0.5, -0.3),
                                 G=24, seed=19)
        x, q = workloads.electrolyte(c, margin=1e-3)
        st = O.make_setup(c.box, 2, c.p, c.M, 0.5, -0.3, lam=c.lam, dtn_grid=24, surface_rule=1)
        check_full(P, c, x, q, prec, st=st, dtn_grid=24, surface_rule=1)


def test_fibonacci_lattice_at_the_literal_sphere_against_ewald(P):
    # the literal sphere (lambda = 2.6) at P = 10 on the FP64 path: with the
    # lattice rule the result lies within 1e-6 of the Ewald sum
    from oracle.ewald import ewald3d
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    L = c.box[0]
    xc = (x - L * np.floor(x / L)) - 0.5 * L
    Ee, _, ge = ewald3d(xc, q, c.box)
    h = P.HSMA(c.box, 3, 10, 610, precision=0, surface_rule=1, **{"lambda": 2.6})
    E, F, _ = h.eval(x, q)
    h.close()
    assert rel(E, Ee) < 1e-6
    assert frms(F, -q[:, None] * ge) < 1e-6


def test_surface_rule_rejects_a_non_fibonacci_count(P):
    h = P.HSMA((10.0, 10.0, 10.0), 3, 6, 800)
    with pytest.raises(P.HSMAError):
        h.set_option("surface_rule", 1)
    h.close()


def test_exact_differences_close_the_fp32_gap_at_bench_size(P):
    # precision 2 against the FP64 path at N = 1e5: the close-pair force error
    # of plain FP32 (coordinates rounded at |x| ~ 50) is gone
    c = workloads.case(2)
    x, q = workloads.electrolyte(c)
    res = {}
    for prec in (0, 1, 2):
        h = P.HSMA(c.box, 3, c.p, c.M, precision=prec)
        E, F, _ = h.eval(x, q)
        res[prec] = (E, F)
        h.close()
    e1, e2 = (rel(res[k][0], res[0][0]) for k in (1, 2))
    f1, f2 = (frms(res[k][1], res[0][1]) for k in (1, 2))
    # forces: the close-pair error goes; the energy (which nearly cancels:
    # E = -2384 for 1e5 ions) keeps the FP32 bound
    assert f2 <= 2e-6 and e2 <= 1e-5, (f2, e2)
    assert f2 < 0.1 * f1


def test_errors_are_reported(P):
    c = workloads.small_case(20, dims=2, box=(20.0, 20.0, 10.0), p=4, M=200, G=8)
    x, q = workloads.electrolyte(c)
    h = P.HSMA(c.box, 2, 4, 200, 0.5, 0.5, dtn_grid=8)
    bad = x.copy(); bad[3, 2] = 10.0
    with pytest.raises(P.HSMAError) as e:
        h.eval(bad, q)
    assert e.value.code == -3
    q2 = q.copy(); q2[0] += 0.5
    with pytest.raises(P.HSMAError) as e:
        h.eval(x, q2)
    assert e.value.code == -2
    with pytest.raises(P.HSMAError) as e:
        h.set_option("lambda", 0.5)
    assert e.value.code == -1
    with pytest.raises(P.HSMAError):
        h.set_option("no_such_option", 1)
    E, F, _ = h.eval(x, q)              # the handle still works after errors
    assert np.isfinite(E) and np.all(np.isfinite(F))
    h.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_degenerate_inputs(P, prec):
    # no particles: an argument error, and the handle stays usable
    h = P.HSMA((10.0, 10.0, 10.0), 3, 4, 200, precision=prec)
    with pytest.raises(P.HSMAError) as e:
        h.eval(np.zeros((0, 3)), np.zeros(0))
    assert e.value.code == -1
    # uncharged particles (one alone, or many): energy, forces and potential
    # are exactly zero, with no division by zero for the lone particle
    rng = np.random.default_rng(3)
    for n in (1, 37):
        x = rng.uniform(0.0, 10.0, (n, 3))
        E, F, pot = h.eval(x, np.zeros(n), potential=True)
        assert E == 0.0 and np.all(F == 0.0) and np.all(pot == 0.0)
    # and a charged system afterwards still matches the oracle
    c = workloads.small_case(64, dims=3, box=(10.0, 10.0, 10.0), p=4, M=200, seed=64)
    x, q = workloads.electrolyte(c)
    ref = O.evaluate(O.make_setup(c.box, 3, 4, 200), x, q)
    E, F, _ = h.eval(x, q)
    h.close()
    assert rel(E, ref["energy"]) <= E_TOL[prec] and frms(F, ref["forces"]) <= F_TOL[prec]
    assert fmax(F, ref["forces"]) <= FMAX * F_TOL[prec]


@pytest.mark.parametrize("prec,tree", [(0, 0), (1, 0), (2, 0), (1, 1)])
def test_non_finite_inputs(P, prec, tree):
    # a non-finite position or charge makes the energy non-finite: the call
    # reports HSMA_ERR_NUMERIC and the handle stays usable
    c = workloads.small_case(2000, dims=3, box=(13.0, 13.0, 13.0), p=6, M=800, seed=19)
    x, q = workloads.electrolyte(c)
    h = P.HSMA(c.box, 3, 6, 800, precision=prec, near_tree=tree)
    for which, i, v in (("x", 5, np.nan), ("x", 1999, np.inf), ("q", 7, np.nan), ("q", 0, -np.inf)):
        xb, qb = x.copy(), q.copy()
        if which == "x":
            xb[i, 1] = v
        else:
            qb[i] = v
        with pytest.raises(P.HSMAError) as e:
            h.eval(xb, qb)
        assert e.value.code == -8, (which, i, v)
    ref = O.evaluate(O.make_setup(c.box, 3, 6, 800), x, q)
    E, F, _ = h.eval(x, q)
    h.close()
    assert rel(E, ref["energy"]) <= E_TOL[prec] and frms(F, ref["forces"]) <= F_TOL[prec]
    assert fmax(F, ref["forces"]) <= FMAX * F_TOL[prec]


def test_repeatable_bitwise(P):
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    h = P.HSMA(c.box, 3, c.p, c.M)
    E1, F1, _ = h.eval(x, q)
    E2, F2, _ = h.eval(x, q)
    assert E1 == E2 and np.array_equal(F1, F2)
    h.close()


def test_device_pointers(P):
    torch = pytest.importorskip("torch")
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    h = P.HSMA(c.box, 3, c.p, c.M)
    E0, F0, p0 = h.eval(x, q, potential=True)
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q).cuda()
    E1, F1, p1 = h.eval(xd, qd, potential=True)
    assert F1.is_cuda and E1 == E0
    assert np.array_equal(F1.cpu().numpy(), F0) and np.array_equal(p1.cpu().numpy(), p0)
    h.close()


# ------------------------------------------------------------ full-size cases
def sampled(P, c, prec, n_samp, margin=0.0, **opt):
    """Full-size run; oracle on a sample of targets plus all check points."""
    x, q = workloads.electrolyte(c, margin=margin)
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(c.N, n_samp, replace=False))
    st = O.make_setup(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], lam=c.lam,
                      dtn_grid=c.dtn_grid)
    ref = O.evaluate(st, x, q, targets=idx)
    h, E, F, pot = run(P, c, x, q, prec, **opt)
    assert int(h.info("Ns")) == ref["Ns"]
    assert frms(F[idx], ref["forces"]) <= F_TOL[prec]
    assert fmax(F[idx], ref["forces"]) <= FMAX * F_TOL[prec], fmax(F[idx], ref["forces"])
    assert pot_err(pot[idx], ref["phi"]) <= F_TOL[prec]
    assert pmax(pot[idx], ref["phi"]) <= FMAX * F_TOL[prec], pmax(pot[idx], ref["phi"])
    Q = h.array("surface_q", c.M)
    assert np.abs(Q - ref["Q"]).max() <= 100 * E_TOL[prec] * np.abs(ref["Q"]).max()
    h.close()
    return E


@pytest.mark.parametrize("prec", [0, 1])
def test_cfg2_100k_sampled(P, prec):
    sampled(P, workloads.case(2), prec, 48)


def test_cfg2_energy_fp32_vs_fp64(P):
    # the whole-system energy of the FP32 path against the FP64 path (the FP64
    # path itself is pinned to the oracle above)
    c = workloads.case(2)
    x, q = workloads.electrolyte(c)
    _, E64, _, _ = run(P, c, x, q, 0)
    _, E32, _, _ = run(P, c, x, q, 1)
    assert rel(E32, E64) <= E_TOL[1]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cfg5_262k_sampled(P, prec):
    # the bench workload (N = 262,144, p = 10, M = 4000) at every precision
    sampled(P, workloads.case(5), prec, 24)


def test_cfg5_exact_differences_reach_fp64_class_forces(P):
    # precision 2 at the bench workload: FP32 pair arithmetic with exactly
    # formed differences agrees with the oracle like an FP64 path (force RMS
    # and every sampled ion within 1e-6 / 2e-5 of the RMS force)
    c = workloads.case(5)
    x, q = workloads.electrolyte(c)
    rng = np.random.default_rng(321)
    idx = np.sort(rng.choice(c.N, 24, replace=False))
    st = O.make_setup(c.box, 3, c.p, c.M, lam=c.lam)
    ref = O.evaluate(st, x, q, targets=idx)
    h, E, F, pot = run(P, c, x, q, 2)
    h.close()
    assert frms(F[idx], ref["forces"]) <= 1e-6, frms(F[idx], ref["forces"])
    assert fmax(F[idx], ref["forces"]) <= 2e-5, fmax(F[idx], ref["forces"])


@pytest.mark.parametrize("gam", [-0.95, 0.0, 0.95, (0.6, -0.3)])
def test_cfg3_2d_20k_stagewise(P, gam):
    # 2D, N = 20000, G = 80: the oracle cannot redo all 13124 check targets in
    # seconds, so each step is checked on its own: check-point sums on a
    # sample, the fit + map from the GPU's own check values, and near + far at
    # sampled particles.  The last case has unequal interfaces.
    import dataclasses
    gt, gb = gam if isinstance(gam, tuple) else (gam, gam)
    c = dataclasses.replace(workloads.case(3, gamma=gt), gammas=(gt, gb))
    x, q = workloads.electrolyte(c)
    st = O.make_setup(c.box, 2, c.p, c.M, gt, gb, lam=c.lam, dtn_grid=c.dtn_grid)
    h, E, F, pot = run(P, c, x, q, 1)
    xc, qc = O.prepare_inputs(st, x, q)
    ipos, iq, isrc, isid = O.near_set(st, xc, qc)
    assert int(h.info("Ns")) == len(iq)
    nc = int(h.info("n_check"))
    cphi = h.array("check_phi", nc)
    cdz = h.array("check_dz", nc)
    rng = np.random.default_rng(7)
    ci = np.sort(rng.choice(nc, 200, replace=False))
    ophi, ograd = O.pair_field(st.check_pts[ci], ipos, iq)
    assert np.abs(cphi[ci] - ophi).max() <= 1e-5 * np.abs(ophi).max()
    assert np.abs(cdz[ci] - ograd[:, 2]).max() <= 1e-5 * np.abs(ograd[:, 2]).max()
    Q = h.array("surface_q", c.M)
    Qo = st.W @ (st.P @ np.concatenate([cphi, cdz]))
    assert np.abs(Q - Qo).max() <= 1e-9 * np.abs(Qo).max()
    ti = np.sort(rng.choice(c.N, 32, replace=False))
    s0 = O.self_shift(st)
    self_idx = np.full(c.N, -1)
    m0 = isid == s0
    self_idx[isrc[m0]] = np.nonzero(m0)[0]
    nphi, ngrad = O.pair_field(xc[ti], ipos, iq, exclude=self_idx[ti])
    fphi, fgrad = O.pair_field(xc[ti], st.ysurf, Q)
    Fr = -qc[ti, None] * (ngrad + fgrad)
    assert frms(F[ti], Fr) <= F_TOL[1]
    assert fmax(F[ti], Fr) <= FMAX * F_TOL[1], fmax(F[ti], Fr)
    h.close()


def test_kernel_variants_graphs_and_tuning_agree(P):
    # every FP32 kernel variant sums the same pair terms in the same source
    # order, so with a fixed chunk count they agree bitwise; CUDA-graph replay
    # changes nothing; autotuned chunking only changes FP64 combine order
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    ref = None
    for tpt in (1, 2, 4, 12, 14, 24):
        for graphs in (0, 1):
            h = P.HSMA(c.box, 3, c.p, c.M, targets_per_thread=tpt, chunks=8, graphs=graphs)
            E, F, pot = h.eval(x, q, potential=True)
            E2, F2, _ = h.eval(x, q)
            h.close()
            assert E == E2 and np.array_equal(F, F2)
            if ref is None:
                ref = (E, F, pot)
            assert E == ref[0] and np.array_equal(F, ref[1]) and np.array_equal(pot, ref[2]), (tpt, graphs)
    h = P.HSMA(c.box, 3, c.p, c.M)            # autotune on (default)
    E, F, _ = h.eval(x, q)
    h.close()
    assert rel(E, ref[0]) <= 1e-12 and frms(F, ref[1]) <= 1e-12


def test_exact_difference_variants_agree(P):
    # the three exact-difference kernels (2 or 4 targets per thread, sums in
    # registers or in shared memory) form the same differences and sum the
    # same pair terms in the same order, so with a fixed chunk count they
    # agree bitwise, with and without graph replay
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    ref = None
    for tpt in (32, 34, 44):
        for graphs in (0, 1):
            h = P.HSMA(c.box, 3, c.p, c.M, precision=2, targets_per_thread=tpt, chunks=8, graphs=graphs)
            E, F, pot = h.eval(x, q, potential=True)
            assert h.info("kernel") == tpt
            h.close()
            if ref is None:
                ref = (E, F, pot)
            assert E == ref[0] and np.array_equal(F, ref[1]) and np.array_equal(pot, ref[2]), (tpt, graphs)


@pytest.mark.parametrize("prec,tpt", [(0, 1), (1, 12), (1, 24), (1, 1), (2, 44)])
def test_fused_reduction_and_dynamic_schedule_change_nothing(P, prec, tpt):
    # the chunk partials summed inside the pair launch (in the fixed order of
    # the separate reduction) and items taken from a counter instead of a
    # static round-robin: bitwise the same results, on a ragged size with
    # several target tiles, at several chunk counts
    c = workloads.small_case(2050, dims=3, box=(12.7, 12.7, 12.7), p=6, M=800, valences=(3, -1), seed=7)
    x, q = workloads.electrolyte(c)
    for chunks in (1, 5, 13):
        ref = None
        for fused in (0, 1, 2):                     # never, where it pays, always
            for dyn in (0, 1):
                opt = dict(chunks=chunks, fused_reduce=fused, dynamic_schedule=dyn)
                if prec:
                    opt["targets_per_thread"] = tpt
                h = P.HSMA(c.box, 3, c.p, c.M, precision=prec, **opt)
                E, F, pot = h.eval(x, q, potential=True)
                E2, F2, _ = h.eval(x, q)            # the counters were left at zero
                assert h.info("fused_reduce") == fused and h.info("dynamic_schedule") == dyn
                if fused != 1:
                    assert h.info("fused_near") == (fused == 2) and h.info("fused_far") == (fused == 2)
                h.close()
                assert E == E2 and np.array_equal(F, F2)
                if ref is None:
                    ref = (E, F, pot)
                assert E == ref[0] and np.array_equal(F, ref[1]) and np.array_equal(pot, ref[2]), opt
