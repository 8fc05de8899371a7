"""GPU MD loop (hsma_md_*, the validation workload of Sec. 4.1) against the
oracle's MD loop (oracle/md.py) driven by the oracle's HSMA, from the same
state: positions, velocities and thermo rows after a few steps of velocity
Verlet with the Nose-Hoover thermostat, FP64 electrostatics.  Also bitwise
reproducibility, NVE energy conservation and the RDF pair counts."""
import numpy as np
import pytest

import workloads

from oracle import hsma as O
from oracle import md as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2104_05260_gb300 import build
    build.build()
    import paper_2104_05260_gb300 as P
    P.lib()
    return P


def system(n_side=4, L=6.0, seed=1, kT=1.0):
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = x + rng.uniform(-0.15, 0.15, x.shape)
    n = len(x)
    q = np.where(rng.permutation(n) % 2 == 0, 1.0, -1.0)
    if n % 2:
        q[np.nonzero(q > 0)[0][0]] = 0.0          # neutral with an odd count
    v = OM.maxwell_velocities(n, kT, 1.0, rng)
    return x, v, q, [L, L, L]


def oracle_run(x, v, q, box, steps, dt, tdamp, lb, p, M):
    st = O.make_setup(box, 3, p, M, prefactor=lb)

    def coul(xx, qq):
        out = O.evaluate(st, xx, qq)
        return out["energy"], out["forces"]
    it = OM.Integrator(coul, dt=dt, kT=1.0, tdamp=tdamp)
    s = OM.State(x, v, q, box)
    rows = []
    for _ in range(steps):
        it.step(s)
        rows.append([s.kinetic(), s.U_lj, s.U_c, s.xi, s.eta, it.extended_energy(s)])
    return s, np.array(rows)


@pytest.mark.parametrize("tdamp", [0.05, 0.0])
def test_md_matches_oracle(P, tdamp):
    x, v, q, box = system()
    lb, p, M, dt, steps = 3.5, 6, 400, 0.004, 12
    h = P.HSMA(box, 3, p, M, precision=0, coulomb_prefactor=lb)
    md = P.MD(h, x, v, q, dt=dt, kT=1.0, tdamp=tdamp)
    t = md.run(steps)
    s, ref = oracle_run(x, v, q, box, steps, dt, tdamp if tdamp > 0 else None, lb, p, M)
    scale = np.abs(ref).max(axis=0) + 1e-300
    assert np.all(np.abs(t - ref) <= 1e-9 * np.maximum(scale, 1.0)), np.abs(t - ref).max(axis=0)
    assert np.abs(md.get("x_unwrapped") - s.unwrapped()).max() < 1e-10
    assert np.abs(md.get("x") - s.x).max() < 1e-10
    assert np.abs(md.get("v") - s.v).max() < 1e-9
    md.close()
    h.close()


def test_md_is_bitwise_reproducible_and_conserves_energy(P):
    x, v, q, box = system(n_side=5, L=8.0, seed=2)
    h = P.HSMA(box, 3, 6, 400, precision=0, coulomb_prefactor=1.0)
    rows = []
    for _ in range(2):
        md = P.MD(h, x, v, q, dt=0.002, kT=1.0, tdamp=0.0)
        rows.append(md.run(300))
        md.close()
    assert np.array_equal(rows[0], rows[1])
    H = rows[0][:, 5]
    # velocity Verlet: bounded energy error; the HSMA forces are not exactly
    # conservative (a fit per configuration), so allow a small drift
    assert np.abs(H - H[0]).max() < 2e-3 * (abs(H[0]) + rows[0][:, 0].mean())
    h.close()


def test_md_rdf_counts_match_oracle(P):
    x, v, q, box = system(n_side=5, L=8.0, seed=3)
    h = P.HSMA(box, 3, 6, 400, precision=1)
    md = P.MD(h, x, v, q, dt=0.002, kT=1.0, tdamp=0.1)
    md.set_option("rdf_bins", 40)
    md.set_option("rdf_rmax", 4.0)
    md.set_option("rdf_every", 1)
    md.run(1)
    counts = md.get("rdf").reshape(3, 40)
    xs = md.get("x")
    cat, an = q > 0, q < 0
    assert int(md.get("state")[4]) == 1
    assert np.array_equal(counts[0], OM.rdf_counts(xs, box, cat, an, 4.0, 40))
    assert np.array_equal(2 * counts[1], OM.rdf_counts(xs, box, cat, cat, 4.0, 40))
    assert np.array_equal(2 * counts[2], OM.rdf_counts(xs, box, an, an, 4.0, 40))
    md.close()
    h.close()


def test_md_thermostat_holds_the_temperature_fp32(P):
    x, v, q, box = system(n_side=6, L=9.0, seed=4, kT=2.0)
    h = P.HSMA(box, 3, 6, 400, precision=1, coulomb_prefactor=1.0)
    md = P.MD(h, x, v, q, dt=0.004, kT=1.0, tdamp=0.1)
    t = md.run(3000)
    n = len(q)
    T = 2 * t[1000:, 0] / (3 * n - 3)
    assert abs(T.mean() - 1.0) < 0.05
    assert np.abs(t[:, 5] - t[0, 5]).max() < 0.02 * abs(t[0, 5]) + 0.05 * n
    md.close()
    h.close()


def test_md_rejects_bad_arguments(P):
    x, v, q, box = system()
    h = P.HSMA(box, 3, 6, 400)
    with pytest.raises(P.HSMAError):
        P.MD(h, x, v, q[:-1] * 0 + 1, dt=0.01)          # sizes / neutrality
    h2 = P.HSMA([3.0, 3.0, 3.0], 3, 4, 100)
    with pytest.raises(P.HSMAError):
        P.MD(h2, x[:8] * 0.5, v[:8], q[:8], dt=0.01)    # box under 3 LJ cells a side
    h.close()
    h2.close()


def test_md_refuses_a_replanned_handle(P):
    x, v, q, box = system()
    h = P.HSMA(box, 3, 6, 400, precision=1)
    md = P.MD(h, x, v, q, dt=0.004)
    md.run(2)
    h.set_option("precision", 0)            # re-plans the handle's buffers and kernels
    h.eval(x, q)
    with pytest.raises(P.HSMAError):
        md.run(1)
    md.close()
    h.close()


def slab_system(n=120, box=(8.0, 8.0, 6.0), seed=5):
    rng = np.random.default_rng(seed)
    c = workloads.small_case(n, dims=2, box=box, seed=seed)
    x, q = workloads.electrolyte(c, min_dist=0.9, margin=0.7)
    v = OM.maxwell_velocities(n, 1.0, 1.0, rng)
    return x, v, q, list(box)


@pytest.mark.parametrize("tdamp", [0.05, 0.0])
def test_slab_md_matches_oracle(P, tdamp):
    # the confined electrolyte of Sec. 4.3: LJ walls, dielectric images (gamma 0.6)
    x, v, q, box = slab_system()
    lb, p, M, dt, steps, gam = 3.5, 6, 400, 0.004, 10, 0.6
    h = P.HSMA(box, 2, p, M, gam, gam, precision=0, coulomb_prefactor=lb, dtn_grid=24)
    md = P.MD(h, x, v, q, dt=dt, kT=1.0, tdamp=tdamp)
    t = md.run(steps)
    st = O.make_setup(box, 2, p, M, gam, gam, dtn_grid=24, prefactor=lb)

    def coul(xx, qq):
        out = O.evaluate(st, xx, qq)
        return out["energy"], out["forces"]
    it = OM.Integrator(coul, dt=dt, kT=1.0, tdamp=tdamp if tdamp > 0 else None)
    s = OM.State(x, v, q, box, slab=True)
    ref = []
    for _ in range(steps):
        it.step(s)
        ref.append([s.kinetic(), s.U_lj, s.U_c, s.xi, s.eta, it.extended_energy(s)])
    ref = np.array(ref)
    scale = np.maximum(np.abs(ref).max(axis=0), 1.0)
    assert np.all(np.abs(t - ref) <= 1e-9 * scale), np.abs(t - ref).max(axis=0)
    assert np.abs(md.get("x_unwrapped") - s.unwrapped()).max() < 1e-10
    assert np.abs(md.get("v") - s.v).max() < 1e-9
    md.close()
    h.close()


def test_slab_density_histogram_counts_every_ion(P):
    x, v, q, box = slab_system(seed=6)
    h = P.HSMA(box, 2, 6, 400, 0.6, 0.6, precision=1, coulomb_prefactor=3.5, dtn_grid=24)
    md = P.MD(h, x, v, q, dt=0.004, kT=1.0, tdamp=0.05)
    md.set_option("zhist_bins", 12)
    md.set_option("rdf_every", 5)
    md.run(50)
    zh = md.get("zhist").reshape(2, 12)
    samples = int(md.get("state")[4])
    assert samples == 10
    assert zh[0].sum() == samples * np.sum(q > 0) and zh[1].sum() == samples * np.sum(q < 0)
    xs = md.get("x")
    assert np.all((xs[:, 2] > 0) & (xs[:, 2] < box[2]))
    md.close()
    h.close()


def test_md_with_the_tree_and_with_exact_differences(P):
    # the MD step graph captures whichever electrostatics path the handle
    # runs: the tree evaluation (persistent kernel, work queue) and the
    # exact-difference pairs give the same short trajectory as the dense
    # paths within their accuracy
    x, v, q, box = system(n_side=8, L=12.0, seed=5)
    out = {}
    for label, opt in (("fp64", dict(precision=0)), ("fp32", dict(precision=1)),
                       ("tree", dict(precision=1, near_tree=1)), ("exact", dict(precision=2))):
        h = P.HSMA(box, 3, 6, 400, coulomb_prefactor=1.0, **opt)
        md = P.MD(h, x, v, q, dt=0.002, kT=1.0, tdamp=0.1)
        rows = md.run(20)
        out[label] = (md.get("x_unwrapped"), rows)
        md.close()
        h.close()
    ref_x, ref_rows = out["fp64"]
    for label, tol in (("fp32", 1e-6), ("tree", 1e-6), ("exact", 1e-8)):
        xs, rows = out[label]
        assert np.abs(xs - ref_x).max() < tol, label
        assert np.allclose(rows[:, 2], ref_rows[:, 2], rtol=1e-4, atol=0), label   # Coulomb energy rows


def test_md_with_hsma_follows_an_ewald_driven_run(P):
    # The paper validates HSMA3D by MD of the Sec. 4.1 electrolyte against a
    # reference solver.  The library's MD loop (FP64 pairs, HSMA at the paper's
    # accuracy setting: p = 10, N_m = 200, unmasked 27-cell near set) against
    # the oracle's MD loop driven by the Ewald sum, from the same start: ions
    # on a jittered lattice at the E1 number density, l_B = 3.5, dt = 0.01,
    # Nose-Hoover damping time 0.1, 60 steps.  A relative force error e moves
    # a trajectory by about e |F| t^2 / 2 (~3e-5 sigma here), so positions must
    # agree to 1e-4 sigma and the Coulomb and extended energies to 1e-5.
    from oracle.ewald import ewald3d
    lb, steps = 3.5, 60
    rng = np.random.default_rng(41)
    n_side = 5
    L = (n_side ** 3 / (3000 / 25.0 ** 3)) ** (1 / 3)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = x + rng.uniform(-0.2, 0.2, x.shape)
    n = len(x)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    q[-1] = 0.0
    v = OM.maxwell_velocities(n, 1.0, 1.0, rng)
    box = [L, L, L]

    def ewald_coulomb(xx, qq):
        xc = (xx - L * np.floor(xx / L)) - 0.5 * L
        E, _, gr = ewald3d(xc, qq, box, tol=1e-14)
        return lb * E, -lb * qq[:, None] * gr
    it = OM.Integrator(ewald_coulomb, dt=0.01, kT=1.0, tdamp=0.1)
    s = OM.State(x, v, q, box)
    rows = []
    for _ in range(steps):
        it.step(s)
        rows.append([s.U_c, it.extended_energy(s)])
    rows = np.array(rows)
    h = P.HSMA(box, 3, 10, 2000, precision=0, coulomb_prefactor=lb, n_monitor=200, sphere_mask=0)
    md = P.MD(h, x, v, q, dt=0.01, kT=1.0, tdamp=0.1)
    t = md.run(steps)
    xg = md.get("x_unwrapped")
    md.close()
    h.close()
    assert np.abs(xg - s.unwrapped()).max() < 1e-4
    # thermo rows: kinetic, U_lj, U_coulomb, xi, eta, extended energy
    assert np.abs(t[:, 2] - rows[:, 0]).max() < 1e-5 * np.abs(rows[:, 0]).max()
    assert np.abs(t[:, 5] - rows[:, 1]).max() < 1e-5 * np.abs(rows[:, 1]).max()
