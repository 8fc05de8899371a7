"""Pins of the oracle's MD loop (the validation workload of Sec. 4.1) to facts
it does not itself compute: the WCA closed form and F = -grad U by finite
differences, time reversibility and second-order energy conservation of
velocity Verlet, the Nose-Hoover thermostat against an independent RK4
solution of its scalar equations for an ideal gas, conservation of the
extended energy, the RDF counts against a brute-force double loop, and for
the slab of Sec. 4.3 the LJ-wall closed form and gradient, reversibility and
confinement."""
import math

import numpy as np
import pytest

from oracle import md
from oracle.ewald import ewald3d


def lattice(n_side, L, jitter, rng):
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    return x + rng.uniform(-jitter, jitter, x.shape)


def ewald_coulomb(box, lb):
    def f(x, q):
        L = np.asarray(box)
        xc = (x - L * np.floor(x / L)) - 0.5 * L
        E, _, g = ewald3d(xc, q, box, tol=1e-14)
        return lb * E, -lb * q[:, None] * g
    return f


def test_wca_closed_form_and_gradient():
    box = [10.0, 10.0, 10.0]
    for r in (0.9, 1.0, 1.1, md.WCA_CUT - 1e-9, 1.2):
        x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        U, F = md.wca(x, box)
        ref = 4 * (r ** -12 - r ** -6) + 1 if r < md.WCA_CUT else 0.0
        assert abs(U - ref) < 1e-12 * max(1.0, abs(ref))
        assert np.allclose(F[0], -F[1], atol=0)
    assert md.wca(np.array([[1.0, 1, 1], [1.0 + md.WCA_CUT - 1e-9, 1, 1]]), box)[0] < 1e-7
    rng = np.random.default_rng(0)
    x = lattice(3, 3.3, 0.15, rng)
    U, F = md.wca(x, [3.3] * 3)
    assert U > 0
    h = 1e-6
    for i, d in ((0, 0), (5, 1), (13, 2)):
        e = np.zeros_like(x); e[i, d] = h
        fd = -(md.wca(x + e, [3.3] * 3)[0] - md.wca(x - e, [3.3] * 3)[0]) / (2 * h)
        assert abs(fd - F[i, d]) < 1e-6 * max(1.0, np.abs(F).max())


def small_system(seed=1, n_side=3, L=4.0):
    rng = np.random.default_rng(seed)
    x = lattice(n_side, L, 0.2, rng)
    n = len(x)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    if n % 2:
        q[-1] = 0.0
    v = md.maxwell_velocities(n, 1.0, 1.0, rng)
    return x, v, q, [L, L, L]


def test_velocity_verlet_is_time_reversible():
    x, v, q, box = small_system()
    it = md.Integrator(ewald_coulomb(box, 1.0), dt=0.005)
    s = md.State(x, v, q, box)
    x0 = s.unwrapped().copy()
    for _ in range(25):
        it.step(s)
    s.v = -s.v
    for _ in range(25):
        it.step(s)
    assert np.abs(s.unwrapped() - x0).max() < 1e-9
    assert np.abs(s.v + v).max() < 1e-9


def test_nve_energy_error_is_second_order():
    x, v, q, box = small_system(seed=2)
    devs = []
    for dt in (0.004, 0.002):
        it = md.Integrator(ewald_coulomb(box, 1.0), dt=dt)
        s = md.State(x, v, q, box)
        it.forces(s)
        H0 = it.extended_energy(s)
        dev = 0.0
        for _ in range(int(round(0.08 / dt))):
            it.step(s)
            dev = max(dev, abs(it.extended_energy(s) - H0))
        devs.append(dev)
    assert 3.0 < devs[0] / devs[1] < 5.0


def test_nose_hoover_matches_rk4_for_an_ideal_gas():
    # no forces: only K and xi evolve, dK/dt = -2 xi K, dxi/dt = (2K - g kT)/Q
    rng = np.random.default_rng(3)
    n, kT, tdamp, dt, steps = 20, 1.0, 0.2, 0.01, 200
    v = md.maxwell_velocities(n, 2.5, 1.0, rng)       # start hot
    s = md.State(rng.uniform(0, 5, (n, 3)), v, np.zeros(n), [5.0] * 3)
    it = md.Integrator(None, dt=dt, kT=kT, tdamp=tdamp, sigma=1e-9)   # WCA range ~0
    K0 = s.kinetic()
    for _ in range(steps):
        it.step(s)
    g = 3 * n - 3
    Q = g * kT * tdamp ** 2

    def rhs(y):
        K, xi = y
        return np.array([-2 * xi * K, (2 * K - g * kT) / Q])
    y = np.array([K0, 0.0])
    h = dt / 20
    for _ in range(steps * 20):
        k1 = rhs(y); k2 = rhs(y + h / 2 * k1); k3 = rhs(y + h / 2 * k2); k4 = rhs(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert abs(s.kinetic() - y[0]) < 1e-3 * K0
    assert abs(s.xi - y[1]) < 1e-3 * max(1.0, abs(y[1]))


def test_nose_hoover_conserves_the_extended_energy_and_thermalises():
    rng = np.random.default_rng(4)
    x = lattice(4, 5.0, 0.2, rng)
    n = len(x)
    v = md.maxwell_velocities(n, 2.0, 1.0, rng)
    s = md.State(x, v, np.zeros(n), [5.0] * 3)
    it = md.Integrator(None, dt=0.002, kT=1.0, tdamp=0.1)
    it.forces(s)
    H0 = it.extended_energy(s)
    temps, drift = [], 0.0
    for k in range(3000):
        it.step(s)
        drift = max(drift, abs(it.extended_energy(s) - H0))
        if k >= 1000:
            temps.append(2 * s.kinetic() / (3 * n - 3))
    assert drift < 2e-3 * abs(H0)
    assert abs(np.mean(temps) - 1.0) < 0.06


def test_rdf_counts_match_brute_force():
    rng = np.random.default_rng(5)
    box = [6.0, 6.0, 6.0]
    x = rng.uniform(0, 6.0, (40, 3))
    a = np.arange(40) % 2 == 0
    h = md.rdf_counts(x, box, a, ~a, 3.0, 12)
    ref = np.zeros(12, dtype=np.int64)
    for i in np.nonzero(~a)[0]:
        for j in np.nonzero(a)[0]:
            d = x[j] - x[i]
            d -= 6.0 * np.round(d / 6.0)
            r = math.sqrt(d @ d)
            if r < 3.0:
                ref[int(r / 0.25)] += 1
    assert np.array_equal(h, ref)


def test_walls_closed_form_and_gradient():
    Lz = 6.0
    for d in (0.3, 0.45, 0.5, md.WCA_CUT * 0.5 - 1e-9, 0.6):
        x = np.array([[1.0, 1.0, d], [2.0, 2.0, 3.0]])
        U, F = md.walls(x, Lz)
        ref = 4 * ((0.5 / d) ** 12 - (0.5 / d) ** 6) + 1 if d < md.WCA_CUT * 0.5 else 0.0
        assert abs(U - ref) < 1e-12 * max(1.0, abs(ref))
        assert F[0, 2] >= 0.0                      # pushed away from the bottom wall
    x = np.array([[1.0, 1.0, 0.4], [2.0, 2.0, Lz - 0.42]])
    U, F = md.walls(x, Lz)
    h = 1e-7
    for i in range(2):
        e = np.zeros_like(x); e[i, 2] = h
        fd = -(md.walls(x + e, Lz)[0] - md.walls(x - e, Lz)[0]) / (2 * h)
        assert abs(fd - F[i, 2]) < 1e-5 * max(1.0, abs(F[i, 2]))
    assert F[1, 2] < 0.0


def test_slab_nve_is_reversible_and_keeps_ions_inside():
    rng = np.random.default_rng(6)
    box = [6.0, 6.0, 4.0]
    x = lattice(3, 4.0, 0.2, rng) + np.array([1.0, 1.0, 0.0])
    x[:, 2] = 0.6 + (x[:, 2] / 4.0) * 2.8
    n = len(x)
    v = md.maxwell_velocities(n, 1.0, 1.0, rng)
    s = md.State(x, v, np.zeros(n), box, slab=True)
    it = md.Integrator(None, dt=0.002)
    x0 = s.unwrapped().copy()
    for _ in range(200):
        it.step(s)
        assert np.all((s.x[:, 2] > 0) & (s.x[:, 2] < box[2]))
    s.v = -s.v
    for _ in range(200):
        it.step(s)
    assert np.abs(s.unwrapped() - x0).max() < 1e-8
    assert np.all(s.img[:, 2] == 0)


def test_hsma_driven_md_follows_the_ewald_driven_run():
    # The paper validates HSMA3D by MD of the Sec. 4.1 electrolyte against a
    # reference solver.  Here: the same start (ions on a jittered lattice at
    # the E1 volume fraction, l_B = 3.5, dt = 0.01, Nose-Hoover with damping
    # time 0.1) run twice through the oracle's MD loop, once with the oracle's
    # HSMA at the paper's accuracy setting (p = 10, N_m = 200, unmasked
    # 27-cell near set, relative force error about 3e-6) and once with the
    # Ewald sum.  A relative force error e moves a trajectory by about
    # e |F| t^2 / 2 before chaos amplifies it: with |F| up to ~30 kT/sigma and
    # t = 0.6 tau that is ~3e-5 sigma, so over 60 steps the two trajectories
    # must stay within 1e-4 sigma of each other; their Coulomb and total
    # energies agree to 1e-5 per step, and the cation-anion pair counts of
    # the RDF histogram are the same.
    from oracle import hsma as O
    lb = 3.5
    rng = np.random.default_rng(41)
    n_side = 5
    L = (n_side ** 3 / (3000 / 25.0 ** 3)) ** (1 / 3)      # E1 number density
    x0 = lattice(n_side, L, 0.2, rng)
    n = len(x0)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    q[-1] = 0.0                                             # 125 ions: one uncharged keeps it neutral
    v0 = md.maxwell_velocities(n, 1.0, 1.0, rng)
    box = [L, L, L]
    st = O.make_setup(box, 3, 10, 2000, n_monitor=200, sphere_mask=False, prefactor=lb)

    def hsma_coulomb(x, qq):
        out = O.evaluate(st, x, qq)
        return out["energy"], out["forces"]

    runs = []
    for coul in (hsma_coulomb, ewald_coulomb(box, lb)):
        s = md.State(x0, v0, q, box)
        it = md.Integrator(coul, dt=0.01, kT=1.0, tdamp=0.1)
        rows, hist = [], np.zeros(40, dtype=np.int64)
        for k in range(60):
            it.step(s)
            rows.append((s.U_c, it.extended_energy(s), s.kinetic()))
            if k % 10 == 9:
                hist += md.rdf_counts(s.x, box, q > 0, q < 0, 4.0, 40)
        runs.append((np.array(rows), s.unwrapped(), hist))
    (rh, xh, gh), (re, xe, ge) = runs
    assert np.abs(xh - xe).max() < 1e-4
    scale = np.abs(re[:, 0]).max()
    assert np.abs(rh[:, 0] - re[:, 0]).max() < 1e-5 * scale
    assert np.abs(rh[:, 1] - re[:, 1]).max() < 1e-5 * np.abs(re[:, 1]).max()
    assert np.array_equal(gh, ge)
