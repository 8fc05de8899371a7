"""Pins of the Ewald ground truth (Sec. 2.1, Eq. 3 and Eq. 4) to facts that do
not come from the oracle itself: a tabulated lattice constant, brute-force
lattice sums, derived closed forms, finite differences and invariances."""
import math
import os

import numpy as np
import pytest

from oracle.ewald import (ewald3d, ewald2d_field, slab_ewald, image_factor,
                          image_z, slab_lmax)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, *v = line.split()
            out[k] = v
    return out


def nacl(L):
    pos, q = [], []
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                pos.append([sx * L / 4, sy * L / 4, sz * L / 4])
                q.append(sx * sy * sz)
    return np.array(pos), np.array(q, float)


def test_madelung_constant():
    alpha = float(golden("madelung_nacl.txt")["alpha"][0])
    for L in (2.0, 7.0):
        pos, q = nacl(L)
        E, phi, grad = ewald3d(pos, q, [L, L, L])
        a = L / 2
        # 4 ion pairs in the cell
        assert abs(-E * a / 4 - alpha) < 1e-12
        assert np.abs(grad).max() < 1e-12      # every ion sits at a centre of symmetry


def brute3d(pos, q, box, K):
    r = np.arange(-K, K + 1)
    sh = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3) * box
    E = 0.0
    for i in range(len(q)):
        d = pos[None, :, :] + sh[:, None, :] - pos[i]
        rr = np.sqrt((d * d).sum(-1))
        rr[np.all(sh == 0, axis=1), i] = np.inf
        E += 0.5 * q[i] * np.sum(q[None, :] / rr)
    return E


def test_ewald3d_vs_brute_force_cubes():
    # a neutral cell with zero dipole: cube-ordered sums converge to the
    # tin-foil value with an error ~ 1/K^2 (quadrupole shells)
    rng = np.random.default_rng(3)
    box = np.array([2.0, 2.5, 3.0])
    a = rng.uniform(-0.4, 0.4, (2, 3)) * box
    pos = np.vstack([a, -a])
    q = np.array([1.0, -1.0, 1.0, -1.0])
    Ee = ewald3d(pos, q, box)[0]
    K1, K2 = 12, 18
    E1, E2 = brute3d(pos, q, box, K1), brute3d(pos, q, box, K2)
    Einf = (K2 ** 2 * E2 - K1 ** 2 * E1) / (K2 ** 2 - K1 ** 2)
    assert abs(E2 - Ee) > 1e-5                    # the raw sum is still off
    assert abs(Einf - Ee) < 2e-6 * abs(Ee)


def random_cell(seed=0, N=6, box=(3.0, 3.5, 4.0)):
    rng = np.random.default_rng(seed)
    box = np.array(box)
    pos = rng.uniform(-0.5, 0.5, (N, 3)) * box
    q = np.array([1, -1, 2, -2, 1, -1.0])[:N]
    return pos, q, box


def test_ewald3d_force_is_minus_energy_gradient():
    pos, q, box = random_cell()
    E, phi, g = ewald3d(pos, q, box)
    h = 1e-5
    for i in range(3):
        for c in range(3):
            p = pos.copy(); p[i, c] += h
            Ep = ewald3d(p, q, box)[0]
            p = pos.copy(); p[i, c] -= h
            Em = ewald3d(p, q, box)[0]
            assert abs(-(Ep - Em) / (2 * h) - (-q[i] * g[i, c])) < 1e-7


def test_ewald3d_splitting_and_invariances():
    pos, q, box = random_cell(1)
    E0 = ewald3d(pos, q, box)[0]
    assert abs(ewald3d(pos, q, box, rcut=2.2)[0] - E0) < 1e-12
    # translation (with wrap) and permutation
    t = np.array([0.37, -1.2, 2.9])
    E1 = ewald3d(pos + t, q, box)[0]
    perm = np.array([3, 0, 5, 1, 4, 2])
    E2 = ewald3d(pos[perm], q[perm], box)[0]
    assert abs(E1 - E0) < 1e-12 and abs(E2 - E0) < 1e-12


def brute2d(pos, q, Lx, Ly, K):
    r = np.arange(-K, K + 1)
    gx, gy = np.meshgrid(r, r, indexing="ij")
    m = (gx ** 2 + gy ** 2) <= K * K
    sh = np.stack([gx[m] * Lx, gy[m] * Ly, 0 * gx[m]], -1).astype(float)
    E = 0.0
    for i in range(len(q)):
        d = pos[None, :, :] + sh[:, None, :] - pos[i]
        rr = np.sqrt((d * d).sum(-1))
        rr[np.all(sh == 0, axis=1), i] = np.inf
        E += 0.5 * q[i] * np.sum(q[None, :] / rr)
    return E


def test_slab_gamma0_vs_brute_force_discs():
    # gamma = 0 is the plain 2D-periodic slab (no images).  Disc-ordered sums of
    # neutral cells converge like 1/K; extrapolate in 1/K.
    rng = np.random.default_rng(5)
    Lx, Ly, Lz = 2.0, 2.5, 1.5
    pos = rng.uniform(-0.5, 0.5, (4, 3)) * np.array([Lx, Ly, Lz])
    q = np.array([1.0, -1.0, 2.0, -2.0])
    E, phi, g, lmax = slab_ewald(pos, q, Lx, Ly, Lz, 0.0, 0.0)
    assert lmax == 0
    Ks = [100, 150, 200, 300]
    Eb = [brute2d(pos, q, Lx, Ly, K) for K in Ks]
    c = np.polyfit([1.0 / K for K in Ks], Eb, 2)
    assert abs(Eb[-1] - E) > 1e-4
    assert abs(c[-1] - E) < 1e-5 * abs(E)


def slab_cell(seed=1):
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = 3.0, 3.5, 2.0
    pos = rng.uniform(-0.5, 0.5, (6, 3)) * np.array([Lx, Ly, Lz])
    q = np.array([1, -1, 2, -2, 1, -1.0])
    return pos, q, Lx, Ly, Lz


def test_slab_gamma_plus_one_is_half_the_doubled_box():
    # gamma_up = gamma_low = 1: the image series is the 3D-periodic system of
    # period 2 Lz holding each charge and its mirror z' = Lz - z (zero z-dipole),
    # so the slab energy is half the doubled box's tin-foil Ewald energy.
    pos, q, Lx, Ly, Lz = slab_cell()
    E, phi, g, _ = slab_ewald(pos, q, Lx, Ly, Lz, 1.0, 1.0)
    mir = pos.copy(); mir[:, 2] = Lz - pos[:, 2]
    E3, _, g3 = ewald3d(np.vstack([pos, mir]), np.concatenate([q, q]), [Lx, Ly, 2 * Lz])
    assert abs(E - 0.5 * E3) < 1e-12 * abs(E3)
    assert np.abs(g - g3[:6]).max() < 1e-11


def test_slab_gamma_minus_one_planar_sum():
    # gamma = -1: the mirror charges flip sign and the doubled cell carries a
    # z-dipole M_z.  A lattice summed layer by layer in z (which the image
    # series is) exceeds the tin-foil value by 2 pi M_z^2 / V.
    pos, q, Lx, Ly, Lz = slab_cell(2)
    E, _, _, _ = slab_ewald(pos, q, Lx, Ly, Lz, -1.0, -1.0)
    mir = pos.copy(); mir[:, 2] = Lz - pos[:, 2]
    P = np.vstack([pos, mir]); Q = np.concatenate([q, -q])
    E3 = ewald3d(P, Q, [Lx, Ly, 2 * Lz])[0]
    Mz = float(Q @ P[:, 2]); Vd = Lx * Ly * 2 * Lz
    assert abs(E - 0.5 * (E3 + 2 * math.pi * Mz ** 2 / Vd)) < 1e-12 * abs(E)


def test_slab_single_interface_is_one_mirror():
    # only the top interface polarisable (gamma_low = 0): the exact solution is
    # the charges plus one mirror image gamma*q at Lz - z, i.e. the reflection
    # across z = +Lz/2.  Built here without image_factor / image_z.
    pos, q, Lx, Ly, Lz = slab_cell(3)
    gam = 0.6
    E, phi, g, _ = slab_ewald(pos, q, Lx, Ly, Lz, gam, 0.0)
    mir = pos.copy(); mir[:, 2] = Lz - pos[:, 2]
    rc = 0.5 * min(Lx, Ly) + 0.5 * Lz
    p1, g1 = ewald2d_field(pos, pos, q, Lx, Ly, rc, exclude=np.arange(6))
    p2, g2 = ewald2d_field(pos, mir, gam * q, Lx, Ly, rc)
    assert np.abs(phi - (p1 + p2)).max() < 1e-11
    assert np.abs(g - (g1 + g2)).max() < 1e-11
    # and the printed (unswapped) factor would put it on the wrong interface
    assert image_factor(1, +1, gam, 0.0) == gam
    assert image_z(0.3, 1, +1, Lz) == Lz - 0.3


def test_slab_force_is_minus_energy_gradient():
    pos, q, Lx, Ly, Lz = slab_cell(4)
    gu, gl = 0.7, -0.4
    E, phi, g, lmax = slab_ewald(pos, q, Lx, Ly, Lz, gu, gl)
    # charge 0 sits 0.05 from the top wall (force ~ -78): central differences
    # with h = 1e-6 keep the O(h^2) truncation below 1e-7 relative
    h = 1e-6
    for i in range(2):
        for c in range(3):
            p = pos.copy(); p[i, c] += h
            Ep = slab_ewald(p, q, Lx, Ly, Lz, gu, gl, lmax=lmax)[0]
            p = pos.copy(); p[i, c] -= h
            Em = slab_ewald(p, q, Lx, Ly, Lz, gu, gl, lmax=lmax)[0]
            F = -q[i] * g[i, c]
            assert abs(-(Ep - Em) / (2 * h) - F) < 1e-7 * max(1.0, abs(F))


def test_slab_splitting_translation_and_truncation():
    pos, q, Lx, Ly, Lz = slab_cell(5)
    gu = gl = 0.9
    E0, _, _, lmax = slab_ewald(pos, q, Lx, Ly, Lz, gu, gl)
    assert abs(slab_ewald(pos, q, Lx, Ly, Lz, gu, gl, rcut=3.1)[0] - E0) < 1e-12
    t = np.array([0.77, -2.1, 0.0])
    assert abs(slab_ewald(pos + t, q, Lx, Ly, Lz, gu, gl)[0] - E0) < 1e-12
    assert abs(slab_ewald(pos, q, Lx, Ly, Lz, gu, gl, lmax=lmax + 4)[0] - E0) < 1e-13
    assert slab_lmax(0.0, 0.0, Lx, Ly, Lz) == 0
