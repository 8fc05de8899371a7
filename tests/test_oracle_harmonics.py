"""Pins of the oracle's harmonic basis (Sec. 2.2, Eq. 5) to mathematics it does
not itself compute: orthonormality under an exact product quadrature, the
addition theorem with an independent Legendre routine, harmonicity by finite
differences and the z-derivative identity by finite differences."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import harmonics as H


def product_rule(n):
    # Gauss-Legendre in cos(theta) x trapezoid in phi: exact for degree < 2n
    t, w = npleg.leggauss(n)
    ph = 2 * math.pi * np.arange(2 * n) / (2 * n)
    T, P = np.meshgrid(np.arccos(t), ph, indexing="ij")
    W = np.outer(w, np.full(2 * n, 2 * math.pi / (2 * n)))
    return T.ravel(), P.ravel(), W.ravel()


@pytest.mark.parametrize("p", [1, 6, 10])
def test_orthonormal(p):
    T, P, W = product_rule(p + 2)
    Y = H.real_sph(p, T, P)
    G = Y.T @ (Y * W[:, None])
    assert np.abs(G - np.eye(H.nbasis(p))).max() < 1e-12


def test_addition_theorem():
    rng = np.random.default_rng(0)
    u = rng.normal(size=(20, 3)); u /= np.linalg.norm(u, axis=1)[:, None]
    v = rng.normal(size=(20, 3)); v /= np.linalg.norm(v, axis=1)[:, None]
    p = 10
    _, tu, pu = H.to_spherical(u)
    _, tv, pv = H.to_spherical(v)
    Yu, Yv = H.real_sph(p, tu, pu), H.real_sph(p, tv, pv)
    cosg = np.sum(u * v, axis=1)
    for n in range(p + 1):
        s = sum(Yu[:, H.idx(n, m)] * Yv[:, H.idx(n, m)] for m in range(-n, n + 1))
        c = np.zeros(n + 1); c[n] = 1.0
        ref = (2 * n + 1) / (4 * math.pi) * npleg.legval(cosg, c)
        assert np.abs(s - ref).max() < 1e-12


def test_solid_harmonics_are_harmonic_and_dz_identity():
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (15, 3))
    p, s, h = 8, 1.3, 1e-4
    S0 = H.solid(p, x, s)
    lap = -6 * S0
    for c in range(3):
        e = np.zeros(3); e[c] = h
        lap += H.solid(p, x + e, s) + H.solid(p, x - e, s)
    assert np.abs(lap / h ** 2).max() < 1e-5
    e = np.array([0, 0, 1e-6])
    fd = (H.solid(p, x + e, s) - H.solid(p, x - e, s)) / 2e-6
    assert np.abs(fd - H.solid_dz(p, x, s)).max() < 1e-8


def test_against_scipy_when_available():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(2)
    th = rng.uniform(0, math.pi, 30)
    ph = rng.uniform(-math.pi, math.pi, 30)
    Y = H.real_sph(7, th, ph)
    for n in range(8):
        for m in range(0, n + 1):
            c = sp.sph_harm_y(n, m, th, ph)      # complex, Condon-Shortley phase
            if m == 0:
                assert np.allclose(Y[:, H.idx(n, 0)], c.real, atol=1e-12)
            else:
                # |real combination| agrees with sqrt(2)|Re|, sqrt(2)|Im|
                assert np.allclose(np.abs(Y[:, H.idx(n, m)]), math.sqrt(2) * np.abs(c.real), atol=1e-12)
                assert np.allclose(np.abs(Y[:, H.idx(n, -m)]), math.sqrt(2) * np.abs(c.imag), atol=1e-12)


def test_cartesian_form_matches_angular_form():
    rng = np.random.default_rng(4)
    x = rng.uniform(-2, 2, (40, 3))
    for p in (1, 6, 10):
        a = H.solid(p, x, 1.7)
        b = H.solid_cart(p, x, 1.7)
        assert np.abs(a - b).max() < 1e-12 * max(1.0, np.abs(a).max())


def test_series_gradient_matches_finite_differences_and_dz_identity():
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (20, 3))
    p, s = 8, 1.3
    coeffs = rng.normal(size=H.nbasis(p) - 1)
    phi, grad = H.series_field(p, x, s, coeffs)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3); e[d] = h
        fd = (H.series_field(p, x + e, s, coeffs)[0] - H.series_field(p, x - e, s, coeffs)[0]) / (2 * h)
        assert np.abs(fd - grad[:, d]).max() < 1e-7 * max(1.0, np.abs(grad).max())
    dz = H.solid_dz(p, x, s)[:, 1:] @ coeffs        # the independent z-derivative
    assert np.abs(dz - grad[:, 2]).max() < 1e-12 * max(1.0, np.abs(dz).max())
