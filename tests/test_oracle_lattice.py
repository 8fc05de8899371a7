"""Pins of the oracle's Fibonacci lattice surface rule (Sec. 3.2: the rule
named by two adjacent Fibonacci numbers F_w < F, claimed to converge as
N_o^-6) to facts it does not compute itself: the lattice structure, closed-form
integrals of monomials and of an exponential over the sphere, the rate of
convergence, the single-layer identity the surface map rests on
(Sec. 2.2, third step), and the end result against the Ewald sum."""
import math

import numpy as np
import pytest

import workloads
from oracle import harmonics as H
from oracle import hsma as O
from oracle.ewald import ewald3d


def test_fibonacci_pairs_and_lattice_structure():
    assert O.fibonacci_pair(89) == (55, 89)          # the paper's default F_w, F
    assert O.fibonacci_pair(2584) == (1597, 2584)
    assert O.fibonacci_pair(13) == (8, 13)
    for M in (8, 12, 14, 90, 800, 2000):
        assert O.fibonacci_pair(M) is None
    with pytest.raises(O.OracleError):
        O.make_setup((10.0, 10.0, 10.0), 3, 6, 800, surface_rule=1)
    y, w = O.fibonacci_lattice(233, 2.5)
    assert np.allclose(np.linalg.norm(y, axis=1), 2.5, rtol=0, atol=1e-13)
    assert np.all(w > 0)
    # every longitude index k = j F_w mod F occurs once (gcd(F_w, F) = 1)
    ph = np.mod(np.arctan2(y[:, 1], y[:, 0]), 2 * math.pi)
    k = np.rint(ph / (2 * math.pi) * 233).astype(int) % 233
    assert sorted(k) == list(range(233))
    # polar angles increase with j and are symmetric about the equator
    assert np.all(np.diff(y[:, 2]) < 0)
    assert np.allclose(y[:, 2], -y[::-1, 2], rtol=0, atol=1e-13)


def test_monomial_integrals_over_the_sphere():
    # int x^a y^b z^c dS over the unit sphere: closed forms
    y, w = O.fibonacci_lattice(233, 1.0)
    X, Y, Z = y.T
    cases = [(np.ones_like(X), 4 * math.pi), (Z * Z, 4 * math.pi / 3), (X ** 4, 4 * math.pi / 5),
             (X * X * Y * Y, 4 * math.pi / 15), (Z ** 6, 4 * math.pi / 7),
             ((X * Y * Z) ** 2, 4 * math.pi / 105), (X * Y ** 3, 0.0), (X * Z, 0.0)]
    for f, ref in cases:
        assert abs(float(np.sum(w * f)) - ref) < 1e-10


def test_exponential_integral_and_convergence_rate():
    # int exp(a . y) dS = 4 pi sinh|a| / |a|; the error falls at least as F^-6
    a = np.array([0.8, -0.5, 1.1])
    na = float(np.linalg.norm(a))
    ref = 4 * math.pi * math.sinh(na) / na
    err = {}
    for F in (89, 144, 233):
        y, w = O.fibonacci_lattice(F, 1.0)
        err[F] = abs(float(np.sum(w * np.exp(y @ a))) - ref) / ref
    assert err[233] < 1e-10
    assert err[233] < err[89] * (89 / 233) ** 6


def test_harmonic_products_are_integrated_exactly():
    # int Y_nm Y_n'm' dS = delta for the real orthonormal harmonics (n, n' <= 8)
    y, w = O.fibonacci_lattice(987, 1.0)
    Y = H.solid(8, y, 1.0)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(len(G))).max() < 1e-12


def test_single_layer_identity():
    # int Y_nm(yhat) / |yhat - r| dS = 4 pi / (2n+1) |r|^n Y_nm(rhat) for |r| < 1,
    # the identity behind the surface charges
    p = 8
    r0 = np.array([[0.3, -0.4, 0.35]])
    y, w = O.fibonacci_lattice(1597, 1.0)
    Y = H.solid(p, y, 1.0)
    lhs = (w / np.linalg.norm(y - r0, axis=1)) @ Y
    n = np.array([n for n in range(p + 1) for _ in range(2 * n + 1)])
    rhs = 4 * math.pi / (2 * n + 1) * H.solid(p, r0, 1.0)[0]
    assert np.abs(lhs - rhs).max() < 1e-8


def test_lattice_rule_reaches_the_literal_sphere_accuracy():
    # the literal sphere of Sec. 3.2 (lambda = 2.6) at P = 10: with the lattice
    # rule the force error against Ewald is far below the golden-spiral rule's
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    L = c.box[0]
    xc = (x - L * np.floor(x / L)) - 0.5 * L
    Ee, _, ge = ewald3d(xc, q, c.box)
    Fe = -q[:, None] * ge

    def err(rule, M):
        out = O.evaluate(O.make_setup(c.box, 3, 10, M, lam=2.6, surface_rule=rule), x, q)
        F = out["forces"]
        return (abs(out["energy"] - Ee) / abs(Ee),
                math.sqrt(np.mean(np.sum((F - Fe) ** 2, 1)) / np.mean(np.sum(Fe ** 2, 1))))
    e1, f1 = err(1, 610)
    e0, f0 = err(0, 800)
    assert f1 < 1e-6 and e1 < 1e-6
    assert f1 < 0.1 * f0
