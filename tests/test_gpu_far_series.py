"""GPU parity of the direct-series far field (option far_field = 1) against
the oracle's series evaluation (the fitted expansion of Sec. 2.2, Eq. 5,
summed at each particle instead of through the surface charges of Eq. 8).

Tolerances: energy error <= 1e-6 of |E| (FP64) and <= 1e-5 of the energy
scale 1/2 sum |q_i Phi_i| (FP32 pair arithmetic, whose rounding scales with
it; the total can nearly cancel); per-ion forces and potentials by relative
RMS.  The images in B are the same integer set.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import hsma as O

pytestmark = pytest.mark.gpu

E_TOL = {0: 1e-6, 1: 1e-5}
F_TOL = {0: 1e-6, 1: 2e-5}


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



def check_series(P, c, x, q, prec, st=None, **opt):
    st = st or O.make_setup(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], lam=c.lam,
                            dtn_grid=c.dtn_grid, **{k: v for k, v in opt.items() if k == "n_monitor"})
    ref = O.evaluate(st, x, q, far="series")
    h = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=prec, far_field=1, **opt)
    E, F, pot = h.eval(x, q, potential=True)
    assert h.info("far_field") == 1 and h.info("far_chunks") == 1
    assert int(h.info("Ns")) == ref["Ns"]
    # FP32 rounding scales with the energy scale 1/2 sum |q_i Phi_i|, not with
    # the (possibly nearly cancelling) total, so the FP32 path is judged there
    scale = abs(ref["energy"]) if prec == 0 else 0.5 * float(np.sum(np.abs(ref["q"] * ref["phi"])))
    assert abs(E - ref["energy"]) <= E_TOL[prec] * scale, (E, ref["energy"], scale)
    assert frms(F, ref["forces"]) <= F_TOL[prec]
    assert fmax(F, ref["forces"]) <= FMAX * F_TOL[prec], fmax(F, ref["forces"])
    assert pot_err(pot, ref["phi"]) <= F_TOL[prec]
    if prec == 0:
        # the coefficients the series kernel consumes (FP32 check sums perturb
        # the high orders, which the fit amplifies; there only the field counts)
        A = h.array("coeffs", len(ref["A"]))
        assert np.abs(A - ref["A"]).max() <= 1e-9 * np.abs(ref["A"]).max()
    h.close()
    return E, F, ref


@pytest.mark.parametrize("prec", [0, 1])
def test_series_cfg1(P, prec):
    c = workloads.case(1)                          # N = 1000, L = 10, p = 6, M = 800
    x, q = workloads.electrolyte(c)
    check_series(P, c, x, q, prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N", [2, 257, 1001])
def test_series_ragged_sizes(P, prec, N):
    L = 10.0 * (N / 1000) ** (1 / 3)
    val = (1, -1) if N % 2 == 0 else (2, -1)
    c = workloads.small_case(N, dims=3, box=(L, L, L), p=4, M=200, valences=val, seed=N)
    x, q = workloads.electrolyte(c)
    check_series(P, c, x, q, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_series_high_order(P, prec):
    # p = 16: 288 coefficients, (2m-1)!! up to 31!! ~ 1.9e17 folded into the
    # host table, so the FP32 recursion stays in range
    L = 6.0
    c = workloads.small_case(300, dims=3, box=(L, L, 1.5 * L), p=16, M=1200, seed=21)
    x, q = workloads.electrolyte(c)
    check_series(P, c, x, q, prec, n_monitor=700)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("gam", [(-0.95, -0.95), (0.95, 0.0)])
def test_series_2d(P, prec, gam):
    c = workloads.small_case(300, dims=2, box=(20.0, 20.0, 10.0), p=6, M=600, gammas=gam,
                             G=24, seed=13)
    x, q = workloads.electrolyte(c)
    check_series(P, c, x, q, prec, dtn_grid=24)


def test_series_and_surface_agree_and_switch(P):
    # the same handle switched between the two far fields: they differ by the
    # surface quadrature's error only, and switching back reproduces the first
    # result bit for bit
    c = workloads.case(1)
    x, q = workloads.electrolyte(c)
    h = P.HSMA(c.box, 3, c.p, c.M, precision=0)
    E0, F0, _ = h.eval(x, q, potential=True)
    h.set_option("far_field", 1)
    E1, F1, _ = h.eval(x, q, potential=True)
    h.set_option("far_field", 0)
    E2, F2, _ = h.eval(x, q, potential=True)
    h.close()
    assert E2 == E0 and np.array_equal(F2, F0)
    assert rel(E1, E0) <= 1e-4 and frms(F1, F0) <= 1e-3
