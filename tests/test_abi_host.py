"""CPU-only checks of the C-ABI library: it builds, loads and exports every
symbol include/hsma.h declares, and its host geometry (sphere, image shifts,
check points, and the composite fit + surface map of Sec. 2.2) agrees with the
oracle's.  No GPU and no device call."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2104_05260_gb300 import build
    build.build()
    import paper_2104_05260_gb300 as P
    P.lib()
    return P


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hsma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hsma_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(P):
    names = declared_symbols()
    assert "hsma_eval" in names and "hsma_submit" in names and len(names) >= 14
    L = P.lib()
    for n in names:
        assert hasattr(L, n), n
        assert n in P.SIGNATURES, n


def test_binding_has_no_fallback(P, monkeypatch):
    monkeypatch.setattr(P, "_lib", None)
    monkeypatch.setattr(P, "LIB_PATH", "/nonexistent/libhsma.so")
    with pytest.raises(RuntimeError):
        P.lib()


def sizes(P, box, dims, p, M, **kw):
    s = P.hsma_geometry_array(box, dims, p, M, "sizes", 8, **kw)
    return dict(n_check=int(s[0]), nv=int(s[1]), nA=int(s[2]), rank=int(s[3]),
                n_shift=int(s[4]), Rc=s[5], Rs=s[6], Rs2=s[7])


@pytest.mark.parametrize("box,p,M,lam", [((10.0, 10.0, 10.0), 6, 800, 0.0),
                                         ((7.0, 9.0, 11.0), 8, 1000, 0.0),
                                         ((10.0, 10.0, 10.0), 10, 4000, 2.6)])
def test_geometry_3d_matches_oracle(P, box, p, M, lam):
    from oracle import hsma
    st = hsma.make_setup(box, 3, p, M, lam=(lam or None))
    sz = sizes(P, box, 3, p, M, lam=lam)
    assert sz["Rs2"] == st.Rs2 and sz["Rs"] == st.Rs     # bitwise: same FP64 op order
    assert sz["rank"] == sz["nA"] == (p + 1) ** 2 - 1
    assert sz["n_shift"] == len(st.shifts)
    sh = P.hsma_geometry_array(box, 3, p, M, "shifts", 5 * sz["n_shift"], lam=lam).reshape(-1, 5)
    assert sorted(map(tuple, sh)) == sorted(map(tuple, st.shifts))   # bitwise
    cp = P.hsma_geometry_array(box, 3, p, M, "check_points", 3 * sz["n_check"], lam=lam)
    assert np.allclose(cp.reshape(-1, 3), st.check_pts, rtol=0, atol=1e-12)
    ys = P.hsma_geometry_array(box, 3, p, M, "surface_points", 3 * M, lam=lam).reshape(-1, 3)
    assert np.allclose(ys, st.ysurf, rtol=0, atol=1e-12)
    T = P.hsma_geometry_array(box, 3, p, M, "T", M * sz["nv"], lam=lam).reshape(M, sz["nv"])
    To = st.W @ st.P
    assert np.abs(T - To).max() < 1e-9 * np.abs(To).max()


@pytest.mark.parametrize("gam", [(-0.95, -0.95), (0.0, 0.0), (0.95, 0.95), (0.5, -0.3)])
def test_geometry_2d_matches_oracle(P, gam):
    from oracle import hsma
    box, p, M, G = (20.0, 20.0, 10.0), 6, 600, 16
    st = hsma.make_setup(box, 2, p, M, gam[0], gam[1], dtn_grid=G)
    sz = sizes(P, box, 2, p, M, gamma_top=gam[0], gamma_bot=gam[1], G=G)
    assert sz["Rs2"] == st.Rs2
    assert sz["rank"] == (p + 1) ** 2 - 1
    kw = dict(gamma_top=gam[0], gamma_bot=gam[1], G=G)
    sh = P.hsma_geometry_array(box, 2, p, M, "shifts", 5 * sz["n_shift"], **kw).reshape(-1, 5)
    assert sorted(map(tuple, sh)) == sorted(map(tuple, st.shifts))
    cp = P.hsma_geometry_array(box, 2, p, M, "check_points", 3 * sz["n_check"], **kw)
    assert np.allclose(cp.reshape(-1, 3), st.check_pts, rtol=0, atol=1e-12)
    T = P.hsma_geometry_array(box, 2, p, M, "T", M * sz["nv"], **kw).reshape(M, sz["nv"])
    To = st.W @ st.P
    assert T.shape == To.shape
    assert np.abs(T - To).max() < 1e-8 * np.abs(To).max()


@pytest.mark.parametrize("dims", [3, 2])
def test_geometry_gradient_rows_match_oracle(P, dims):
    # the gradient-periodicity rows: the host builds their basis gradients by
    # an analytic recursion, the oracle by complex steps of the polynomial form
    from oracle import hsma
    box = (10.0, 10.0, 10.0) if dims == 3 else (20.0, 20.0, 10.0)
    p, M, G, w = 6, 600, 16, 0.1
    st = hsma.make_setup(box, dims, p, M, 0.4, -0.2, dtn_grid=G, grad_rows=True, grad_weight=w)
    kw = dict(gamma_top=0.4, gamma_bot=-0.2, G=G, grad_weight=w)
    sz = sizes(P, box, dims, p, M, **kw)
    assert sz["rank"] == (p + 1) ** 2 - 1
    assert sz["nv"] == st.P.shape[1] == sizes(P, box, dims, p, M, G=G)["nv"] + 6 * st.n_mon
    T = P.hsma_geometry_array(box, dims, p, M, "T", M * sz["nv"], **kw).reshape(M, sz["nv"])
    To = st.W @ st.P
    assert np.abs(T - To).max() < 1e-8 * np.abs(To).max()
    # the rows change the map (the gradient block is not empty)
    assert np.abs(To[:, -6 * st.n_mon:]).max() > 1e-3 * np.abs(To).max()


@pytest.mark.parametrize("dims,M", [(3, 987), (2, 610)])
def test_geometry_fibonacci_lattice_matches_oracle(P, dims, M):
    # the surface rule of Sec. 3.2 (F_w/F lattice): points and the weighted map
    from oracle import hsma
    box = (10.0, 10.0, 10.0) if dims == 3 else (20.0, 20.0, 10.0)
    p, G = 6, 16
    st = hsma.make_setup(box, dims, p, M, 0.4, -0.2, dtn_grid=G, surface_rule=1)
    kw = dict(gamma_top=0.4, gamma_bot=-0.2, G=G, surface_rule=1)
    sz = sizes(P, box, dims, p, M, **kw)
    ys = P.hsma_geometry_array(box, dims, p, M, "surface_points", 3 * M, **kw).reshape(-1, 3)
    assert np.allclose(ys, st.ysurf, rtol=0, atol=1e-12)
    T = P.hsma_geometry_array(box, dims, p, M, "T", M * sz["nv"], **kw).reshape(M, sz["nv"])
    To = st.W @ st.P
    assert np.abs(T - To).max() < 1e-8 * np.abs(To).max()
    # a different map from the golden-spiral rule at the same M
    T0 = P.hsma_geometry_array(box, dims, p, M, "T", M * sz["nv"], gamma_top=0.4, gamma_bot=-0.2,
                               G=G).reshape(M, sz["nv"])
    assert np.abs(T - T0).max() > 1e-2 * np.abs(To).max()
    with pytest.raises(P.HSMAError):
        P.hsma_geometry_array(box, dims, p, M + 1, "sizes", 8, surface_rule=1)   # not Fibonacci


def test_geometry_rejects_bad_arguments(P):
    with pytest.raises(P.HSMAError):
        P.hsma_geometry_array((10, 10, 10), 3, 6, 10, "sizes", 8)       # M < (p+1)^2
    with pytest.raises(P.HSMAError):
        P.hsma_geometry_array((10, 10, 10), 4, 6, 800, "sizes", 8)      # dims
    with pytest.raises(P.HSMAError):
        P.hsma_geometry_array((10, 10, 10), 3, 6, 800, "sizes", 8, lam=0.9)
    with pytest.raises(P.HSMAError):
        P.hsma_geometry_array((20, 20, 10), 2, 6, 800, "sizes", 8, gamma_top=1.2)
    # size limits: p <= 40 and M (p+1)^2 <= 2^31, refused before any
    # allocation (here and in hsma_create, which checks before any CUDA call)
    m_max = 2 ** 31 // 41 ** 2
    for p, M in ((41, 2000), (40, m_max + 1), (6, 2 ** 31 - 1)):
        with pytest.raises(P.HSMAError) as e:
            P.hsma_geometry_array((10, 10, 10), 3, p, M, "sizes", 8)
        assert e.value.code == -1, (p, M)
        with pytest.raises(P.HSMAError) as e:
            P.hsma_create((10, 10, 10), 3, p, M)
        assert e.value.code == -1, (p, M)
    # an output too small for the composite operator is refused before it is formed
    with pytest.raises(P.HSMAError) as e:
        P.hsma_geometry_array((10, 10, 10), 3, 6, 800, "T", 10)
    assert e.value.code == -1
