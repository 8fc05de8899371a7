"""Pins of the 2D fit's face rows (reading R5 of the oracle) against the exact
field of the dielectric slab (Sec. 2.1, Eq. 4).

The potential inside a neutral slab between two planar interfaces satisfies,
on each face, continuity of Phi and of eps dPhi/dz.  Outside there are no
charges, so every nonzero Fourier mode of Phi decays away from the slab and
dPhi_out/dn = -Lambda Phi with Lambda the Dirichlet-to-Neumann map (|h| per
mode); the zero mode carries no field for a neutral system.  With
eps_c : eps_out = (1 + g) : (1 - g) this gives, on each face,

    (1 + g) dPhi/dn + (1 - g) Lambda Phi = 0.

The exact slab field comes from the image-layer Ewald sum (oracle.ewald),
which is pinned elsewhere to brute force and closed forms.  Sampled on a
G x G grid, the discrete map Lambda_G differs from Lambda only by aliasing
of modes above the grid's Nyquist wavenumber; with every charge and image at
least a distance d from the face these carry exp(-|h| d), so the residual
falls quickly with G.  Planted mistakes in the row expression (the factors
(1 +- g) swapped, the bottom normal's sign flipped, |h| replaced by h^2) are
shown to break the pin.
"""
import math

import numpy as np
import pytest

from oracle import hsma
from oracle.ewald import slab_field

BOX = (4.0, 4.0, 4.0)
Q = np.array([1.0, -1.0, 2.0, -2.0, 1.0, -1.0])


def charges():
    # box-centred positions at least 1.5 from both faces (|z| <= 0.5, Lz = 4)
    rng = np.random.default_rng(3)
    n = len(Q)
    return np.column_stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(-0.5, 0.5, n)])


_FIELD = {}


def face_field(gt, gb, G):
    """Exact phi and dphi/dz on the top and bottom face grids."""
    key = (gt, gb, G)
    if key not in _FIELD:
        Lx, Ly, Lz = BOX
        out = []
        for pts in hsma.face_grid(BOX, G):
            phi, grad, _ = slab_field(pts, charges(), Q, Lx, Ly, Lz, gt, gb, tol=1e-16, chunk=4096)
            out.append((phi, grad[:, 2]))
        _FIELD[key] = out
    return _FIELD[key]


def residuals(gt, gb, G):
    """Relative RMS residual of the oracle's face rows on the exact field, per face."""
    Lx, Ly, _ = BOX
    res = []
    for f, g in ((0, gt), (1, gb)):
        phi, dz = face_field(gt, gb, G)[f]
        sn = hsma.FACE_SIGNS[f]
        r = hsma.dtn_rows(phi, dz, g, sn, Lx, Ly)
        # scale: the two terms of the row taken separately (correct factors)
        lam = hsma.dtn_lambda(phi.reshape(G, G), Lx, Ly).ravel()
        scale = math.sqrt(np.mean(((1.0 + g) * dz) ** 2) + np.mean(((1.0 - g) * lam) ** 2))
        res.append(float(np.sqrt(np.mean(r ** 2))) / scale)
    return res


@pytest.mark.parametrize("gt,gb", [(-0.95, -0.95), (0.0, 0.0), (0.6, 0.0), (0.95, 0.95)])
def test_face_rows_vanish_on_the_exact_slab_field(gt, gb):
    coarse = residuals(gt, gb, 12)
    fine = residuals(gt, gb, 20)
    for rc, rf in zip(coarse, fine):
        assert rf <= 1e-8
        assert rf < 1e-2 * rc          # aliasing error falls with the grid


def test_planted_mistakes_in_the_face_rows_are_seen(monkeypatch):
    gt, gb, G = 0.6, 0.0, 20
    assert max(residuals(gt, gb, G)) < 1e-8
    # (a) the factors (1 + g) and (1 - g) swapped (visible on the top face, g = 0.6)
    with monkeypatch.context() as m:
        m.setattr(hsma, "dtn_weights", lambda g, sn: ((1.0 - g) * sn, 1.0 + g))
        assert residuals(gt, gb, G)[0] > 1e-2
    # (b) the outward normal of the bottom face taken as +z
    with monkeypatch.context() as m:
        m.setattr(hsma, "FACE_SIGNS", (1.0, 1.0))
        assert residuals(gt, gb, G)[1] > 1e-2
    # (c) Lambda with |h| replaced by |h|^2
    def squared(field2d, Lx, Ly):
        n = field2d.shape[0]
        hx = 2.0 * math.pi * np.fft.fftfreq(n) * n / Lx
        hy = 2.0 * math.pi * np.fft.fftfreq(n) * n / Ly
        h2 = hx[:, None] ** 2 + hy[None, :] ** 2
        return np.real(np.fft.ifft2(np.fft.fft2(field2d) * h2))
    with monkeypatch.context() as m:
        m.setattr(hsma, "dtn_lambda", squared)
        r = residuals(gt, gb, G)
        assert r[0] > 1e-2 and r[1] > 1e-2


def test_dtn_map_of_a_plane_wave():
    # Lambda_G cos(h.x) = |h| cos(h.x) for every mode the grid resolves; a
    # non-square face catches a transposed axis
    Lx, Ly, G = 3.0, 5.0, 16
    xa = -0.5 * Lx + (np.arange(G) + 0.5) * (Lx / G)
    ya = -0.5 * Ly + (np.arange(G) + 0.5) * (Ly / G)
    X, Y = np.meshgrid(xa, ya, indexing="ij")
    for i, j in ((1, 0), (0, 1), (2, 3), (-3, 1), (7, -5)):
        hx, hy = 2 * math.pi * i / Lx, 2 * math.pi * j / Ly
        f = np.cos(hx * X + hy * Y)
        got = hsma.dtn_lambda(f, Lx, Ly)
        assert np.abs(got - math.hypot(hx, hy) * f).max() < 1e-13 * math.hypot(hx, hy) * G
        s = np.sin(hx * X + hy * Y)
        assert np.abs(hsma.dtn_lambda(s, Lx, Ly) - math.hypot(hx, hy) * s).max() < 1e-13 * math.hypot(hx, hy) * G
    assert np.abs(hsma.dtn_lambda(np.full((G, G), 2.5), Lx, Ly)).max() < 1e-14


@pytest.mark.parametrize("gt,gb", [(0.6, 0.0), (-0.95, -0.95)])
def test_fit_operator_uses_the_face_rows(gt, gb):
    # the design matrix's face blocks are the face rows of the basis, and P (built
    # with the transposed map for speed) equals pinv(D) times the explicit
    # right-hand side -w [face rows of Phi_B] for any check vector
    box, p, G = (6.0, 5.0, 4.0), 4, 8
    st = hsma.make_setup(box, 2, p, 100, gt, gb, dtn_grid=G)
    Lx, Ly, _ = box
    nm, nk = st.n_mon, int(np.sum(st.keep))
    wd = st.Rc / G
    from oracle import harmonics as H
    top, bot = hsma.face_grid(box, G)
    for f, pts in enumerate((top, bot)):
        g = (gt, gb)[f]
        B = H.solid(p, pts, st.Rc)[:, 1:]
        dB = H.solid_dz(p, pts, st.Rc)[:, 1:]
        blk = st.D[nk + f * G * G: nk + (f + 1) * G * G]
        assert np.allclose(blk, wd * hsma.dtn_rows(B, dB, g, hsma.FACE_SIGNS[f], Lx, Ly), rtol=0, atol=1e-13)
    U, sv, Vt = np.linalg.svd(st.D, full_matrices=False)
    keep = sv > hsma.SVD_RCOND * sv[0]
    pinv = (Vt.T[:, keep] / sv[keep]) @ U.T[keep]
    rng = np.random.default_rng(5)
    nc = len(st.check_pts)
    for _ in range(3):
        v = rng.normal(size=2 * nc)
        phi, dz = v[:nc], v[nc:]
        kidx = np.nonzero(st.keep)[0]
        rhs = [phi[nm + kidx] - phi[kidx]]
        for f in range(2):
            o = 2 * nm + f * G * G
            g = (gt, gb)[f]
            rhs.append(-wd * hsma.dtn_rows(phi[o:o + G * G], dz[o:o + G * G], g, hsma.FACE_SIGNS[f], Lx, Ly))
        A = pinv @ np.concatenate(rhs)
        assert np.allclose(st.P @ v, A, rtol=0, atol=1e-10 * np.abs(A).max())
