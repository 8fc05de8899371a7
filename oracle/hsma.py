"""CPU HSMA3D / HSMA2D, step by step (TEST INFRASTRUCTURE).

This is the parity target of the CUDA path.  It follows Sec. 2.2 in the
paper's order, in plain FP64 with sums in fixed index order:

 1. Near set (Sec. 2.2, first step): every periodic image -- and in 2D every
    dielectric reflection image of Sec. 2.1, Eq. 4 -- of every source whose
    position lies inside the auxiliary sphere B of radius R_s.
 2. Split (Sec. 2.2, Eq. 5): Phi = Phi_B + sum_{n<=P} A_n^m r^n Y_n^m.
 3. Fit (Sec. 2.2, Eq. 6): the A_n^m minimise || M A - Y || over monitoring
    points; M depends only on geometry, Y only on Phi_B at the points.
 4. Surface mapping (Sec. 2.2, third step): the harmonic series is replaced by
    M point charges on the sphere (a quadrature of a single-layer integral).
 5. Final sum (Sec. 2.2, last step): near images + surface charges onto the
    particles, done directly.
 6. Energy and force (Sec. 3.1): E = 1/2 sum_i q_i Phi(r_i), F_i = -q_i grad Phi(r_i).

Readings of passages the paper leaves open (each is also listed in the design
notes of the repository):

 R1 Self term: Phi(r_i) omits only the k = 0 (and, in 2D, l = 0) copy of i;
    the periodic and reflection images of i are kept.
 R2 Sphere: B is centred on the box centre, R_c is half the box diagonal (B
    circumscribes the cell, Sec. 2.2) and R_s = lambda R_c (Sec. 3.2).  An image
    is in B when |x|^2 < R_s^2, evaluated in FP64 in the order
    ((x*x + y*y) + z*z); a tie counts as outside.
 R3 Surface points: M points of the spherical Fibonacci (golden spiral) set on
    radius R_s, z_m = 1 - (2m+1)/M, phi_m = 2 pi m / golden, equal weights
    4 pi R_s^2 / M.  (The paper's F_w/F lattice rule cannot produce an
    arbitrary M.)
 R4 3D fit operator: periodicity of the potential.  N_m golden-spiral points
    r_c on radius R_c; w(r) = r - L o rnd(r/L) with rnd rounding half away
    from zero.  Row: sum A [b(r_c) - b(w(r_c))] = Phi_B(w(r_c)) - Phi_B(r_c),
    b_nm = (r/R_c)^n Y_nm.  A_0^0 cancels and is dropped (exact for neutral
    systems).  Solved with an SVD pseudo-inverse, relative cut-off 1e-13.
 R5 2D fit operator: rows of R4 with x, y wrapped only (rows with w = r_c are
    dropped), plus rows of the dielectric (Dirichlet-to-Neumann) condition on a
    G x G periodic grid on each face z = +-Lz/2:
        (1 + g) dPhi/dn + (1 - g) Lambda_G Phi = 0
    with dn the outward normal derivative, g that face's gamma and Lambda_G the
    periodic discrete DtN map (2D DFT, multiply by |h|, inverse DFT).  These
    rows are weighted by R_c / G (a grid-size-independent surface average in
    potential units).  The face rows are pinned to the exact slab field: on
    the image-series Ewald potential of a neutral slab they vanish up to the
    grid's aliasing (residual below 1e-8 of the terms, falling with G), and
    swapped (1 +- g), a flipped normal or |h|^2 for |h| break that pin.  The
    paper's own discretisation of the DtN integral (the 2D-dilation formula)
    is not available; this periodic-grid reading stands in for it.
 R6 Surface charges: the single layer sigma = sum A_nm (2n+1) R_s^(n-1)/(4 pi) Y_nm
    reproduces sum A_nm r^n Y_nm inside B (Laplace expansion of 1/|r - y|), so
    Q_m = sum A_nm (2n+1) R_s^(n+1) / M Y_nm(y_m / R_s).
 R7 Image factors: Sec. 2.1, Eq. 4 with g_up/g_low in gamma_l^+ swapped (the
    first upper image reflects across the top interface).  See ``ewald``.
 R8 Neutrality: |sum q| > 1e-10 sum |q| is an error; otherwise the residual is
    removed as q_i -= sum q / N.
 R12 Unmasked near set (optional): every image of every shift of the table is
    near, whether inside B or not (3D: the full 27 cells at lambda <= sqrt 3).
    The far sources then start at 1.5 cells from the centre, so the series of
    Eq. 5 converges faster inside the circumsphere, at about 4.5 times the
    near-field cost.  The fit and the surface map are unchanged.
 R13 Gradient-periodicity rows (optional, off by default; not in the paper's
    fit): for every periodic row of R4/R5 three more rows, one per Cartesian
    component d, require the field to be periodic as well:
        w_g sum A [d_d b(r_c) - d_d b(w(r_c))] = w_g [d_d Phi_B(w(r_c)) - d_d Phi_B(r_c)]
    with weight w_g = grad_weight * R_c (length units, so these rows are in
    potential units like those of R4).  They are appended after all other rows;
    the raw check vector gains d_x, d_y, d_z Phi_B at the 2 N_m monitoring
    points and wraps.
 R18 Fibonacci lattice surface rule (optional, surface_rule=1; Sec. 3.2 names
    the rule by two adjacent Fibonacci numbers F_w < F and claims N_o^-6
    convergence): M = F points, F_w the Fibonacci number before F.  The
    rank-1 lattice u_j = (j + 1/2)/F, s_j = (j F_w mod F)/F on the unit
    square is mapped to the sphere by theta = pi psi(u), phi = 2 pi s, with
    the periodising map psi(u) = u^3 (10 - 15 u + 6 u^2), psi'(u) =
    30 u^2 (1 - u)^2.  The weight of point j is the Jacobian over F,
        w_j = 2 pi^2 psi'(u_j) sin(theta_j) / F   (unit sphere),
    and R6 becomes Q_j = sum A_nm (2n+1) R_s^(n+1) w_j / (4 pi) Y_nm(yhat_j).
    The integrand's periodic extension in u has its first jump in the fifth
    derivative, so the rule converges as F^-6 on smooth integrands.

Coordinates at the API: 3D box [0,Lx)x[0,Ly)x[0,Lz) (positions are wrapped);
2D slab [0,Lx)x[0,Ly)x(0,Lz) (x, y wrapped; z must be inside).  Internally
everything is box-centred: x_c = (x - L floor(x/L)) - L/2.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import harmonics as H
from .ewald import image_factor

GOLDEN = (1.0 + math.sqrt(5.0)) / 2.0
NEUTRAL_TOL = 1e-10
SVD_RCOND = 1e-13
GRAD_WEIGHT = 0.1        # R13: w_g / R_c


class OracleError(ValueError):
    pass


def rnd_half_away(x):
    """Round half away from zero (R4)."""
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def fibonacci_pair(M):
    """(F_w, F) with F = M for a Fibonacci number M >= 13 (R18), else None."""
    a, b = 8, 13
    while b < M:
        a, b = b, a + b
    return (a, b) if b == M else None


def fibonacci_lattice(M, radius):
    """Fibonacci lattice rule on the sphere (R18): M points of the radius and
    their weights on the unit sphere (summing to 4 pi up to O(M^-6))."""
    Fw, F = fibonacci_pair(M)
    j = np.arange(F, dtype=np.int64)
    u = (j + 0.5) / F
    s = ((j * Fw) % F) / F
    psi = u ** 3 * (10.0 - 15.0 * u + 6.0 * u * u)
    dpsi = 30.0 * u * u * (1.0 - u) ** 2
    th = math.pi * psi
    ph = 2.0 * math.pi * s
    y = radius * np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=-1)
    w = 2.0 * math.pi ** 2 * dpsi * np.sin(th) / F
    return y, w


def golden_spiral(n, radius):
    """Spherical Fibonacci point set (R3): n points on a sphere of the radius."""
    m = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * m + 1.0) / n
    ph = 2.0 * math.pi * m / GOLDEN
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return radius * np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=-1)


# ---------------------------------------------------------------------------
# Set-up: everything that depends on geometry only (the paper's "Init")
# ---------------------------------------------------------------------------
@dataclass
class Setup:
    dims: int
    box: tuple
    p: int
    M: int
    lam: float
    n_monitor: int
    gamma_top: float
    gamma_bot: float
    dtn_grid: int
    prefactor: float
    Rc: float = 0.0
    Rs: float = 0.0
    Rs2: float = 0.0
    shifts: np.ndarray = field(default=None)   # (S, 5): sx, sy, zsign, zoff, factor
    check_pts: np.ndarray = field(default=None)  # targets of the check-point sum
    n_mon: int = 0
    keep: np.ndarray = field(default=None)     # rows kept (2D periodic rows)
    P: np.ndarray = field(default=None)        # raw check values -> scaled A (n >= 1)
    W: np.ndarray = field(default=None)        # scaled A -> surface charges
    ysurf: np.ndarray = field(default=None)    # (M, 3) surface points
    rank: int = 0
    sing: np.ndarray = field(default=None)
    grad_rows: bool = False                    # R13
    grad_weight: float = 0.0
    sphere_mask: bool = True                   # R2 (False: R12)
    surface_rule: int = 0                      # R3 (1: R18)
    wsurf: np.ndarray = field(default=None)    # (M,) R18 weights on the unit sphere
    D: np.ndarray = field(default=None)        # the fit's design matrix (rows as in P's comment)


def shift_table(dims, box, Rs, gamma_top=0.0, gamma_bot=0.0):
    """Image shifts whose cell can reach inside B (R2, R7).

    Each row is (sx, sy, zsign, zoff, factor): the image of a centred source
    (x, y, z) with charge q is (x + sx, y + sy, zsign * z + zoff) with charge
    factor * q.  3D: k in [-K, K]^3 with K_d = ceil(R_s / L_d - 1/2).  2D:
    (kx, ky) as in 3D, times the direct layer and the reflection layers
    l = 1..ceil(R_s / Lz - 1/2) of both sets; layers with factor 0 are left out.
    """
    Lx, Ly, Lz = box
    K = [int(math.ceil(Rs / L - 0.5)) for L in box]
    rows = []
    if dims == 3:
        for kx in range(-K[0], K[0] + 1):
            for ky in range(-K[1], K[1] + 1):
                for kz in range(-K[2], K[2] + 1):
                    rows.append((kx * Lx, ky * Ly, 1.0, kz * Lz, 1.0))
    else:
        layers = [(1.0, 0.0, 1.0)]
        for l in range(1, K[2] + 1):
            for sign in (+1, -1):
                f = image_factor(l, sign, gamma_top, gamma_bot)
                if f != 0.0:
                    layers.append(((-1.0) ** l, sign * (l * Lz), f))
        for kx in range(-K[0], K[0] + 1):
            for ky in range(-K[1], K[1] + 1):
                for (zs, zo, f) in layers:
                    rows.append((kx * Lx, ky * Ly, zs, zo, f))
    return np.array(rows, dtype=np.float64)


def dtn_lambda(field2d, Lx, Ly):
    """Periodic discrete DtN map of a G x G face field (R5): F^-1 |h| F."""
    G = field2d.shape[0]
    kx = np.fft.fftfreq(G) * G
    ky = np.fft.fftfreq(G) * G
    hx = 2.0 * math.pi * kx / Lx
    hy = 2.0 * math.pi * ky / Ly
    habs = np.sqrt(hx[:, None] ** 2 + hy[None, :] ** 2)
    return np.real(np.fft.ifft2(np.fft.fft2(field2d) * habs))


# Sign of the outward normal of the two faces, in face_grid order (top, bottom):
# dPhi/dn = FACE_SIGNS[f] * dPhi/dz.
FACE_SIGNS = (1.0, -1.0)


def dtn_weights(g, sn):
    """Coefficients (c_z, c_L) of a face row of R5, c_z dPhi/dz + c_L Lambda_G Phi:
    (1 + g) dPhi/dn + (1 - g) Lambda_G Phi with dPhi/dn = sn dPhi/dz.  The
    form follows from continuity of Phi and of eps dPhi/dz across the face,
    dPhi_out/dn = -Lambda Phi outside (no charges there, decay away from the
    slab) and eps_c : eps_out = (1 + g) : (1 - g) (Sec. 2.1, Eq. 4's g)."""
    return (1.0 + g) * sn, (1.0 - g)


def dtn_rows(phi, dphidz, g, sn, Lx, Ly):
    """The face condition of R5 applied to a field sampled on one face's
    G x G grid (face_grid order): (1 + g) dPhi/dn + (1 - g) Lambda_G Phi.
    phi and dphidz are (G*G,) or (G*G, k) arrays; each column is one field."""
    cz, cl = dtn_weights(g, sn)
    phi = np.asarray(phi, dtype=np.float64)
    G = int(round(math.sqrt(phi.shape[0])))
    cols = phi.reshape(G * G, -1)
    lam = np.stack([dtn_lambda(cols[:, c].reshape(G, G), Lx, Ly).ravel()
                    for c in range(cols.shape[1])], axis=1)
    return (cz * np.asarray(dphidz, dtype=np.float64).reshape(G * G, -1) + cl * lam).reshape(phi.shape)


def face_grid(box, G):
    """G x G grid on the top face (z = +Lz/2) then the bottom face (R5)."""
    Lx, Ly, Lz = box
    xa = -0.5 * Lx + (np.arange(G) + 0.5) * (Lx / G)
    ya = -0.5 * Ly + (np.arange(G) + 0.5) * (Ly / G)
    X, Y = np.meshgrid(xa, ya, indexing="ij")
    top = np.stack([X.ravel(), Y.ravel(), np.full(G * G, 0.5 * Lz)], -1)
    bot = np.stack([X.ravel(), Y.ravel(), np.full(G * G, -0.5 * Lz)], -1)
    return top, bot


def make_setup(box, dims, p, M, gamma_top=0.0, gamma_bot=0.0, lam=None,
               n_monitor=None, dtn_grid=80, prefactor=1.0, grad_rows=False,
               grad_weight=GRAD_WEIGHT, sphere_mask=True, surface_rule=0):
    """Geometry-only preparation: sphere, shifts, check points, fit, map.
    grad_rows adds the gradient-periodicity rows of R13; sphere_mask=False
    takes the unmasked near set of R12; surface_rule=1 the Fibonacci lattice
    rule of R18 (M must be a Fibonacci number >= 13)."""
    box = tuple(float(b) for b in box)
    if dims not in (2, 3):
        raise OracleError("dims must be 2 or 3")
    if p < 1 or M < (p + 1) ** 2:
        raise OracleError("need p >= 1 and M >= (p+1)^2")
    if abs(gamma_top) > 1 or abs(gamma_bot) > 1:
        raise OracleError("|gamma| must be <= 1")
    if surface_rule not in (0, 1) or (surface_rule == 1 and fibonacci_pair(M) is None):
        raise OracleError("surface_rule 1 needs M to be a Fibonacci number >= 13")
    if lam is None:
        lam = 1.3 if dims == 3 else 1.6
    if n_monitor is None:
        n_monitor = 2 * (p + 1) ** 2
    if dims == 3:
        gamma_top = gamma_bot = 0.0
    Lx, Ly, Lz = box
    st = Setup(dims, box, p, M, float(lam), int(n_monitor), float(gamma_top),
               float(gamma_bot), int(dtn_grid), float(prefactor))
    st.grad_rows = bool(grad_rows)
    st.grad_weight = float(grad_weight)
    st.sphere_mask = bool(sphere_mask)
    st.surface_rule = int(surface_rule)
    st.Rc = 0.5 * math.sqrt((Lx * Lx + Ly * Ly) + Lz * Lz)
    st.Rs = st.lam * st.Rc
    st.Rs2 = st.Rs * st.Rs
    st.shifts = shift_table(dims, box, st.Rs, gamma_top, gamma_bot)

    nb = H.nbasis(p)
    mon = golden_spiral(st.n_monitor, st.Rc)
    L = np.array(box)
    if dims == 3:
        wrap = mon - L * rnd_half_away(mon / L)
        keep = np.ones(st.n_monitor, dtype=bool)
    else:
        wrap = mon.copy()
        wrap[:, :2] = mon[:, :2] - L[:2] * rnd_half_away(mon[:, :2] / L[:2])
        keep = np.any(wrap != mon, axis=1)
    st.n_mon = st.n_monitor
    st.keep = keep
    # periodic rows, A_0^0 column dropped
    Bm = H.solid(p, mon, st.Rc)[:, 1:]
    Bw = H.solid(p, wrap, st.Rc)[:, 1:]
    Dper = (Bm - Bw)[keep]
    # design matrix rows: periodic rows first, then (2D) the two faces
    if dims == 3:
        st.check_pts = np.vstack([mon, wrap])
        D = Dper
    else:
        G = st.dtn_grid
        top, bot = face_grid(box, G)
        st.check_pts = np.vstack([mon, wrap, top, bot])
        wd = st.Rc / G
        blocks = [Dper]
        for pts, g, sn in ((top, gamma_top, FACE_SIGNS[0]), (bot, gamma_bot, FACE_SIGNS[1])):
            B = H.solid(p, pts, st.Rc)[:, 1:]
            dB = H.solid_dz(p, pts, st.Rc)[:, 1:]
            blocks.append(wd * dtn_rows(B, dB, g, sn, Lx, Ly))
        D = np.vstack(blocks)
    n_base_rows = D.shape[0]
    if st.grad_rows:
        # R13: one row per kept monitoring point and component, component-major
        wg = st.grad_weight * st.Rc
        Gm = H.solid_grad(p, mon, st.Rc)[:, 1:, :]
        Gw = H.solid_grad(p, wrap, st.Rc)[:, 1:, :]
        D = np.vstack([D] + [wg * (Gm[:, :, d] - Gw[:, :, d])[keep] for d in range(3)])
    U, sv, Vt = np.linalg.svd(D, full_matrices=False)
    cut = SVD_RCOND * sv[0]
    inv = np.where(sv > cut, 1.0 / np.where(sv > cut, sv, 1.0), 0.0)
    st.rank = int(np.sum(sv > cut))
    st.sing = sv
    st.D = D
    pinv = (Vt.T * inv) @ U.T              # (nb-1, rows)

    # P maps the raw check vector v to A: A = pinv @ rhs(v).
    # 3D: v = Phi_B at [mon ; wrap], rhs = Phi_B(wrap) - Phi_B(mon).
    # 2D: v = [Phi_B at check pts ; dPhi_B/dz at check pts]; face rows have
    #     rhs = -wd [(1+g) sn dPhi_B/dz + (1-g) Lambda_G Phi_B]; Lambda_G is a
    #     real symmetric operator, so pinv_face @ Lambda_G = (Lambda_G applied
    #     to each row of pinv_face).
    nm = st.n_mon
    kidx = np.nonzero(keep)[0]
    Pper = pinv[:, :len(kidx)]
    if dims == 3:
        P = np.zeros((nb - 1, 2 * nm))
        P[:, kidx] -= Pper
        P[:, nm + kidx] += Pper
    else:
        ncheck = 2 * nm + 2 * G * G
        P = np.zeros((nb - 1, 2 * ncheck))
        P[:, kidx] -= Pper
        P[:, nm + kidx] += Pper
        r0 = len(kidx)
        for f, (g, sn) in enumerate(((gamma_top, FACE_SIGNS[0]), (gamma_bot, FACE_SIGNS[1]))):
            cz, cl = dtn_weights(g, sn)
            Pf = pinv[:, r0 + f * G * G: r0 + (f + 1) * G * G]
            LPf = np.stack([dtn_lambda(Pf[c].reshape(G, G), Lx, Ly).ravel()
                            for c in range(nb - 1)], axis=0)
            off = 2 * nm + f * G * G
            P[:, off:off + G * G] += -wd * cl * LPf
            P[:, ncheck + off:ncheck + off + G * G] += -wd * cz * Pf
    if st.grad_rows:
        # raw vector gains [d_x Phi_B ; d_y Phi_B ; d_z Phi_B] at [mon ; wrap]
        nv0 = P.shape[1]
        Pg = np.zeros((nb - 1, 6 * nm))
        nk = len(kidx)
        for d in range(3):
            Pd = wg * pinv[:, n_base_rows + d * nk: n_base_rows + (d + 1) * nk]
            Pg[:, 2 * nm * d + kidx] -= Pd
            Pg[:, 2 * nm * d + nm + kidx] += Pd
        P = np.hstack([P, Pg])
        assert P.shape[1] == nv0 + 6 * nm
    st.P = P

    if st.surface_rule == 0:
        # surface map (R6): Q_m = sum_nm A_nm (2n+1) R_s^(n+1) / M Y_nm(yhat_m)
        st.ysurf = golden_spiral(M, st.Rs)
        Y = H.solid(p, st.ysurf, st.Rs)       # (r/R_s)^n Y_nm = Y_nm at r = R_s
        nfac = np.array([(2 * n + 1) * st.Rs ** (n + 1) / (M * st.Rc ** n)
                         for n in range(p + 1) for _ in range(2 * n + 1)])
        st.W = (Y * nfac[None, :])[:, 1:]
    else:
        # R18: Q_j = sum_nm A_nm (2n+1) R_s^(n+1) w_j / (4 pi) Y_nm(yhat_j)
        st.ysurf, st.wsurf = fibonacci_lattice(M, st.Rs)
        Y = H.solid(p, st.ysurf, st.Rs)
        nfac = np.array([(2 * n + 1) * st.Rs ** (n + 1) / (4.0 * math.pi * st.Rc ** n)
                         for n in range(p + 1) for _ in range(2 * n + 1)])
        st.W = (Y * nfac[None, :] * st.wsurf[:, None])[:, 1:]
    return st


# ---------------------------------------------------------------------------
# Per-evaluation steps (the paper's "Compute")
# ---------------------------------------------------------------------------
def prepare_inputs(st, x, q):
    """Validate, wrap and centre the positions; remove the neutral residual (R8)."""
    x = np.array(x, dtype=np.float64).reshape(-1, 3)
    q = np.array(q, dtype=np.float64).ravel()
    if len(q) < 1 or len(x) != len(q):
        raise OracleError("bad sizes")
    tot = float(np.sum(q))
    if abs(tot) > NEUTRAL_TOL * float(np.sum(np.abs(q))):
        raise OracleError("not neutral")
    q = q - tot / len(q)
    Lx, Ly, Lz = st.box
    xc = np.empty_like(x)
    for d, L in ((0, Lx), (1, Ly)):
        xc[:, d] = (x[:, d] - L * np.floor(x[:, d] / L)) - 0.5 * L
    if st.dims == 3:
        xc[:, 2] = (x[:, 2] - Lz * np.floor(x[:, 2] / Lz)) - 0.5 * Lz
    else:
        if np.any(x[:, 2] <= 0.0) or np.any(x[:, 2] >= Lz):
            raise OracleError("z outside the slab")
        xc[:, 2] = x[:, 2] - 0.5 * Lz
    return xc, q


def near_set(st, xc, q):
    """Images inside B (step 1, R2), or every image of the table (R12):
    positions, charges, source index, shift index."""
    pos, chg, src, sid = [], [], [], []
    for s, (sx, sy, zs, zo, f) in enumerate(st.shifts):
        px = xc[:, 0] + sx
        py = xc[:, 1] + sy
        pz = zs * xc[:, 2] + zo
        r2 = (px * px + py * py) + pz * pz
        inside = (r2 < st.Rs2) if st.sphere_mask else np.ones(len(px), dtype=bool)
        j = np.nonzero(inside)[0]
        pos.append(np.stack([px[j], py[j], pz[j]], -1))
        chg.append(f * q[j])
        src.append(j)
        sid.append(np.full(len(j), s))
    return (np.concatenate(pos), np.concatenate(chg),
            np.concatenate(src), np.concatenate(sid))


def self_shift(st):
    """Index of the identity shift (k = 0, direct layer) in the table."""
    t = st.shifts
    hit = np.nonzero((t[:, 0] == 0) & (t[:, 1] == 0) & (t[:, 2] == 1.0)
                     & (t[:, 3] == 0) & (t[:, 4] == 1.0))[0]
    return int(hit[0])


def pair_field(tgt, src, qs, exclude=None, budget=4_000_000):
    """Plain direct sum (steps 5 and the check-point sum).

    phi(t) = sum_s q_s / |x_s - t|,  grad(t) = sum_s q_s (x_s - t) / |x_s - t|^3,
    with source exclude[t] (if >= 0) left out of target t's sums.
    """
    tgt = np.asarray(tgt, dtype=np.float64)
    nt, ns = len(tgt), len(src)
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3))
    chunk = max(1, budget // max(1, ns))
    for t0 in range(0, nt, chunk):
        t1 = min(nt, t0 + chunk)
        d = src[None, :, :] - tgt[t0:t1, None, :]
        r2 = np.sum(d * d, axis=-1)
        if exclude is not None:
            for t in range(t0, t1):
                if exclude[t] >= 0:
                    r2[t - t0, exclude[t]] = np.inf
        inv = 1.0 / np.sqrt(r2)
        qi = qs[None, :] * inv
        phi[t0:t1] = np.sum(qi, axis=1)
        grad[t0:t1] = np.einsum("ts,tsc->tc", qi * inv * inv, d)
    return phi, grad


def check_raw(st, cphi, cgrad):
    """Raw check-point vector v in the layout ``P`` expects."""
    v = cphi if st.dims == 3 else np.concatenate([cphi, cgrad[:, 2]])
    if st.grad_rows:
        nm2 = 2 * st.n_mon
        v = np.concatenate([v, cgrad[:nm2, 0], cgrad[:nm2, 1], cgrad[:nm2, 2]])
    return v


def evaluate(st, x, q, targets=None, Q=None, far="surface"):
    """One HSMA evaluation.

    Returns a dict with energy (None when ``targets`` selects a subset),
    phi, grad, forces (at the selected targets, prefactor applied to energy
    and forces only), the check-point values, the coefficients A (scaled
    basis, n >= 1), the surface charges Q and N_s.  Passing the surface
    charges Q of an earlier call on the same input skips steps 3 and 4.
    far="series" evaluates the fitted series of Eq. 5 directly at the ions
    instead of the surface charges (a cheaper alternative at small p).
    """
    xc, qc = prepare_inputs(st, x, q)
    n = len(qc)
    ipos, iq, isrc, isid = near_set(st, xc, qc)
    cphi = cgrad = A = None
    if Q is None:
        # step 3: Phi_B at the check points, then the fit
        cphi, cgrad = pair_field(st.check_pts, ipos, iq)
        A = st.P @ check_raw(st, cphi, cgrad)
        # step 4: surface charges
        Q = st.W @ A
    # step 5: near + far at the particles (self copy excluded, R1)
    sel = np.arange(n) if targets is None else np.asarray(targets)
    s0 = self_shift(st)
    self_idx = np.full(n, -1)
    m0 = isid == s0
    self_idx[isrc[m0]] = np.nonzero(m0)[0]
    nphi, ngrad = pair_field(xc[sel], ipos, iq, exclude=self_idx[sel])
    if far == "series":
        # the truncated series of Sec. 2.2, Eq. 5 itself (no surface charges)
        if A is None:
            raise OracleError("the series far field needs the fitted coefficients")
        fphi, fgrad = H.series_field(st.p, xc[sel], st.Rc, A)
    else:
        fphi, fgrad = pair_field(xc[sel], st.ysurf, Q)
    phi = nphi + fphi
    grad = ngrad + fgrad
    out = dict(phi=phi, grad=grad, forces=-st.prefactor * qc[sel, None] * grad,
               near_phi=nphi, far_phi=fphi, check_phi=cphi, check_grad=cgrad,
               A=A, Q=Q, Ns=len(iq), q=qc, xc=xc)
    out["energy"] = (0.5 * st.prefactor * float(np.dot(qc, phi))) if targets is None else None
    return out
