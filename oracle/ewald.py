"""Ewald ground truth for the plain definitions in Sec. 2.1 (TEST INFRASTRUCTURE).

The HSMA result is an approximation, so the oracle first needs the exact
answer it approximates:

* Sec. 2.1, Eq. 3 -- the fully periodic Coulomb sum over k in Z^3.  A neutral
  cell makes it conditionally convergent; the HSMA fit imposes periodicity of
  the potential, which selects the conducting ("tin-foil") boundary, so the
  ground truth is Ewald summation without the dipole term.
* Sec. 2.1, Eq. 4 -- the 2D-periodic slab between two planar dielectric
  interfaces at z = +-Lz/2, written as the direct 2D-periodic sum plus the
  reflection image series.  The image of order l of charge q at z sits at
  (-1)^l z + l Lz (upper set) or (-1)^l z - l Lz (lower set) and carries the
  factor gamma_l^+ = g_up^ceil(l/2) g_low^floor(l/2) (upper) or
  gamma_l^- = g_low^ceil(l/2) g_up^floor(l/2) (lower).  (The printed Eq. 4
  swaps up/low in gamma_l^+; the first upper image is the reflection across the
  top interface, so it must carry g_up.  The two agree when g_up == g_low.)
  Each image layer is itself neutral, so each layer's interaction with the
  central charges is one 2D-periodic Ewald sum (Parry's form).

Units are Gaussian with eps_c = 1 (Sec. 2.1, Eq. 2): phi = sum q / r.
All coordinates here are box-centred: the cell is [-L/2, L/2]^3 (Sec. 2.1).
"""
import math

import numpy as np
from scipy.special import erfc, erf, erfcx

TWO_OVER_SQRT_PI = 2.0 / math.sqrt(math.pi)


def _lattice(nmax):
    r = np.arange(-nmax[0], nmax[0] + 1)
    s = np.arange(-nmax[1], nmax[1] + 1)
    t = np.arange(-nmax[2], nmax[2] + 1)
    g = np.stack(np.meshgrid(r, s, t, indexing="ij"), -1).reshape(-1, 3)
    return g.astype(np.float64)


# ---------------------------------------------------------------------------
# 3D: Ewald summation, conducting boundary (Sec. 2.1, Eq. 3)
# ---------------------------------------------------------------------------
def ewald3d(pos, q, box, rcut=None, tol=1e-16, chunk=64):
    """Energy, per-particle potential and potential gradient of Eq. 3.

    phi[i] is the potential at r_i from every charge and every periodic image
    except the k = 0 copy of i itself; grad[i] is its gradient with respect to
    the field point.  E = 1/2 sum_i q_i phi[i]; the force is -q_i grad[i].

    Real space:   sum_j sum_n' q_j erfc(a|d|)/|d|,     d = r_j + n.L - r_i
    Reciprocal:   (4 pi / V) sum_{k != 0} exp(-k^2/4a^2)/k^2 Re(S(k) e^{-ik.r_i})
    Self:         -2 a q_i / sqrt(pi)
    The splitting parameter a and both cut-offs are set from ``tol`` so that the
    neglected terms are below ``tol`` relative to a unit pair term.
    """
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    n = len(q)
    V = box[0] * box[1] * box[2]
    if rcut is None:
        rcut = float(box.min())
    s = math.sqrt(-math.log(tol))
    a = s / rcut
    kmax = 2.0 * a * s

    # real space: every image within rcut of every particle
    nmax = [int(math.ceil(rcut / box[d])) + 1 for d in range(3)]
    shifts = _lattice(nmax) * box
    is_zero = np.all(shifts == 0.0, axis=1)
    phi = np.zeros(n)
    grad = np.zeros((n, 3))
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        # d[t, j, s] = r_j + shift_s - r_t
        d = (pos[None, :, None, :] + shifts[None, None, :, :]
             - pos[i0:i1, None, None, :])
        r = np.sqrt(np.sum(d * d, axis=-1))
        keep = r < rcut
        # drop the self term (j == t, shift 0)
        for t in range(i0, i1):
            keep[t - i0, t, is_zero] = False
        rr = np.where(keep, r, 1.0)
        e = np.where(keep, erfc(a * rr) / rr, 0.0)
        phi[i0:i1] += np.einsum("tjs,j->t", e, q)
        # d/dr_t of erfc(a|d|)/|d| with d = src - r_t:  + [erfc/r^2 + 2a/sqrt(pi) e^{-a^2r^2}/r] d/r
        g = np.where(keep, (erfc(a * rr) / rr ** 2
                            + a * TWO_OVER_SQRT_PI * np.exp(-(a * rr) ** 2) / rr) / rr, 0.0)
        grad[i0:i1] += np.einsum("tjs,tjsc,j->tc", g, d, q)

    # reciprocal space
    mmax = [int(math.floor(kmax * box[d] / (2.0 * math.pi))) + 1 for d in range(3)]
    m = _lattice(mmax)
    m = m[np.any(m != 0, axis=1)]
    kv = 2.0 * math.pi * m / box
    k2 = np.sum(kv * kv, axis=1)
    sel = k2 <= kmax * kmax
    kv, k2 = kv[sel], k2[sel]
    fk = np.exp(-k2 / (4.0 * a * a)) / k2
    kr = pos @ kv.T                        # (n, K)
    c, sn = np.cos(kr), np.sin(kr)
    Sre = q @ c                            # S(k) = sum_j q_j e^{i k.r_j}
    Sim = q @ sn
    # Re(S e^{-ik.r}) = Sre cos + Sim sin ;  Im(S e^{-ik.r}) = Sim cos - Sre sin
    phi += (4.0 * math.pi / V) * ((c * Sre + sn * Sim) @ fk)
    grad += (4.0 * math.pi / V) * (((sn * -Sre + c * Sim) * fk) @ kv)

    # self term
    phi -= a * TWO_OVER_SQRT_PI * q
    energy = 0.5 * float(np.dot(q, phi))
    return energy, phi, grad


# ---------------------------------------------------------------------------
# 2D: Parry-type Ewald sum of one 2D-periodic neutral set (Sec. 2.1, Eq. 4)
# ---------------------------------------------------------------------------
def _g(h, dz, a):
    """exp(h dz) erfc(a dz + h/2a), evaluated without overflow."""
    y = a * dz + h / (2.0 * a)
    pos = y >= 0.0
    ys = np.where(pos, y, 0.0)
    # y >= 0: exp(h dz) erfc(y) = exp(-a^2 dz^2 - h^2/4a^2) erfcx(y)
    v_pos = np.exp(-(a * dz) ** 2 - (h / (2.0 * a)) ** 2) * erfcx(ys)
    # y < 0 needs dz < 0, so exp(h dz) < 1
    v_neg = np.exp(np.where(pos, 0.0, h * dz)) * erfc(np.where(pos, 0.0, y))
    return np.where(pos, v_pos, v_neg)


def ewald2d_field(tgt, src, qs, Lx, Ly, rcut, tol=1e-16, exclude=None, chunk=32):
    """Potential and gradient at ``tgt`` from the 2D-periodic set (src, qs).

    The set is periodic in x, y with periods Lx, Ly and must be neutral.
      phi(t) = sum_j sum_n' q_j erfc(a rho)/rho
             + (pi/A) sum_{h != 0} (1/h) sum_j q_j cos(h.(s_j - t)) [g(h,dz) + g(h,-dz)]
             - (2 pi/A) sum_j q_j [dz erf(a dz) + exp(-a^2 dz^2)/(a sqrt(pi))]
    with dz = z_j - z_t and g(h, dz) = exp(h dz) erfc(a dz + h/2a).
    ``exclude[t] = j`` drops the n = 0 copy of source j for target t and adds
    the self correction -2 a q_j / sqrt(pi) (used when src includes tgt).
    """
    tgt = np.asarray(tgt, dtype=np.float64)
    src = np.asarray(src, dtype=np.float64)
    qs = np.asarray(qs, dtype=np.float64)
    A = Lx * Ly
    s = math.sqrt(-math.log(tol))
    a = s / rcut
    hmax = 2.0 * a * s
    nt = len(tgt)
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3))

    nx = int(math.ceil(rcut / Lx)) + 1
    ny = int(math.ceil(rcut / Ly)) + 1
    gx, gy = np.meshgrid(np.arange(-nx, nx + 1), np.arange(-ny, ny + 1), indexing="ij")
    shifts = np.stack([gx.ravel() * Lx, gy.ravel() * Ly, 0.0 * gx.ravel()], -1)
    is_zero = np.all(shifts == 0.0, axis=1)

    mx = int(math.floor(hmax * Lx / (2.0 * math.pi))) + 1
    my = int(math.floor(hmax * Ly / (2.0 * math.pi))) + 1
    hx, hy = np.meshgrid(np.arange(-mx, mx + 1), np.arange(-my, my + 1), indexing="ij")
    hv = np.stack([2.0 * math.pi * hx.ravel() / Lx, 2.0 * math.pi * hy.ravel() / Ly], -1)
    hn = np.sqrt(np.sum(hv * hv, axis=1))
    sel = (hn > 0.0) & (hn <= hmax)
    hv, hn = hv[sel], hn[sel]

    for t0 in range(0, nt, chunk):
        t1 = min(nt, t0 + chunk)
        T = tgt[t0:t1]
        # --- real space
        d = src[None, :, None, :] + shifts[None, None, :, :] - T[:, None, None, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        keep = r < rcut
        if exclude is not None:
            for t in range(t0, t1):
                j = exclude[t]
                if j >= 0:
                    keep[t - t0, j, is_zero] = False
        rr = np.where(keep, r, 1.0)
        e = np.where(keep, erfc(a * rr) / rr, 0.0)
        phi[t0:t1] += np.einsum("tjs,j->t", e, qs)
        g = np.where(keep, (erfc(a * rr) / rr ** 2
                            + a * TWO_OVER_SQRT_PI * np.exp(-(a * rr) ** 2) / rr) / rr, 0.0)
        grad[t0:t1] += np.einsum("tjs,tjsc,j->tc", g, d, qs)

        # --- reciprocal space, h != 0
        dxy = src[None, :, :2] - T[:, None, :2]            # (t, j, 2)
        dz = src[None, :, 2] - T[:, None, 2]               # (t, j)
        for k in range(len(hn)):
            h = hn[k]
            ph = dxy @ hv[k]                               # h.(s_j - t)
            gp = _g(h, dz, a)
            gm = _g(h, -dz, a)
            c = np.cos(ph)
            sn = np.sin(ph)
            pre = math.pi / (A * h)
            phi[t0:t1] += pre * ((c * (gp + gm)) @ qs)
            # d/dt_xy cos(h.(s-t)) = h sin(h.(s-t)) ;  d/dz_t [g(h,dz)+g(h,-dz)] = -h [g(h,dz) - g(h,-dz)]
            sg = (sn * (gp + gm)) @ qs
            grad[t0:t1, 0] += pre * hv[k, 0] * sg
            grad[t0:t1, 1] += pre * hv[k, 1] * sg
            grad[t0:t1, 2] += pre * (-h) * ((c * (gp - gm)) @ qs)

        # --- h = 0
        phi[t0:t1] -= (2.0 * math.pi / A) * ((dz * erf(a * dz)
                                              + np.exp(-(a * dz) ** 2) / (a * math.sqrt(math.pi))) @ qs)
        # d/dz_t [dz erf(a dz) + ...] = -erf(a dz)
        grad[t0:t1, 2] += (2.0 * math.pi / A) * (erf(a * dz) @ qs)

    if exclude is not None:
        for t in range(nt):
            j = exclude[t]
            if j >= 0:
                phi[t] -= a * TWO_OVER_SQRT_PI * qs[j]
    return phi, grad


def image_factor(l, sign, g_up, g_low):
    """Charge factor of the order-l image (Sec. 2.1, Eq. 4, read as above).

    sign = +1: upper set (Omega_up), factor g_up^ceil(l/2) g_low^floor(l/2).
    sign = -1: lower set (Omega_low), factor g_low^ceil(l/2) g_up^floor(l/2).
    """
    c, f = (l + 1) // 2, l // 2
    if sign > 0:
        return (g_up ** c) * (g_low ** f)
    return (g_low ** c) * (g_up ** f)


def image_z(z, l, sign, Lz):
    """z of the order-l image of a charge at z (Sec. 2.1, Eq. 4): (-1)^l z +- l Lz."""
    return ((-1.0) ** l) * z + sign * (l * Lz)


def slab_lmax(g_up, g_low, Lx, Ly, Lz, eps=1e-16):
    """Number of image orders kept by the ground truth.

    Layer l lies at least (l - 1) Lz away from the slab, so its non-constant
    part decays like exp(-2 pi (l-1) Lz / max(Lx, Ly)); its constant part is
    killed by neutrality.  Stop when |gamma|^l times that is below eps.
    """
    g = max(abs(g_up), abs(g_low))
    if g == 0.0:
        return 0
    l = 1
    while True:
        if (g ** l) * math.exp(-2.0 * math.pi * (l - 1) * Lz / max(Lx, Ly)) < eps:
            return l
        l += 1
        if l > 400:
            return l


def slab_field(tgt, pos, q, Lx, Ly, Lz, g_up, g_low, rcut=None, tol=1e-16, lmax=None, exclude=None,
               chunk=32):
    """Potential and gradient of the dielectric slab (Sec. 2.1, Eq. 4) at the
    points ``tgt``: the direct 2D-periodic sum of the charges (pos, q) plus
    every image layer l = 1..lmax of both sets.  pos are box-centred with
    |z| < Lz/2; ``exclude`` as in ewald2d_field (direct layer only).
    Returns (phi, grad, lmax)."""
    tgt = np.asarray(tgt, dtype=np.float64)
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if rcut is None:
        rcut = 0.5 * min(Lx, Ly) + 0.5 * Lz
    if lmax is None:
        lmax = slab_lmax(g_up, g_low, Lx, Ly, Lz)
    phi, grad = ewald2d_field(tgt, pos, q, Lx, Ly, rcut, tol, exclude=exclude, chunk=chunk)
    for l in range(1, lmax + 1):
        for sign in (+1, -1):
            f = image_factor(l, sign, g_up, g_low)
            if f == 0.0:
                continue
            img = pos.copy()
            img[:, 2] = image_z(pos[:, 2], l, sign, Lz)
            p, gr = ewald2d_field(tgt, img, f * q, Lx, Ly, rcut, tol, chunk=chunk)
            phi += p
            grad += gr
    return phi, grad, lmax


def slab_ewald(pos, q, Lx, Ly, Lz, g_up, g_low, rcut=None, tol=1e-16, lmax=None):
    """Energy, potential and gradient of the dielectric slab (Sec. 2.1, Eq. 4).

    pos are box-centred, |z| < Lz/2.  phi[i] = direct 2D-periodic sum (self
    excluded) + sum over image layers l = 1..lmax of both sets.
    Returns (energy, phi, grad, lmax).
    """
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    phi, grad, lmax = slab_field(pos, pos, q, Lx, Ly, Lz, g_up, g_low, rcut=rcut, tol=tol, lmax=lmax,
                                 exclude=np.arange(len(q)))
    energy = 0.5 * float(np.dot(q, phi))
    return energy, phi, grad, lmax
