"""Real spherical and solid harmonics for the truncated far-field series
(TEST INFRASTRUCTURE).

Sec. 2.2, Eq. 5 writes the potential of the charges outside the auxiliary
sphere B as sum_{n<=P} sum_{|m|<=n} A_n^m r^n Y_n^m, with (P+1)^2 basis
functions.  The oracle uses the real orthonormal form of Y_n^m:

    Y_n0      = c_n0 P_n(cos t)
    Y_nm (m>0) = sqrt(2) c_nm P_n^m(cos t) cos(m f)
    Y_n,-m     = sqrt(2) c_nm P_n^m(cos t) sin(m f)
    c_nm      = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!)

with P_n^m the associated Legendre functions without the Condon-Shortley
phase.  Entry (n, m) sits at column n*n + n + m.

Any real orthonormal basis of the degree-n harmonics gives the same fitted
potential and the same surface charges, so this choice of signs is free.
"""
import math

import numpy as np


def nbasis(p):
    return (p + 1) * (p + 1)


def idx(n, m):
    return n * n + n + m


def assoc_legendre(nmax, t):
    """P_n^m(t) for 0 <= m <= n <= nmax, no Condon-Shortley phase.

    Textbook recursion:
      P_m^m     = (2m-1)!! (1 - t^2)^(m/2)
      P_{m+1}^m = (2m+1) t P_m^m
      (n-m) P_n^m = (2n-1) t P_{n-1}^m - (n+m-1) P_{n-2}^m
    Returns an array of shape (nmax+1, nmax+1) + t.shape indexed [n, m].
    """
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros((nmax + 1, nmax + 1) + t.shape)
    s = np.sqrt(np.maximum(0.0, 1.0 - t * t))
    pmm = np.ones_like(t)
    for m in range(nmax + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * s
        out[m, m] = pmm
        if m + 1 <= nmax:
            out[m + 1, m] = (2 * m + 1) * t * pmm
        for n in range(m + 2, nmax + 1):
            out[n, m] = ((2 * n - 1) * t * out[n - 1, m] - (n + m - 1) * out[n - 2, m]) / (n - m)
    return out


def real_sph(nmax, theta, phi):
    """Real orthonormal Y_nm(theta, phi); shape theta.shape + ((nmax+1)^2,)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    P = assoc_legendre(nmax, np.cos(theta))
    out = np.zeros(theta.shape + (nbasis(nmax),))
    for n in range(nmax + 1):
        for m in range(0, n + 1):
            c = math.sqrt((2 * n + 1) / (4.0 * math.pi)
                          * math.factorial(n - m) / math.factorial(n + m))
            if m == 0:
                out[..., idx(n, 0)] = c * P[n, 0]
            else:
                out[..., idx(n, m)] = math.sqrt(2.0) * c * P[n, m] * np.cos(m * phi)
                out[..., idx(n, -m)] = math.sqrt(2.0) * c * P[n, m] * np.sin(m * phi)
    return out


def to_spherical(xyz):
    xyz = np.asarray(xyz, dtype=np.float64)
    r = np.sqrt(np.sum(xyz * xyz, axis=-1))
    rs = np.where(r > 0.0, r, 1.0)
    theta = np.arccos(np.clip(xyz[..., 2] / rs, -1.0, 1.0))
    phi = np.arctan2(xyz[..., 1], xyz[..., 0])
    return r, theta, phi


def solid(nmax, xyz, scale):
    """Scaled regular solid harmonics (r/scale)^n Y_nm at the points xyz."""
    r, theta, phi = to_spherical(xyz)
    Y = real_sph(nmax, theta, phi)
    rn = np.stack([(r / scale) ** n for n in range(nmax + 1)], axis=-1)
    out = np.empty_like(Y)
    for n in range(nmax + 1):
        for m in range(-n, n + 1):
            out[..., idx(n, m)] = rn[..., n] * Y[..., idx(n, m)]
    return out


def solid_dz(nmax, xyz, scale):
    """d/dz of the scaled solid harmonics.

    For any real orthonormal family, d/dz (r^n Y_nm) is a multiple of
    r^(n-1) Y_(n-1)m with the same m:
        d/dz (r^n Y_nm) = sqrt((2n+1)/(2n-1) (n-m)(n+m)) r^(n-1) Y_(n-1)m
    (the z-derivative keeps the azimuthal factor; the constant follows from the
    normalisation).  With the scaling (r/s)^n this gains a factor 1/s.
    """
    S = solid(nmax, xyz, scale)
    out = np.zeros_like(S)
    for n in range(1, nmax + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            if am > n - 1:
                continue
            c = math.sqrt((2 * n + 1) / (2 * n - 1) * (n - am) * (n + am))
            out[..., idx(n, m)] = (c / scale) * S[..., idx(n - 1, m)]
    return out


def solid_cart(nmax, xyz, scale):
    """The same scaled solid harmonics as ``solid``, written as polynomials in
    Cartesian coordinates so the input may be complex (for complex-step
    derivatives).

    (x + iy)^m = C_m + i S_m is carried as the real pair (C_m, S_m); the
    polar factor r^n P_n^m(cos t) / sin^m t is the polynomial V_n^m(z, r^2)
    with V_m^m = (2m-1)!!, V_{m+1}^m = (2m+1) z V_m^m and
    (n-m) V_n^m = (2n-1) z V_{n-1}^m - (n+m-1) r^2 V_{n-2}^m.
    """
    xyz = np.asarray(xyz) / scale
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    r2 = x * x + y * y + z * z
    out = np.zeros(xyz.shape[:-1] + (nbasis(nmax),), dtype=np.result_type(xyz, float))
    C = np.ones_like(x)
    S = np.zeros_like(x)
    for m in range(nmax + 1):
        dfact = 1.0
        for k in range(2 * m - 1, 1, -2):
            dfact *= k
        V = [None] * (nmax + 1)
        V[m] = dfact * np.ones_like(x)
        if m + 1 <= nmax:
            V[m + 1] = (2 * m + 1) * z * V[m]
        for n in range(m + 2, nmax + 1):
            V[n] = ((2 * n - 1) * z * V[n - 1] - (n + m - 1) * r2 * V[n - 2]) / (n - m)
        for n in range(m, nmax + 1):
            c = math.sqrt((2 * n + 1) / (4.0 * math.pi)
                          * math.factorial(n - m) / math.factorial(n + m))
            if m == 0:
                out[..., idx(n, 0)] = c * V[n]
            else:
                out[..., idx(n, m)] = math.sqrt(2.0) * c * V[n] * C
                out[..., idx(n, -m)] = math.sqrt(2.0) * c * V[n] * S
        C, S = x * C - y * S, x * S + y * C
    return out


def solid_grad(nmax, xyz, scale):
    """Gradient of the scaled solid harmonics at the points xyz, shape
    xyz.shape[:-1] + ((nmax+1)^2, 3), by complex-step differentiation of the
    polynomial form (exact to rounding: no subtraction)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    h = 1e-30
    out = np.empty(xyz.shape[:-1] + (nbasis(nmax), 3))
    for d in range(3):
        z = xyz.astype(np.complex128)
        z[..., d] += 1j * h
        out[..., d] = solid_cart(nmax, z, scale).imag / h
    return out


def series_field(nmax, xyz, scale, coeffs):
    """phi = sum_k coeffs[k] S_k(xyz) over the basis without k = 0 (the
    constant), and its gradient."""
    xyz = np.asarray(xyz, dtype=np.float64)
    phi = solid_cart(nmax, xyz, scale)[..., 1:] @ coeffs
    grad = np.einsum("...kd,k->...d", solid_grad(nmax, xyz, scale)[..., 1:, :], coeffs)
    return phi, grad
