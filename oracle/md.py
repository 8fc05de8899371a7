"""Molecular dynamics of a primitive-model electrolyte (TEST INFRASTRUCTURE).

The validation workload of Sec. 4.1: ions are soft spheres of diameter sigma
that repel through the shifted-truncated Lennard-Jones potential (cut at its
minimum 2^(1/6) sigma, energy coupling eps = kT), and interact through
Coulomb's law with Bjerrum length l_B (energy l_B kT q_i q_j / r, the
electrostatic solver's prefactor).  Canonical ensemble with a Nose-Hoover
thermostat; velocity-Verlet integration.

One step of length dt, in this order (a symmetric Trotter splitting of the
Nose-Hoover equations of motion, thermostat chain of length one):

  thermostat half step:  G = (2K - g kT) / Q;  xi += G dt/4
                         v *= exp(-xi dt/2);  eta += xi dt/2
                         G = (2K - g kT) / Q;  xi += G dt/4   (K after scaling)
  kick:                  v += (dt/2) F / m
  drift:                 x += dt v, wrapped into the box (image counters kept)
  forces:                F = F_LJ(x) + F_coulomb(x)
  kick:                  v += (dt/2) F / m
  thermostat half step   (as above)

with Q = g kT tdamp^2 and g = 3N - 3 degrees of freedom (the centre-of-mass
momentum is conserved).  The extended energy H = K + U + Q xi^2/2 + g kT eta
is conserved by the flow.  Readings: the paper states the damping time of its
thermostat but not its chain length or the degrees of freedom; a single
thermostat and g = 3N - 3 are taken here.  With the thermostat off the step
is plain velocity Verlet (NVE).

Slabs (Sec. 4.3): with walls, the box is periodic in x and y only and the
ions are kept in 0 < z < Lz by shifted-truncated LJ walls at z = 0 and
z = Lz (energy 4 e_w [(s_w/d)^12 - (s_w/d)^6] + e_w for a distance d to the
wall below 2^(1/6) s_w); positions wrap in x and y only.

Everything is FP64 NumPy; the Coulomb forces come from a callable (the
oracle's HSMA or Ewald sum).
"""
import math

import numpy as np

WCA_CUT = 2.0 ** (1.0 / 6.0)


def wca(x, box, sigma=1.0, eps=1.0, periodic=(True, True, True)):
    """Energy and forces of the shifted-truncated LJ repulsion, minimum image
    in the periodic directions, all pairs i < j."""
    x = np.asarray(x, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    per = np.array(periodic, dtype=bool)
    n = len(x)
    F = np.zeros_like(x)
    U = 0.0
    rc2 = (WCA_CUT * sigma) ** 2
    for i in range(n - 1):
        d = x[i + 1:] - x[i]
        d[:, per] -= L[per] * np.round(d[:, per] / L[per])
        r2 = np.sum(d * d, axis=1)
        m = r2 < rc2
        if not np.any(m):
            continue
        s2 = sigma * sigma / r2[m]
        s6 = s2 * s2 * s2
        U += float(np.sum(4.0 * eps * (s6 * s6 - s6) + eps))
        # force on j (the partner) along d: 24 eps (2 s12 - s6) / r^2 * d
        f = (24.0 * eps * (2.0 * s6 * s6 - s6) / r2[m])[:, None] * d[m]
        F[i + 1:][m] += f
        F[i] -= f.sum(axis=0)
    return U, F


def walls(x, Lz, sigma_w=0.5, eps_w=1.0):
    """Energy and forces of shifted-truncated LJ walls at z = 0 and z = Lz."""
    z = np.asarray(x, dtype=np.float64)[:, 2]
    F = np.zeros((len(z), 3))
    U = 0.0
    rc = WCA_CUT * sigma_w
    for d, sign in ((z, 1.0), (Lz - z, -1.0)):     # distance to the wall, direction away from it
        m = d < rc
        s6 = (sigma_w / d[m]) ** 6
        U += float(np.sum(4.0 * eps_w * (s6 * s6 - s6) + eps_w))
        F[m, 2] += sign * 24.0 * eps_w * (2.0 * s6 * s6 - s6) / d[m]
    return U, F


class State:
    """Positions (wrapped into [0, L), in x and y only for a slab), image
    counters, velocities, thermostat."""

    def __init__(self, x, v, q, box, mass=1.0, slab=False):
        self.slab = bool(slab)
        self.box = np.asarray(box, dtype=np.float64)
        self.x = np.array(x, dtype=np.float64)
        self.img = np.zeros(self.x.shape, dtype=np.int64)
        self.wrap()
        self.v = np.array(v, dtype=np.float64)
        self.q = np.array(q, dtype=np.float64)
        self.m = float(mass)
        self.xi = 0.0
        self.eta = 0.0
        self.F = None
        self.U = None

    def wrap(self):
        """x into [0, L) per component, the image counters keeping x + img L.
        The quotient x / L can round across an integer; the two fix-ups put
        such a coordinate back inside."""
        k = np.floor(self.x / self.box)
        if self.slab:
            k[:, 2] = 0.0
        self.x -= k * self.box
        L = np.broadcast_to(self.box, self.x.shape)
        hi = self.x >= L
        if self.slab:
            hi[:, 2] = False
        self.x[hi] -= L[hi]
        k[hi] += 1
        lo = self.x < 0.0
        if self.slab:
            lo[:, 2] = False
        self.x[lo] += L[lo]
        k[lo] -= 1
        top = lo & (self.x >= L)
        self.x[top] = 0.0
        k[top] += 1
        self.img += k.astype(np.int64)

    def kinetic(self):
        return 0.5 * self.m * float(np.sum(self.v * self.v))

    def unwrapped(self):
        return self.x + self.img * self.box


class Integrator:
    """Velocity Verlet with an optional Nose-Hoover thermostat (see header).

    coulomb(x, q) -> (energy, forces) is the electrostatic solver; None leaves
    Coulomb out.  tdamp None means NVE."""

    def __init__(self, coulomb, dt, kT=1.0, tdamp=None, sigma=1.0, eps=1.0, wall_sigma=0.5, wall_eps=1.0):
        self.coulomb = coulomb
        self.dt = float(dt)
        self.kT = float(kT)
        self.tdamp = tdamp
        self.sigma = sigma
        self.eps = eps
        self.wall_sigma = wall_sigma
        self.wall_eps = wall_eps

    def forces(self, s):
        U, F = wca(s.x, s.box, self.sigma, self.eps, periodic=(True, True, not s.slab))
        if s.slab:
            Uw, Fw = walls(s.x, s.box[2], self.wall_sigma, self.wall_eps)
            U += Uw
            F = F + Fw
        Uc = 0.0
        if self.coulomb is not None:
            Uc, Fc = self.coulomb(s.x, s.q)
            F = F + Fc
        s.U_lj, s.U_c = U, Uc
        s.U = U + Uc
        s.F = F

    def _thermostat_half(self, s):
        g = 3 * len(s.x) - 3
        Q = g * self.kT * self.tdamp ** 2
        h = 0.5 * self.dt
        K = s.kinetic()
        s.xi += (2.0 * K - g * self.kT) / Q * (h / 2)
        f = math.exp(-s.xi * h)
        s.v *= f
        s.eta += s.xi * h
        K = s.kinetic()
        s.xi += (2.0 * K - g * self.kT) / Q * (h / 2)

    def step(self, s):
        if s.F is None:
            self.forces(s)
        if self.tdamp is not None:
            self._thermostat_half(s)
        s.v += (0.5 * self.dt / s.m) * s.F
        s.x += self.dt * s.v
        s.wrap()
        self.forces(s)
        s.v += (0.5 * self.dt / s.m) * s.F
        if self.tdamp is not None:
            self._thermostat_half(s)

    def extended_energy(self, s):
        H = s.kinetic() + s.U
        if self.tdamp is not None:
            g = 3 * len(s.x) - 3
            Q = g * self.kT * self.tdamp ** 2
            H += 0.5 * Q * s.xi ** 2 + g * self.kT * s.eta
        return H


def rdf_counts(x, box, mask_a, mask_b, rmax, nbins):
    """Pair counts of species a around species b in nbins shells of width
    rmax/nbins (minimum image), the histogram g(r) is built from."""
    L = np.asarray(box, dtype=np.float64)
    xa, xb = x[mask_a], x[mask_b]
    h = np.zeros(nbins, dtype=np.int64)
    for p in xb:
        d = xa - p
        d -= L * np.round(d / L)
        r = np.sqrt(np.sum(d * d, axis=1))
        r = r[(r > 0) & (r < rmax)]
        h += np.bincount((r * (nbins / rmax)).astype(np.int64), minlength=nbins)[:nbins]
    return h


def maxwell_velocities(n, kT, mass, rng):
    """Gaussian velocities at temperature kT with zero total momentum."""
    v = rng.normal(0.0, math.sqrt(kT / mass), (n, 3))
    v -= v.mean(axis=0)
    return v
