"""Seeded synthetic electrolytes shaped like the paper's workloads.

Shared by the tests, ``bench.py`` and ``__graft_entry__.smoke()``; it holds no
part of the method's arithmetic (positions and charges only), so both the
oracle and the CUDA path can be fed from it.

The paper's workloads are MD states of primitive electrolytes (Sec. 4.1,
Sec. 4.3) and SPC/E water (Sec. 4.2).  They are not available, so each case is
a neutral mixture of point charges with positions drawn uniformly (NumPy
PCG64, seed = case number) and valences assigned by a seeded permutation of
the valence multiset.  ``margin`` keeps slab charges away from the walls, as
the paper's LJ walls do (Sec. 4.3).
"""
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Case:
    name: str
    dims: int
    box: tuple
    counts: dict                # valence -> number of ions
    p: int
    M: int
    lam: float
    gammas: tuple = (0.0, 0.0)  # (gamma_top, gamma_bot), 2D only
    dtn_grid: int = 80
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return int(sum(self.counts.values()))


def cubic_box_for_density(N, rho):
    L = (N / rho) ** (1.0 / 3.0)
    return (L, L, L)


def case(n, gamma=0.95):
    """The five workload shapes (sizes, valences, harmonic order, M)."""
    if n == 1:
        return Case("hsma3d_n1000_L10_p6_M800", 3, (10.0, 10.0, 10.0),
                    {+1: 500, -1: 500}, p=6, M=800, lam=1.3, seed=1)
    if n == 2:
        return Case("hsma3d_n100000_rho0.1_p8_M2000", 3, cubic_box_for_density(100000, 0.1),
                    {+1: 50000, -1: 50000}, p=8, M=2000, lam=1.3, seed=2)
    if n == 3:
        return Case(f"hsma2d_n20000_20x20x10_g{gamma:+.2f}_p8_M1500", 2, (20.0, 20.0, 10.0),
                    {+1: 10000, -1: 10000}, p=8, M=1500, lam=1.6,
                    gammas=(gamma, gamma), dtn_grid=80, seed=3)
    if n == 5:
        return Case("hsma3d_n262144_rho0.1_p10_M4000", 3, cubic_box_for_density(262144, 0.1),
                    {+2: 87381, -1: 174762, 0: 1}, p=10, M=4000, lam=1.3, seed=5)
    raise KeyError(n)


def electrolyte(c, margin=0.0, seed=None, min_dist=0.0):
    """Positions (N, 3) in the API box and charges (N,) for a case.

    min_dist > 0 gives the "paper-like" variant: candidates drawn in the same
    way are rejected while closer than min_dist (periodic minimum image in the
    periodic directions) to an accepted ion, mimicking the soft cores of the
    paper's Lennard-Jones electrolytes (Sec. 4.1: sigma-sized ions)."""
    rng = np.random.Generator(np.random.PCG64(c.seed if seed is None else seed))
    N = c.N
    Lx, Ly, Lz = c.box
    lo = max(margin, 1e-9 * Lz)

    def draw(n):
        y = np.empty((n, 3))
        y[:, 0] = rng.uniform(0.0, Lx, n)
        y[:, 1] = rng.uniform(0.0, Ly, n)
        y[:, 2] = rng.uniform(0.0, Lz, n) if c.dims == 3 else rng.uniform(lo, Lz - lo, n)
        return y

    if min_dist <= 0.0:
        x = draw(N)
    else:
        x = _hard_core(draw, N, c.box, c.dims, min_dist)
    q = np.concatenate([np.full(k, float(v)) for v, k in sorted(c.counts.items())])
    q = q[rng.permutation(N)]
    return x, q


def _hard_core(draw, N, box, dims, dmin, max_tries=200):
    """Sequential rejection sampling on a cell grid (cells >= dmin wide)."""
    L = np.asarray(box, dtype=np.float64)
    nc = np.maximum(1, np.floor(L / dmin).astype(int))
    cell = L / nc
    per = (True, True, dims == 3)
    grid = {}
    out = np.empty((N, 3))
    n = 0
    d2 = dmin * dmin
    for _ in range(max_tries):
        for y in draw(2 * (N - n) + 64):
            ci = np.minimum((y / cell).astype(int), nc - 1)
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        k = [ci[0] + dx, ci[1] + dy, ci[2] + dz]
                        for a in range(3):
                            if per[a]:
                                k[a] %= nc[a]
                        for j in grid.get(tuple(k), ()):
                            dv = out[j] - y
                            for a in range(3):
                                if per[a]:
                                    dv[a] -= L[a] * round(dv[a] / L[a])
                            if dv @ dv < d2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                out[n] = y
                grid.setdefault(tuple(ci), []).append(n)
                n += 1
                if n == N:
                    return out
    raise RuntimeError("hard-core sampling did not place every ion")


def small_case(N, dims=3, box=None, p=6, M=800, lam=None, gammas=(0.0, 0.0), seed=11,
               valences=(+1, -1), G=32):
    """A neutral +-1 (or given valence pair) electrolyte of N ions (N even)."""
    if box is None:
        box = (10.0, 10.0, 10.0) if dims == 3 else (20.0, 20.0, 10.0)
    if lam is None:
        lam = 1.3 if dims == 3 else 1.6
    a, b = valences
    # neutral: na * a + nb * b = 0
    if a == -b:
        counts = {a: N // 2, b: N - N // 2}
    else:
        g = math.gcd(abs(a), abs(b))
        unit = abs(b) // g + abs(a) // g
        k = N // unit
        counts = {a: k * abs(b) // g, b: k * abs(a) // g}
        rest = N - sum(counts.values())
        if rest:
            counts[0] = rest
    return Case(f"small_{dims}d_n{N}", dims, tuple(float(v) for v in box), counts,
                p=p, M=M, lam=lam, gammas=gammas, dtn_grid=G, seed=seed)


def serving_stream(n_req=512, seed=4, rho=0.1, nmin=1000, nmax=50000):
    """Request shapes for the served workload: N log-uniform (even), p in {6,8,10}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(n_req):
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        N -= N % 2
        p = int(rng.choice([6, 8, 10]))
        out.append(dict(N=N, p=p, M=4 * p * p + 400, box=cubic_box_for_density(N, rho),
                        seed=int(rng.integers(1 << 31))))
    return out


def poisson_arrivals(n_req, rate_per_s, seed=4):
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n_req))
