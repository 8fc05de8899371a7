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


def electrolyte(c, margin=0.0, seed=None):
    """Positions (N, 3) in the API box and charges (N,) for a case."""
    rng = np.random.Generator(np.random.PCG64(c.seed if seed is None else seed))
    N = c.N
    Lx, Ly, Lz = c.box
    x = np.empty((N, 3))
    x[:, 0] = rng.uniform(0.0, Lx, N)
    x[:, 1] = rng.uniform(0.0, Ly, N)
    if c.dims == 3:
        x[:, 2] = rng.uniform(0.0, Lz, N)
    else:
        lo = max(margin, 1e-9 * Lz)
        x[:, 2] = rng.uniform(lo, Lz - lo, N)
    q = np.concatenate([np.full(k, float(v)) for v, k in sorted(c.counts.items())])
    q = q[rng.permutation(N)]
    return x, q


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
