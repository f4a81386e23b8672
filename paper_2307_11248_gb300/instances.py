"""Seeded synthetic QAP instances (inputs only; no search arithmetic here).

The paper measures on QAPLIB instances (Section 6.1: the uniform "a" family,
the asymmetric random "b" family, lipa).  Those files are not available, so
the workloads use synthetic stand-ins of the same shapes and value
distributions:

* ``uniform_instance``   - dense uniform integers with a zero diagonal,
                           symmetric or asymmetric (the "a"/"b" families).
* ``grid_instance``      - Manhattan distances on a rectangular grid with a
                           sparse symmetric flow (a facility-layout instance).
* ``lognormal_instance`` - skewed, 70 % dense flows over uniform distances,
                           symmetric or asymmetric.
* ``batch_instances``    - many instances of uneven size for the batched form.
* ``poisson_requests``   - a stream of solve requests with exponential
                           inter-arrival gaps for the serving loop.

Every generator takes an explicit integer seed and uses numpy's PCG64, so the
same call gives the same matrices on every machine.  Matrices are returned as
int64 numpy arrays, row-major, shape (n, n).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _sym_from_upper(n: int, vals: np.ndarray) -> np.ndarray:
    """Place `vals` row-major into the strict upper triangle and mirror it."""
    M = np.zeros((n, n), dtype=np.int64)
    iu = np.triu_indices(n, 1)
    M[iu] = vals
    M[(iu[1], iu[0])] = vals
    return M


def _offdiag(n: int, vals: np.ndarray) -> np.ndarray:
    """Place `vals` row-major into the off-diagonal cells; zero diagonal."""
    M = np.zeros((n, n), dtype=np.int64)
    mask = ~np.eye(n, dtype=bool)
    M[mask] = vals
    return M


def uniform_matrix(rng, n, lo, hi, symmetric):
    if symmetric:
        return _sym_from_upper(n, rng.integers(lo, hi + 1, size=n * (n - 1) // 2))
    return _offdiag(n, rng.integers(lo, hi + 1, size=n * (n - 1)))


def uniform_instance(n: int, seed: int, symmetric: bool, lo: int = 0, hi: int = 99):
    """F and D with off-diagonal entries uniform in [lo, hi], zero diagonal.

    F is drawn first, then D, from one generator seeded with `seed`.
    """
    rng = _rng(seed)
    F = uniform_matrix(rng, n, lo, hi, symmetric)
    D = uniform_matrix(rng, n, lo, hi, symmetric)
    return F, D


def grid_distances(n: int) -> np.ndarray:
    """Manhattan distances between the first n cells (row-major) of a grid
    with floor(sqrt(n)) rows and ceil(n / rows) columns."""
    rows = max(1, int(math.isqrt(n)))
    cols = -(-n // rows)
    cells = np.arange(n)
    y, x = cells // cols, cells % cols
    return (np.abs(y[:, None] - y[None, :]) + np.abs(x[:, None] - x[None, :])).astype(np.int64)


def grid_instance(n: int, seed: int, density: float = 0.3, lo: int = 1, hi: int = 20):
    """D = grid Manhattan distances; F symmetric, each off-diagonal pair
    non-zero with probability `density`, non-zero values uniform in [lo, hi]."""
    rng = _rng(seed)
    m = n * (n - 1) // 2
    present = rng.random(m) < density
    vals = rng.integers(lo, hi + 1, size=m)
    F = _sym_from_upper(n, np.where(present, vals, 0))
    return F, grid_distances(n)


def lognormal_instance(n: int, seed: int, symmetric: bool, mu: float = 2.0, sigma: float = 1.5,
                       cap: int = 10000, density: float = 0.7, dlo: int = 1, dhi: int = 100):
    """F = round(exp(mu + sigma z)) capped at `cap`, present with probability
    `density` (absent entries are 0); D off-diagonal uniform in [dlo, dhi];
    zero diagonals."""
    rng = _rng(seed)
    m = n * (n - 1) // 2 if symmetric else n * (n - 1)
    z = rng.standard_normal(m)
    present = rng.random(m) < density
    vals = np.minimum(np.rint(np.exp(mu + sigma * z)), cap).astype(np.int64)
    vals = np.where(present, vals, 0)
    F = _sym_from_upper(n, vals) if symmetric else _offdiag(n, vals)
    D = uniform_matrix(rng, n, dlo, dhi, symmetric)
    return F, D


@dataclass
class Instance:
    F: np.ndarray
    D: np.ndarray
    symmetric: bool
    kind: str

    @property
    def n(self):
        return self.F.shape[0]


def batch_instances(count: int, seed: int, nmin: int = 20, nmax: int = 150):
    """`count` instances with n uniform in [nmin, nmax]; even-numbered ones
    symmetric, odd-numbered asymmetric, all from ``lognormal_instance``.
    Instance k is seeded with (seed, k) so any instance can be rebuilt alone."""
    sizes = _rng(seed).integers(nmin, nmax + 1, size=count)
    out = []
    for k in range(count):
        sym = (k % 2 == 0)
        F, D = lognormal_instance(int(sizes[k]), seed * 1_000_003 + k + 1, sym)
        out.append(Instance(F, D, sym, "lognormal"))
    return out


@dataclass
class Request:
    rid: int
    arrival_s: float
    inst: Instance


def poisson_requests(count: int, seed: int, rate_per_s: float = 2000.0, nmin: int = 12,
                     nmax: int = 256):
    """A stream of `count` solve requests: exponential gaps of mean 1/rate,
    n uniform in [nmin, nmax], generator uniform over {symmetric uniform,
    asymmetric uniform, grid}; request k's instance is seeded with (seed, k)."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = rng.integers(nmin, nmax + 1, size=count)
    kinds = rng.integers(0, 3, size=count)
    reqs = []
    for k in range(count):
        n, s = int(sizes[k]), seed * 1_000_003 + k + 1
        if kinds[k] == 0:
            F, D = uniform_instance(n, s, True)
            inst = Instance(F, D, True, "uniform-sym")
        elif kinds[k] == 1:
            F, D = uniform_instance(n, s, False)
            inst = Instance(F, D, False, "uniform-asym")
        else:
            F, D = grid_instance(n, s)
            inst = Instance(F, D, True, "grid")
        reqs.append(Request(k, float(arrivals[k]), inst))
    return reqs


def periodic_tenure(n: int):
    """Tenure range [floor(0.9 n), ceil(1.1 n)] redrawn every 2n iterations."""
    return (max(1, (9 * n) // 10), (11 * n + 9) // 10, 2 * n)


def paper_tenure(n: int):
    """The paper's tenure range [0.1 n, 0.33 n] (Section 4.3), redrawn per
    move: tmin = max(1, floor(n/10)), tmax = max(tmin, ceil(33 n / 100))."""
    tmin = max(1, n // 10)
    return (tmin, max(tmin, (33 * n + 99) // 100), 0)


# ---------------------------------------------------------------------------
# The named workloads (instance seed = workload number - 1, search seed =
# 1000 + workload number).
# ---------------------------------------------------------------------------

def workload_sym12():
    """n=12 symmetric uniform [0,99], 2opt from 32 random starts."""
    F, D = uniform_instance(12, 0, True)
    return dict(F=F, D=D, walks=32, seed=1001)


def workload_asym50():
    """n=50 asymmetric uniform [0,99], tabu 256 walks x 5000 iterations."""
    F, D = uniform_instance(50, 1, False)
    return dict(F=F, D=D, walks=256, iters=5000, tenure=periodic_tenure(50), seed=1002)


def workload_grid100():
    """n=100 grid instance, 2opt then tabu, 1024 walks x 10000 iterations."""
    F, D = grid_instance(100, 2)
    return dict(F=F, D=D, walks=1024, iters=10000, tenure=periodic_tenure(100), seed=1003)


def workload_batch512():
    """512 lognormal instances of n in [20,150], 64 tabu walks x 5000 each."""
    return dict(instances=batch_instances(512, 3), walks=64, iters=5000, seed=1004)
