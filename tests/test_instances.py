"""The seeded synthetic inputs follow their stated recipe (sizes, value
ranges, symmetry, zero diagonals, densities, distributions), are
deterministic in their seeds, and the named workloads carry the stated
search settings.  CPU only."""
import math

import numpy as np

from paper_2307_11248_gb300 import instances


def offdiag(M):
    return M[~np.eye(M.shape[0], dtype=bool)]


def test_uniform_instance_recipe():
    F, D = instances.uniform_instance(40, 5, symmetric=False)
    for M in (F, D):
        assert M.dtype == np.int64 and M.shape == (40, 40)
        assert (np.diag(M) == 0).all()
        v = offdiag(M)
        assert v.min() >= 0 and v.max() <= 99
        assert abs(v.mean() - 49.5) < 3           # uniform on [0, 99]
    assert not (F == F.T).all() and not (D == D.T).all()
    Fs, Ds = instances.uniform_instance(40, 5, symmetric=True)
    assert (Fs == Fs.T).all() and (Ds == Ds.T).all()
    F2, D2 = instances.uniform_instance(40, 5, symmetric=False)
    assert (F2 == F).all() and (D2 == D).all()      # deterministic in the seed
    F3, _ = instances.uniform_instance(40, 6, symmetric=False)
    assert not (F3 == F).all()


def test_grid_distances_are_manhattan():
    D = instances.grid_distances(100)                  # 10 x 10 grid
    assert D.max() == 18 and D[0, 99] == 18 and D[0, 9] == 9 and D[0, 10] == 1
    for i, j in [(3, 77), (45, 54), (12, 12)]:
        assert D[i, j] == abs(i // 10 - j // 10) + abs(i % 10 - j % 10)
    assert (D == D.T).all() and (np.diag(D) == 0).all()
    D7 = instances.grid_distances(7)                   # 2 rows, 4 columns, first 7 cells
    assert D7[0, 6] == 1 + 2


def test_grid100_workload_recipe():
    w = instances.workload_grid100()
    F, D = w["F"], w["D"]
    assert F.shape == (100, 100) and (F == F.T).all() and (np.diag(F) == 0).all()
    assert (D == instances.grid_distances(100)).all()
    upper = F[np.triu_indices(100, 1)]
    nz = upper[upper != 0]
    assert nz.min() >= 1 and nz.max() <= 20
    assert abs(nz.size / upper.size - 0.3) < 0.03     # 30 % of the pairs carry flow
    assert (w["walks"], w["iters"], w["seed"]) == (1024, 10000, 1003)
    assert w["tenure"] == instances.periodic_tenure(100) == (90, 110, 200)


def test_named_small_workloads():
    s = instances.workload_sym12()
    assert s["F"].shape == (12, 12) and (s["F"] == s["F"].T).all() and s["walks"] == 32
    assert s["seed"] == 1001
    a = instances.workload_asym50()
    assert a["F"].shape == (50, 50) and not (a["F"] == a["F"].T).all()
    assert (a["walks"], a["iters"], a["seed"]) == (256, 5000, 1002)
    assert a["tenure"] == (45, 55, 100)


def test_lognormal_instance_recipe():
    F, D = instances.lognormal_instance(120, 9, symmetric=False)
    v = offdiag(F)
    assert (np.diag(F) == 0).all() and (np.diag(D) == 0).all()
    assert v.min() >= 0 and v.max() <= 10000
    # present with probability 0.7, and then non-zero unless exp(2 + 1.5 z)
    # rounds to 0, i.e. z < (ln 0.5 - 2) / 1.5
    z0 = (math.log(0.5) - 2.0) / 1.5
    expect = 0.7 * (1 - 0.5 * (1 + math.erf(z0 / math.sqrt(2))))
    assert abs((v != 0).mean() - expect) < 0.015
    nz = v[v != 0]
    # log of round(exp(2 + 1.5 z)): median exp(2), spread 1.5 (rounding and
    # the cap move the quartiles only slightly)
    assert abs(np.median(nz) - math.exp(2.0)) < 1.0
    q1, q3 = np.percentile(np.log(nz), [25, 75])
    assert abs((q3 - q1) - 2 * 0.6745 * 1.5) < 0.25
    d = offdiag(D)
    assert d.min() >= 1 and d.max() <= 100
    Fs, Ds = instances.lognormal_instance(60, 9, symmetric=True)
    assert (Fs == Fs.T).all() and (Ds == Ds.T).all()


def test_batch512_recipe():
    w = instances.workload_batch512()
    insts = w["instances"]
    assert len(insts) == 512 and (w["walks"], w["iters"], w["seed"]) == (64, 5000, 1004)
    ns = np.array([i.n for i in insts])
    assert ns.min() >= 20 and ns.max() <= 150 and ns.min() < 30 and ns.max() > 140
    for k in (0, 1, 2, 511):
        inst = insts[k]
        assert inst.symmetric == (k % 2 == 0)
        assert ((inst.F == inst.F.T).all() and (inst.D == inst.D.T).all()) == inst.symmetric
    assert max(int(i.F.max()) for i in insts) <= 10000
    assert max(int(i.F.max()) for i in insts) > 127    # int16 flows: the int64 family
    # any instance rebuilds alone from (seed, k)
    k = 37
    again = instances.lognormal_instance(int(insts[k].n), 3 * 1_000_003 + k + 1,
                                         insts[k].symmetric)
    assert (again[0] == insts[k].F).all() and (again[1] == insts[k].D).all()


def test_poisson_requests_recipe():
    reqs = instances.poisson_requests(4000, seed=1)
    gaps = np.diff([r.arrival_s for r in reqs])
    assert reqs[0].arrival_s == 0.0 and (gaps >= 0).all()
    assert abs(gaps.mean() - 1 / 2000) < 0.05 / 2000   # rate 2000 per second
    ns = np.array([r.inst.n for r in reqs])
    assert ns.min() >= 12 and ns.max() <= 256
    kinds = {r.inst.kind for r in reqs}
    assert kinds == {"uniform-sym", "uniform-asym", "grid"}


def test_tenure_rules():
    assert instances.periodic_tenure(50) == (45, 55, 100)
    assert instances.periodic_tenure(1) == (1, 2, 2)
    assert instances.paper_tenure(100) == (10, 33, 0)
    assert instances.paper_tenure(5) == (1, 2, 0)
    assert instances.paper_tenure(3) == (1, 1, 0)
    for n in range(2, 257):
        tmin, tmax, period = instances.paper_tenure(n)
        assert 1 <= tmin <= tmax and period == 0
        assert tmin == max(1, math.floor(0.1 * n))
        assert tmax == max(tmin, math.ceil(0.33 * n - 1e-9))
