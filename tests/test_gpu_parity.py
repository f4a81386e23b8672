"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Integer work, so the bar is bit-exact: every walk's best permutation, best
cost, final cost, best iteration, iteration count, status, 2opt move count
and both trajectory hashes must equal the oracle's.
"""
import numpy as np
import pytest

import oracle
import paper_2307_11248_gb300 as q
from paper_2307_11248_gb300 import instances

pytestmark = pytest.mark.gpu

FIELDS = ["best_p", "best_cost", "final_cost", "best_iter", "iters_done", "status",
          "descent_moves", "hash", "descent_hash"]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is available")
    oracle.build()
    q.lib()
    return torch


def run_both(F, D, walks, *, seed, iters=0, tenure=(1, 1, 0), aspiration=True, descend=False,
             max_descent=-1, walk_base=0, starts=None, force_int64=False, threads=0,
             launch=q.LAUNCH_PERSISTENT, walk_ids=None):
    with q.Instance(F, D, force_int64=force_int64) as inst:
        prm = q.make_params(walks, seed=seed, iters=iters, tenure=tenure, aspiration=aspiration,
                            descend=descend, max_descent=max_descent, walk_base=walk_base,
                            launch=launch, threads_per_walk=threads)
        g = inst.search(prm, starts)
        info = inst.info
    ids = walk_ids if walk_ids is not None else np.arange(walk_base, walk_base + walks)
    o = oracle.run_walks(F, D, walks, seed=seed, iters=iters, tenure=tenure,
                         aspiration=aspiration, descend=descend, max_descent=max_descent,
                         walk_ids=ids, starts=starts)
    return g, o, info


def assert_same(g, o, fields=FIELDS, rows=None):
    for k in fields:
        a = g[k] if rows is None else g[k][rows]
        b = o[k]
        assert np.array_equal(a.astype(np.int64), b.astype(np.int64)), (
            f"{k} differs at walks {np.nonzero((a != b).reshape(len(a), -1).any(1))[0][:8]}")


def rand_instance(seed, n, lo=-20, hi=20, diag=True, sym=False):
    rng = np.random.default_rng(seed)
    F = rng.integers(lo, hi + 1, size=(n, n))
    D = rng.integers(max(lo, -128), min(hi, 127) + 1, size=(n, n))
    if sym:
        F = np.triu(F) + np.triu(F, 1).T
        D = np.triu(D) + np.triu(D, 1).T
    if not diag:
        np.fill_diagonal(F, 0)
        np.fill_diagonal(D, 0)
    return F.astype(np.int64), D.astype(np.int64)


# ---------------------------------------------------------------------------
# Eq. 1
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,sym", [(2, False), (9, True), (50, False), (181, False)])
def test_cost_matches_oracle(n, sym):
    F, D = rand_instance(n, n, lo=-99, hi=99, sym=sym)
    rng = np.random.default_rng(1)
    P = np.stack([rng.permutation(n) for _ in range(37)]).astype(np.int32)
    with q.Instance(F, D) as inst:
        got = inst.cost(P)
    assert got.tolist() == [oracle.cost(F, D, p) for p in P]


def test_cost_rejects_non_permutation():
    F, D = rand_instance(3, 6)
    with q.Instance(F, D) as inst:
        with pytest.raises(q.QapError) as e:
            inst.cost(np.array([[0, 1, 2, 3, 4, 4]]))
    assert e.value.status == q.EINVAL


# ---------------------------------------------------------------------------
# the named workloads
# ---------------------------------------------------------------------------

def test_sym12_2opt_bit_exact():
    w = instances.workload_sym12()
    g, o, info = run_both(w["F"], w["D"], w["walks"], seed=w["seed"], descend=True)
    assert info["delta_bytes"] == 4 and info["sym_flow"] and info["sym_dist"]
    assert_same(g, o)
    # 2opt results are local minima
    for k in range(4):
        p = g["best_p"][k]
        assert oracle.cost(w["F"], w["D"], p) == g["best_cost"][k]
        assert all(oracle.delta(w["F"], w["D"], p, r, s) >= 0
                   for r in range(12) for s in range(r + 1, 12))


def test_asym50_tabu_reduced_bit_exact():
    w = instances.workload_asym50()
    g, o, _ = run_both(w["F"], w["D"], 24, seed=w["seed"], iters=1500, tenure=w["tenure"])
    assert_same(g, o)
    assert (g["iters_done"] == 1500).all()


def test_asym50_full_size_sampled_walks():
    """The full workload (256 walks x 5000 iterations) in the persistent
    launch the benchmark times; sampled walks checked against the oracle."""
    w = instances.workload_asym50()
    with q.Instance(w["F"], w["D"]) as inst:
        prm = q.make_params(w["walks"], seed=w["seed"], iters=w["iters"], tenure=w["tenure"])
        g = inst.search(prm)
    rows = np.array([0, 1, 101, 254, 255])
    o = oracle.run_walks(w["F"], w["D"], len(rows), seed=w["seed"], iters=w["iters"],
                         tenure=w["tenure"], walk_ids=rows)
    assert_same(g, o, rows=rows)
    # every walk: best_p is a permutation whose Eq. 1 cost is best_cost
    n = 50
    assert (np.sort(g["best_p"], axis=1) == np.arange(n)).all()
    with q.Instance(w["F"], w["D"]) as inst:
        assert np.array_equal(inst.cost(g["best_p"]), g["best_cost"])
    assert (g["best_cost"] <= g["final_cost"]).all()


def test_grid100_descend_then_tabu_reduced_bit_exact():
    w = instances.workload_grid100()
    g, o, info = run_both(w["F"], w["D"], 12, seed=w["seed"], iters=600, tenure=w["tenure"],
                          descend=True)
    assert info["sym_flow"] and info["sym_dist"]
    assert_same(g, o)
    assert (g["descent_moves"] > 0).all()


def test_grid100_full_iterations_sampled_walks():
    """Walks 3 and 700 of the n=100 grid workload at its full 10000
    iterations (walk_base selects the walk id, so draws match the full run)."""
    w = instances.workload_grid100()
    for wid in (3, 700):
        g, o, _ = run_both(w["F"], w["D"], 1, seed=w["seed"], iters=w["iters"],
                           tenure=w["tenure"], descend=True, walk_base=wid)
        assert_same(g, o)


@pytest.mark.parametrize("k", [0, 1, 5, 12])
def test_lognormal_batch_instances_int64(k):
    inst = instances.batch_instances(16, 3)[k]
    n = inst.n
    tn = instances.periodic_tenure(n)
    g, o, info = run_both(inst.F, inst.D, 6, seed=1004, iters=400, tenure=tn, force_int64=True)
    assert info["delta_bytes"] == 8
    assert_same(g, o)


# ---------------------------------------------------------------------------
# arithmetic paths and launch-shape independence
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,sym,diag", [(2, False, True), (3, False, True), (5, True, True),
                                        (17, False, True), (31, True, False), (64, False, True),
                                        (97, False, False), (181, True, False)])
def test_signed_values_and_diagonals(n, sym, diag):
    F, D = rand_instance(100 + n, n, lo=-120, hi=120, diag=diag, sym=sym)
    iters = 300 if n < 100 else 60
    tn = (max(1, n // 4), max(1, n // 2), 0)
    g, o, _ = run_both(F, D, 5, seed=77, iters=iters, tenure=tn, descend=(n % 2 == 1))
    assert_same(g, o)


@pytest.mark.parametrize("n,sym,descend", [(200, True, False), (256, True, True),
                                            (190, False, False), (256, False, True)])
def test_large_n_global_workspace(n, sym, descend):
    """n > 181: deltas and tabu stamps in a device workspace; asymmetric
    n = 256 also reads F from global memory."""
    F, D = instances.uniform_instance(n, 300 + n, symmetric=sym)
    iters = 60
    tn = instances.periodic_tenure(n)
    g, o, info = run_both(F, D, 3, seed=19, iters=iters, tenure=tn, descend=descend,
                          max_descent=40)
    assert_same(g, o)
    assert (g["iters_done"] == iters).all()


def test_large_n_plain_and_persistent_agree():
    F, D = instances.grid_instance(230, 4)
    prm = dict(seed=2, iters=40, tenure=(10, 30, 0))
    g1, o, _ = run_both(F, D, 2, launch=q.LAUNCH_PLAIN, **prm)
    assert_same(g1, o)


def test_force_int64_gives_same_results():
    w = instances.workload_asym50()
    a, o, ia = run_both(w["F"], w["D"], 8, seed=5, iters=700, tenure=w["tenure"])
    b, _, ib = run_both(w["F"], w["D"], 8, seed=5, iters=700, tenure=w["tenure"],
                        force_int64=True)
    assert ia["delta_bytes"] == 4 and ib["delta_bytes"] == 8
    assert_same(a, o)
    assert_same(b, o)


@pytest.mark.parametrize("threads", [128, 256, 512, 1024])
def test_threads_per_walk_do_not_change_results(threads):
    F, D = rand_instance(7, 40, lo=0, hi=99, diag=False)
    g, o, _ = run_both(F, D, 9, seed=3, iters=500, tenure=(20, 40, 80), threads=threads)
    assert_same(g, o)


def test_plain_launch_equals_persistent():
    F, D = rand_instance(8, 23, lo=0, hi=60, diag=False)
    g, o, _ = run_both(F, D, 7, seed=4, iters=250, tenure=(5, 9, 0),
                       launch=q.LAUNCH_PLAIN)
    assert_same(g, o)


def test_walk_base_selects_the_same_walks():
    F, D = rand_instance(9, 19, lo=0, hi=50, diag=False)
    with q.Instance(F, D) as inst:
        full = inst.search(q.make_params(8, seed=11, iters=200, tenure=(3, 8, 0)))
        part = inst.search(q.make_params(3, seed=11, iters=200, tenure=(3, 8, 0), walk_base=5))
    for k in FIELDS:
        assert np.array_equal(full[k][5:8], part[k])


# ---------------------------------------------------------------------------
# degenerate cases
# ---------------------------------------------------------------------------

def test_stall_when_every_move_is_tabu():
    F, D = rand_instance(10, 3, lo=0, hi=9, diag=False)
    g, o, _ = run_both(F, D, 4, seed=2, iters=10, tenure=(100, 100, 0), aspiration=False)
    assert_same(g, o)
    assert (g["status"] == 1).all() and (g["iters_done"] == 3).all()


def test_zero_iterations_and_descent_cap():
    F, D = rand_instance(11, 30, lo=0, hi=99, diag=False)
    g, o, _ = run_both(F, D, 4, seed=6, iters=0)
    assert_same(g, o)
    g, o, _ = run_both(F, D, 4, seed=6, iters=0, descend=True, max_descent=3)
    assert_same(g, o)
    assert (g["descent_moves"] == 3).all()


def test_given_starts():
    F, D = rand_instance(12, 26, lo=0, hi=99, diag=False)
    rng = np.random.default_rng(0)
    starts = np.stack([rng.permutation(26) for _ in range(5)]).astype(np.int32)
    g, o, _ = run_both(F, D, 5, seed=8, iters=300, tenure=(4, 9, 13), starts=starts)
    assert_same(g, o)


def test_n_beyond_256_is_unsupported():
    F = np.zeros((257, 257), dtype=np.int64)
    with pytest.raises(q.QapError) as e:
        q.qap_create(F, F)
    assert e.value.status == q.EUNSUPPORTED


def test_invalid_parameters_are_rejected():
    F, D = rand_instance(13, 10)
    with q.Instance(F, D) as inst:
        for kw in [dict(iters=10, tenure=(0, 3, 0)), dict(iters=10, tenure=(5, 3, 0)),
                   dict(iters=-1), dict(phase_x=2), dict(phase_x=-1)]:
            with pytest.raises(q.QapError) as e:
                inst.search(q.make_params(2, seed=1, **kw))
            assert e.value.status == q.EINVAL
        bad = np.tile(np.arange(10, dtype=np.int32), (2, 1))
        bad[1, 0] = 1
        with pytest.raises(q.QapError) as e:
            inst.search(q.make_params(2, seed=1), starts=bad)
        assert e.value.status == q.EINVAL
        with pytest.raises(q.QapError) as e:
            inst.search(q.make_params(2, seed=1, threads_per_walk=300))
        assert e.value.status == q.EINVAL


def test_convenience_entry_points():
    w = instances.workload_sym12()
    with q.Instance(w["F"], w["D"]) as inst:
        bp, bc, moves = q.qap_2opt(inst.h, 6, w["seed"])
        tp, tc, ti, ts = q.qap_tabu(inst.h, 6, 100, (3, 6, 0), True, 9)
    o = oracle.run_walks(w["F"], w["D"], 6, seed=w["seed"], descend=True)
    assert np.array_equal(bp, o["best_p"]) and np.array_equal(bc, o["best_cost"])
    assert np.array_equal(moves, o["descent_moves"])
    t = oracle.run_walks(w["F"], w["D"], 6, seed=9, iters=100, tenure=(3, 6, 0))
    assert np.array_equal(tp, t["best_p"]) and np.array_equal(tc, t["best_cost"])
    assert np.array_equal(ti, t["best_iter"]) and np.array_equal(ts, t["status"])


def test_async_search_in_cuda_graph(gpu):
    torch = gpu
    w = instances.workload_asym50()
    with q.Instance(w["F"], w["D"]) as inst:
        prm = q.make_params(16, seed=w["seed"], iters=300, tenure=w["tenure"])
        outs = inst.device_outputs(16)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            inst.search_async(prm, outs, stream=s)  # first run outside capture
        s.synchronize()
        first = {k: v.clone() for k, v in outs.items()}
        for v in outs.values():
            v.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            inst.search_async(prm, outs, stream=s)
        g.replay()
        torch.cuda.synchronize()
        for k in outs:
            assert torch.equal(outs[k], first[k]), k
    o = oracle.run_walks(w["F"], w["D"], 16, seed=w["seed"], iters=300, tenure=w["tenure"])
    assert np.array_equal(first["best_cost"].cpu().numpy(), o["best_cost"])
    assert np.array_equal(first["hash"].cpu().numpy().view(np.uint64), o["hash"])


@pytest.mark.parametrize("n,sym,form,products", [
    (2, False, 0, 1), (3, False, 0, 1), (5, False, 0, 1), (17, False, 0, 1), (50, False, 0, 1),
    (100, False, 0, 1), (50, True, 0, 1), (100, True, 0, 1), (170, False, 0, 0),
    (5, False, 1, 0), (50, False, 1, 0), (50, True, 1, 0), (100, False, 1, 0)])
def test_phase_x_forms_bit_exact(n, sym, form, products):
    """Phase X from maintained products (int8 flows, when M fits shared
    memory: the automatic form) and by dot products (asked for, or where the
    products do not apply): both equal the oracle."""
    F, D = instances.uniform_instance(n, 420 + n, symmetric=sym)
    prm = q.make_params(4, seed=13, iters=200, tenure=(3, 9, 0), descend=True, phase_x=form)
    with q.Instance(F, D) as inst:
        assert inst.plan(prm)["products"] == products
        g = inst.search(prm)
    o = oracle.run_walks(F, D, 4, seed=13, iters=200, tenure=(3, 9, 0), descend=True)
    for k in ["best_p", "best_cost", "final_cost", "best_iter", "iters_done", "hash",
              "descent_hash", "descent_moves"]:
        assert np.array_equal(g[k].astype(np.int64), o[k].astype(np.int64)), k
