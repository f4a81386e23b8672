"""GPU parity of the int64 element path: instances whose values fall outside
the narrow paths (F beyond int16, D beyond int8, or dot-product sums that
could reach 2^31) run with int64 flows, distances and arithmetic.  Section
2.1 puts no range on F or D; every input whose bound B = (n^2 + 8n + 32)
max|F| max|D| stays below 2^62 is searched, bit-exact with the oracle."""
import numpy as np
import pytest

import oracle
import paper_2307_11248_gb300 as q
from paper_2307_11248_gb300 import instances

pytestmark = pytest.mark.gpu

FIELDS = ["best_p", "best_cost", "final_cost", "best_iter", "iters_done", "status", "hash",
          "descent_hash", "descent_moves"]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is available")
    oracle.build()
    q.lib()
    return torch


def assert_same(g, o, tag):
    for f in FIELDS:
        assert np.array_equal(g[f].astype(np.int64), o[f].astype(np.int64)), (tag, f)


def case(k):
    rng = np.random.default_rng(9000 + k)
    n = int(rng.choice([2, 3, 5, 9, 16, 17, 33, 48, 64, 90, 101, 127, 150, 181, 182, 220, 256]))
    sym = bool(rng.integers(2))
    kind = int(rng.integers(3))
    if kind == 0:      # distances beyond a byte
        F = rng.integers(0, 100, size=(n, n))
        D = rng.integers(-30000, 30001, size=(n, n))
    elif kind == 1:    # flows up to 2^20, signed distances beyond a byte
        F = rng.integers(-(1 << 20), (1 << 20) + 1, size=(n, n))
        D = rng.integers(-3000, 3001, size=(n, n))
    else:              # flows and distances both large
        F = rng.integers(0, (1 << 20) + 1, size=(n, n))
        D = rng.integers(0, 30001, size=(n, n))
    F, D = F.astype(np.int64), D.astype(np.int64)
    if sym:
        F = np.triu(F) + np.triu(F, 1).T
        D = np.triu(D) + np.triu(D, 1).T
    if rng.integers(2):
        np.fill_diagonal(F, 0)
        np.fill_diagonal(D, 0)
    crit = int(rng.integers(3))
    lam = int(rng.choice([0, 0, 5, 1000]))
    descend = bool(rng.integers(2))
    tmin = int(rng.integers(1, max(2, n // 3) + 1))
    tn = (tmin, tmin + int(rng.integers(0, 5)), int(rng.choice([0, 0, 7, 2 * n])))
    iters = int(rng.integers(20, 100)) if n <= 150 else 30
    asp = bool(rng.integers(4) > 0)
    return n, F, D, crit, lam, descend, tn, iters, asp


@pytest.mark.parametrize("k", range(24))
def test_wide_random_configurations_bit_exact(k):
    n, F, D, crit, lam, descend, tn, iters, asp = case(k)
    W = 3
    prm = q.make_params(W, seed=300 + k, iters=iters, tenure=tn, aspiration=asp,
                        descend=descend, max_descent=60, criterion=crit, freq_penalty=lam)
    with q.Instance(F, D) as inst:
        assert inst.info["flow_bytes"] == 8 and inst.info["dist_bytes"] == 8
        assert inst.info["delta_bytes"] == 8
        g = inst.search(prm)
    o = oracle.run_walks(F, D, W, seed=300 + k, iters=iters, tenure=tn, aspiration=asp,
                         descend=descend, max_descent=60, criterion=crit, penalty=lam)
    assert_same(g, o, k)


def test_int16_extremes_at_n256_take_the_wide_path():
    """F in {-32768, 32767}, D in {-128, 127}, asymmetric, n = 256: int16 and
    int8 storage would hold the values, but 2n products of 2^22 reach 2^31,
    so the instance runs on the int64 path."""
    rng = np.random.default_rng(77)
    n = 256
    F = np.where(rng.integers(2, size=(n, n)) == 1, -32768, 32767).astype(np.int64)
    D = np.where(rng.integers(2, size=(n, n)) == 1, -128, 127).astype(np.int64)
    tn = (20, 40, 0)
    prm = q.make_params(3, seed=5, iters=40, tenure=tn, descend=True, max_descent=20)
    with q.Instance(F, D) as inst:
        assert inst.info["flow_bytes"] == 8
        plan = inst.plan(prm)
        assert plan["workspace"] == 1
        g = inst.search(prm)
    o = oracle.run_walks(F, D, 3, seed=5, iters=40, tenure=tn, descend=True, max_descent=20)
    assert_same(g, o, "n256 extremes")


def test_int16_extremes_at_n255_stay_narrow():
    rng = np.random.default_rng(78)
    n = 255
    F = np.where(rng.integers(2, size=(n, n)) == 1, -32768, 32767).astype(np.int64)
    D = np.where(rng.integers(2, size=(n, n)) == 1, -128, 127).astype(np.int64)
    tn = (20, 40, 0)
    prm = q.make_params(2, seed=6, iters=30, tenure=tn)
    with q.Instance(F, D) as inst:
        assert inst.info["flow_bytes"] == 2 and inst.info["dist_bytes"] == 1
        g = inst.search(prm)
    o = oracle.run_walks(F, D, 2, seed=6, iters=30, tenure=tn)
    assert_same(g, o, "n255 extremes")


def test_huge_flows_small_distances():
    """Flows of 2^40 with distances up to 2^12: B = 592 * 2^52 < 2^62 at
    n = 20 (592 = n^2 + 8n + 32)."""
    rng = np.random.default_rng(79)
    n = 20
    F = rng.integers(-(1 << 40), (1 << 40) + 1, size=(n, n)).astype(np.int64)
    D = rng.integers(-(1 << 12), (1 << 12) + 1, size=(n, n)).astype(np.int64)
    tn = (3, 7, 0)
    prm = q.make_params(4, seed=8, iters=200, tenure=tn, descend=True)
    with q.Instance(F, D) as inst:
        g = inst.search(prm)
        P = np.stack([rng.permutation(n) for _ in range(5)]).astype(np.int32)
        assert inst.cost(P).tolist() == [oracle.cost(F, D, p) for p in P]
    o = oracle.run_walks(F, D, 4, seed=8, iters=200, tenure=tn, descend=True)
    assert_same(g, o, "huge flows")


def test_bound_beyond_the_int64_path_is_refused():
    n = 20
    F = np.full((n, n), 1 << 40, dtype=np.int64)
    D = np.full((n, n), 1 << 16, dtype=np.int64)
    with pytest.raises(q.QapError) as e:
        q.qap_create(F, D)
    assert e.value.status == q.EOVERFLOW


@pytest.mark.parametrize("n,sym", [(40, False), (100, True), (140, False), (181, True)])
def test_wide_plans_with_p_in_shared_or_global_memory(n, sym):
    """Distances up to 1000 on the register plans: P in shared memory while
    it fits, else in the per-CTA workspace."""
    F, D = instances.uniform_instance(n, 950 + n, symmetric=sym)
    D = D * 10  # up to 990: beyond int8
    tn = instances.periodic_tenure(n)
    prm = q.make_params(4, seed=12, iters=150, tenure=tn, descend=True)
    with q.Instance(F, D) as inst:
        assert inst.info["flow_bytes"] == 8
        plan = inst.plan(prm)
        assert plan["workspace"] == 0
        g = inst.search(prm)
    o = oracle.run_walks(F, D, 4, seed=12, iters=150, tenure=tn, descend=True)
    assert_same(g, o, n)


def test_batch_with_one_wide_instance_runs_wide():
    """One instance with distances beyond a byte puts the whole batch on the
    int64 path; every instance still equals its oracle search."""
    Fs, Ds = [], []
    for k, n in enumerate([12, 37, 50, 23]):
        F, D = instances.uniform_instance(n, 60 + k, symmetric=(k % 2 == 0))
        Fs.append(F)
        Ds.append(D)
    Ds[2] = Ds[2] * 300  # up to 29700
    W, tn = 3, (4, 10, 0)
    with q.Batch(Fs, Ds) as b:
        assert b.info["delta_bytes"] == 8
        g = b.search(q.make_params(W, seed=14, iters=120, tenure=tn, descend=True))
    for i, (F, D) in enumerate(zip(Fs, Ds)):
        n = F.shape[0]
        o = oracle.run_walks(F, D, W, seed=14, iters=120, tenure=tn, descend=True)
        rows = slice(i * W, (i + 1) * W)
        for f in FIELDS:
            if f == "best_p":
                assert np.array_equal(g[f][rows, :n], o[f]), (i, f)
            else:
                assert np.array_equal(g[f][rows].astype(np.int64), o[f].astype(np.int64)), (i, f)


def test_server_request_on_the_wide_path():
    F, D = instances.uniform_instance(30, 61, symmetric=False)
    D = D * 500
    tn = (5, 9, 0)
    prm = q.make_params(4, seed=15, iters=100, tenure=tn)
    with q.Server(slots=4, mem_bytes=64 << 20) as sv:
        res, _ = sv.wait(sv.submit(F, D, prm), timeout_ms=60000)
    o = oracle.run_walks(F, D, 4, seed=15, iters=100, tenure=tn)
    assert_same(res, o, "server")
