"""GPU parity of the batched form: many instances of uneven n in one
persistent launch.  Each instance's walks must equal the oracle's walks of
that instance alone (same walk ids), bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2307_11248_gb300 as q
from paper_2307_11248_gb300 import instances

pytestmark = pytest.mark.gpu

FIELDS = ["best_cost", "final_cost", "best_iter", "iters_done", "status", "descent_moves",
          "hash", "descent_hash"]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is available")
    oracle.build()
    q.lib()
    return torch


def check_instance(g, inst_idx, W, F, D, **kw):
    n = F.shape[0]
    rows = slice(inst_idx * W, (inst_idx + 1) * W)
    o = oracle.run_walks(F, D, W, walk_ids=np.arange(W), **kw)
    for k in FIELDS:
        assert np.array_equal(g[k][rows].astype(np.int64), o[k].astype(np.int64)), (inst_idx, k)
    assert np.array_equal(g["best_p"][rows, :n], o["best_p"]), (inst_idx, "best_p")


@pytest.mark.parametrize("phase_x", [q.PHASE_X_AUTO, q.PHASE_X_DOTS])
def test_lognormal_batch_int64_bit_exact(phase_x):
    """Lognormal int16 flows with int64 deltas: the maintained-products
    classes (automatic) and the dot-product ones (asked for) equal the
    oracle."""
    insts = instances.batch_instances(10, 3)
    W, iters = 4, 300
    with q.Batch([i.F for i in insts], [i.D for i in insts], force_int64=True) as b:
        assert b.info["delta_bytes"] == 8 and b.info["count"] == 10
        tn = (20, 40, 60)
        prm = q.make_params(W, seed=1004, iters=iters, tenure=tn, phase_x=phase_x)
        classes, _ = b.classes(prm)
        forms = {c["products"] for c in classes}
        assert forms <= ({1, 2} if phase_x == q.PHASE_X_AUTO else {0}), forms
        g = b.search(prm)
    for i, inst in enumerate(insts):
        check_instance(g, i, W, inst.F, inst.D, seed=1004, iters=iters, tenure=tn)


def test_uniform_batch_int8_descend_then_tabu():
    Fs, Ds = [], []
    for k, n in enumerate([12, 37, 50, 23, 64, 9]):
        F, D = instances.uniform_instance(n, 50 + k, symmetric=(k % 2 == 0))
        Fs.append(F)
        Ds.append(D)
    W = 5
    with q.Batch(Fs, Ds) as b:
        assert b.info["delta_bytes"] == 4
        g = b.search(q.make_params(W, seed=7, iters=250, tenure=(5, 15, 30), descend=True))
    for i in range(len(Fs)):
        check_instance(g, i, W, Fs[i], Ds[i], seed=7, iters=250, tenure=(5, 15, 30),
                       descend=True)


def test_tenure_per_n_matches_each_instance_rule():
    Fs, Ds = [], []
    for k, n in enumerate([20, 33, 47]):
        F, D = instances.uniform_instance(n, 70 + k, symmetric=False)
        Fs.append(F)
        Ds.append(D)
    W = 3
    with q.Batch(Fs, Ds) as b:
        g = b.search(q.make_params(W, seed=8, iters=300, tenure=(90, 110, 200), tenure_per_n=True))
    for i in range(3):
        check_instance(g, i, W, Fs[i], Ds[i], seed=8, iters=300,
                       tenure=instances.periodic_tenure(Fs[i].shape[0]))


def test_batch_equals_single_instance_searches():
    Fs, Ds = [], []
    for k, n in enumerate([30, 45, 20]):
        F, D = instances.lognormal_instance(n, 90 + k, symmetric=False)
        Fs.append(F)
        Ds.append(D)
    W = 6
    prm = q.make_params(W, seed=3, iters=400, tenure=(4, 12, 0), walk_base=17)
    with q.Batch(Fs, Ds, force_int64=True) as b:
        g = b.search(prm)
    for i in range(3):
        with q.Instance(Fs[i], Ds[i], force_int64=True) as inst:
            s = inst.search(prm)
        for k in FIELDS:
            assert np.array_equal(g[k][i * W:(i + 1) * W], s[k]), (i, k)
        assert np.array_equal(g["best_p"][i * W:(i + 1) * W, :Fs[i].shape[0]], s["best_p"])


def test_batch_async_in_cuda_graph(gpu):
    torch = gpu
    insts = instances.batch_instances(6, 11)
    W = 3
    prm = q.make_params(W, seed=5, iters=200, tenure=(10, 20, 40))
    with q.Batch([i.F for i in insts], [i.D for i in insts], force_int64=True) as b:
        outs = b.device_outputs(W)
        s = torch.cuda.Stream()
        b.search_async(prm, outs, stream=s)  # first call writes the tables
        s.synchronize()
        first = {k: v.clone() for k, v in outs.items()}
        for v in outs.values():
            v.zero_()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            b.search_async(prm, outs, stream=s)
        graph.replay()
        graph.replay()
        torch.cuda.synchronize()
        for k in outs:
            assert torch.equal(outs[k], first[k]), k
    g = {k: v.cpu().numpy() for k, v in first.items()}
    g["hash"] = g["hash"].view(np.uint64)
    g["descent_hash"] = g["descent_hash"].view(np.uint64)
    for i, inst in enumerate(insts):
        check_instance(g, i, W, inst.F, inst.D, seed=5, iters=200, tenure=(10, 20, 40))


def test_full_batch512_sampled_walks():
    """The full workload (512 instances, n in [20, 150], 64 walks x 5000
    iterations, int64) in one persistent launch; sampled walks of sampled
    instances checked against the oracle, every walk checked for a valid
    permutation and its Eq. 1 cost."""
    w = instances.workload_batch512()
    insts = w["instances"]
    W, iters = w["walks"], w["iters"]
    # each instance's own tenure rule: [0.9n, 1.1n] redrawn every 2n
    with q.Batch([i.F for i in insts], [i.D for i in insts], force_int64=True) as b:
        g = b.search(q.make_params(W, seed=w["seed"], iters=iters, tenure=(90, 110, 200),
                                   tenure_per_n=True))
    assert (g["iters_done"] == iters).all() and (g["status"] == 0).all()
    rng = np.random.default_rng(0)
    for i in rng.choice(len(insts), size=3, replace=False):
        inst = insts[i]
        rows = [int(i * W + k) for k in (0, W - 1)]
        o = oracle.run_walks(inst.F, inst.D, 2, seed=w["seed"], iters=iters,
                             tenure=instances.periodic_tenure(inst.n), walk_ids=np.array([0, W - 1]))
        for k in FIELDS:
            assert np.array_equal(g[k][rows].astype(np.int64), o[k].astype(np.int64)), (i, k)
        assert np.array_equal(g["best_p"][rows, :inst.n], o["best_p"])
    for i in rng.choice(len(insts), size=20, replace=False):
        inst = insts[i]
        P = g["best_p"][i * W:(i + 1) * W, :inst.n]
        assert (np.sort(P, axis=1) == np.arange(inst.n)).all()
        with q.Instance(inst.F, inst.D, force_int64=True) as one:
            assert np.array_equal(one.cost(P), g["best_cost"][i * W:(i + 1) * W])


def test_batch_with_large_instances_uses_workspace():
    Fs, Ds = [], []
    for k, n in enumerate([240, 30, 190, 77]):
        F, D = instances.uniform_instance(n, 500 + k, symmetric=(k % 2 == 0))
        Fs.append(F)
        Ds.append(D)
    W = 2
    prm = q.make_params(W, seed=4, iters=50, tenure=(90, 110, 200), tenure_per_n=True)
    with q.Batch(Fs, Ds) as b:
        assert b.plan(prm)["pairs_per_thread"] == 40
        g = b.search(prm)
    for i in range(len(Fs)):
        check_instance(g, i, W, Fs[i], Ds[i], seed=4, iters=50,
                       tenure=instances.periodic_tenure(Fs[i].shape[0]))


def test_size_classes_match_single_instance_searches():
    """Instances of very different n take different plans (one launch per
    size class, run on forked streams); every walk still equals the same
    walk of a single-instance search."""
    Fs, Ds = [], []
    for k, n in enumerate([12, 200, 60, 13, 100, 61]):
        F, D = instances.uniform_instance(n, 700 + k, symmetric=(k % 3 == 0))
        Fs.append(F)
        Ds.append(D)
    W = 3
    prm = q.make_params(W, seed=12, iters=120, tenure=(3, 9, 0), descend=True)
    with q.Batch(Fs, Ds) as b:
        pl = b.plan(prm)
        assert pl["classes"] >= 3 and pl["pairs_per_thread"] == 40  # n = 200 leads
        g = b.search(prm)
        g2 = b.search(prm)  # cached classes, second launch
    for k in FIELDS:
        assert np.array_equal(g[k], g2[k]), k
    for i in range(len(Fs)):
        with q.Instance(Fs[i], Ds[i]) as inst:
            s = inst.search(prm)
        for k in FIELDS:
            assert np.array_equal(g[k][i * W:(i + 1) * W], s[k]), (i, k)
        assert np.array_equal(g["best_p"][i * W:(i + 1) * W, :Fs[i].shape[0]], s["best_p"])


def test_autotune_keeps_results_and_reports_classes():
    """The autotuner times every plan that holds each size class and keeps
    the fastest; the walks it then runs are the same walks."""
    Fs, Ds = [], []
    for k, n in enumerate([20, 95, 100, 45, 190]):
        F, D = instances.uniform_instance(n, 40 + k, symmetric=(k % 2 == 1))
        Fs.append(F)
        Ds.append(D)
    W = 8
    prm = q.make_params(W, seed=21, iters=150, tenure=(5, 15, 0))
    with q.Batch(Fs, Ds) as b:
        before = b.search(prm)
        report = b.autotune(prm, trial_iters=60)
        after = b.search(prm)
        pl = b.plan(prm)
    assert len(report) >= 3
    assert sum(r["instances"] for r in report) == len(Fs)
    for r in report:
        assert r["candidates"] >= 1 and r["trial_ms"] > 0
        assert r["trial_ms"] <= r["rule_ms"] or r["rule_ms"] < 0
    assert any(r["candidates"] >= 2 for r in report)
    assert pl["classes"] >= 1
    for k in FIELDS:
        assert np.array_equal(before[k], after[k]), k
    for i, F in enumerate(Fs):  # best_p rows beyond n are padding
        rows = slice(i * W, (i + 1) * W)
        assert np.array_equal(before["best_p"][rows, :F.shape[0]], after["best_p"][rows, :F.shape[0]])


def test_autotune_rejects_fixed_thread_counts():
    F, D = instances.uniform_instance(30, 1, symmetric=False)
    with q.Batch([F], [D]) as b:
        with pytest.raises(q.QapError) as e:
            b.autotune(q.make_params(2, seed=1, iters=10, tenure=(1, 2, 0), threads_per_walk=256))
        assert e.value.status == q.EINVAL


def test_best_walk_per_instance_matches_the_oracle():
    """The host reduction over walks (a walk's best, then the minimum over
    walks, ties to the lowest walk) on a batch search's outputs."""
    insts = instances.batch_instances(5, 17)
    W = 6
    tn = (5, 15, 30)
    with q.Batch([i.F for i in insts], [i.D for i in insts], force_int64=True) as b:
        g = b.search(q.make_params(W, seed=41, iters=150, tenure=tn))
    idx = q.qap_best_walks(g["best_cost"], W)
    for i, inst in enumerate(insts):
        o = oracle.run_walks(inst.F, inst.D, W, seed=41, iters=150, tenure=tn)
        k = int(np.argmin(o["best_cost"]))
        assert idx[i] == k
        assert g["best_cost"][i * W + k] == o["best_cost"][k]
        assert np.array_equal(g["best_p"][i * W + k, :inst.n], o["best_p"][k])
