"""The batch entry point that allocates nothing (qap_batch_search_noalloc).

Some callers cannot allocate device memory while they search: a host runtime
whose own allocator owns all of the GPU's memory, or a latency-critical path
where a cudaMalloc and the synchronisation it can bring are not allowed.
For them the library keeps the tables of this entry point in one static
device array.  These tests check, through the C-ABI, that two calls in a row
give exactly the results of the ordinary batch entry point and of the CPU
oracle (integer search, so the bar is equality), that a first call leaves the
device's free memory unchanged, and that the call refuses what its fixed
array cannot hold.  The file sorts last so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle
import paper_2307_11248_gb300 as q
from paper_2307_11248_gb300 import instances

pytestmark = pytest.mark.gpu

FIELDS = ["best_cost", "final_cost", "best_iter", "iters_done", "status", "descent_moves",
          "hash", "descent_hash"]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is available")
    oracle.build()
    q.lib()
    return t


def _instances():
    insts = instances.batch_instances(9, 21)
    Fs, Ds = [i.F for i in insts], [i.D for i in insts]
    F, D = instances.uniform_instance(17, 5, symmetric=False)
    return Fs + [F], Ds + [D]


def _noalloc(b, prm, outs, stream):
    q.qap_batch_search_noalloc(b.h, prm, {k: v.data_ptr() for k, v in outs.items()},
                               b.p_stride, stream.cuda_stream)


def test_first_call_leaves_free_device_memory_unchanged(torch):
    """The process's first call of the allocation-free entry point (this test
    comes first in the file), on a fresh batch: the device's free memory is
    the same before and after the call.  The library's kernels are loaded beforehand by an
    ordinary search of another batch with the same launch plan, and the
    module holding the static array by an Eq. 1 call, so that lazy loading
    of code does not count as the call's allocation."""
    W, iters = 3, 50
    prm = q.make_params(W, seed=3, iters=iters, tenure=(90, 110, 200), tenure_per_n=True)
    Fs, Ds = _instances()
    stream = torch.cuda.Stream()
    with q.Batch(Fs, Ds, force_int64=True) as warm:
        outs = warm.device_outputs(W)
        warm.search_async(prm, outs, stream=stream)
        stream.synchronize()
        plan = warm.plan(prm)
    with q.Instance(Fs[0], Ds[0]) as one:
        one.cost(np.arange(Fs[0].shape[0], dtype=np.int32)[None, :])
    with q.Batch(Fs, Ds, force_int64=True) as b:
        assert b.plan(prm)["threads_per_walk"] == plan["threads_per_walk"]
        outs = b.device_outputs(W)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        _noalloc(b, prm, outs, stream)
        stream.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert (outs["iters_done"] == iters).all()


def test_noalloc_equals_batch_search_and_oracle_on_two_calls(torch):
    W, iters = 4, 300
    prm = q.make_params(W, seed=77, iters=iters, tenure=(90, 110, 200), tenure_per_n=True,
                        descend=True)
    Fs, Ds = _instances()
    with q.Batch(Fs, Ds, force_int64=True) as b:
        stream = torch.cuda.Stream()
        ref = b.device_outputs(W)
        b.search_async(prm, ref, stream=stream)
        stream.synchronize()
        got = []
        for call in range(2):
            outs = b.device_outputs(W)
            _noalloc(b, prm, outs, stream)
            stream.synchronize()
            for k in ref:
                assert torch.equal(outs[k], ref[k]), (call, k)
            got.append({k: v.cpu().numpy() for k, v in outs.items()})
        assert (ref["iters_done"] == iters).all()
    # each instance's walks against the oracle's walks of that instance alone
    for i, (F, D) in enumerate(zip(Fs, Ds)):
        n = F.shape[0]
        o = oracle.run_walks(F, D, W, seed=77, iters=iters, tenure=instances.periodic_tenure(n),
                             descend=True, walk_ids=np.arange(W))
        rows = slice(i * W, (i + 1) * W)
        for g in got:
            for k in FIELDS:
                assert np.array_equal(g[k][rows].astype(np.int64), o[k].astype(np.int64)), (i, k)
            assert np.array_equal(g["best_p"][rows, :n], o["best_p"]), (i, "best_p")


def test_noalloc_gives_back_the_callers_device(torch):
    Fs, Ds = _instances()
    prm = q.make_params(2, seed=1, iters=20, tenure=(2, 4, 0))
    with q.Batch(Fs, Ds, force_int64=True) as b:
        outs = b.device_outputs(2)
        stream = torch.cuda.Stream()
        before = torch.cuda.current_device()
        _noalloc(b, prm, outs, stream)
        stream.synchronize()
        assert torch.cuda.current_device() == before


def test_noalloc_rejects_sizes_beyond_its_limit(torch):
    Fs, Ds = _instances()
    with q.Batch(Fs, Ds, force_int64=True) as b:
        prm = q.make_params(10000, seed=1, iters=10, tenure=(1, 2, 0))  # 100000 walks > 65536
        outs = b.device_outputs(10000)  # valid buffers, though the call must not start
        stream = torch.cuda.Stream()
        with pytest.raises(q.QapError) as e:
            _noalloc(b, prm, outs, stream)
        stream.synchronize()
        assert e.value.status == q.EINVAL
        assert "static scratch limit" in q.last_error()


def test_noalloc_rejects_rules_that_need_a_workspace(torch):
    Fs, Ds = _instances()
    with q.Batch(Fs, Ds, force_int64=True) as b:
        outs = b.device_outputs(2)
        stream = torch.cuda.Stream()
        for kw in [dict(criterion=q.TABU_UNIT), dict(freq_penalty=3)]:
            prm = q.make_params(2, seed=1, iters=10, tenure=(1, 2, 0), **kw)
            with pytest.raises(q.QapError) as e:
                _noalloc(b, prm, outs, stream)
            assert e.value.status == q.EUNSUPPORTED
        stream.synchronize()


def test_noalloc_refuses_a_capturing_stream(torch):
    """Its tables are copied from host memory that the next call
    overwrites, so the call does not let itself be recorded into a graph."""
    Fs, Ds = _instances()
    prm = q.make_params(2, seed=1, iters=10, tenure=(1, 2, 0))
    with q.Batch(Fs, Ds, force_int64=True) as b:
        outs = b.device_outputs(2)
        stream = torch.cuda.Stream()
        _noalloc(b, prm, outs, stream)  # the first call on the device: outside capture
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        status = None
        with torch.cuda.graph(g, stream=stream):
            outs["best_cost"].add_(0)  # something for the graph to hold
            try:
                _noalloc(b, prm, outs, stream)
            except q.QapError as e:
                status = e.status
        assert status == q.EUNSUPPORTED
        assert "captured" in q.last_error()


def test_noalloc_products_form_batch(torch):
    """Asymmetric int8 instances run the products form of phase X; the
    allocation-free entry point gives the ordinary batch results and the
    oracle's with it."""
    Fs, Ds = [], []
    for k, n in enumerate([12, 50, 33, 64]):
        F, D = instances.uniform_instance(n, 880 + k, symmetric=False)
        Fs.append(F)
        Ds.append(D)
    W = 3
    prm = q.make_params(W, seed=5, iters=200, tenure=(4, 12, 0), descend=True)
    with q.Batch(Fs, Ds) as b:
        assert b.plan(prm)["products"] == 1
        stream = torch.cuda.Stream()
        ref = b.device_outputs(W)
        b.search_async(prm, ref, stream=stream)
        stream.synchronize()
        outs = b.device_outputs(W)
        _noalloc(b, prm, outs, stream)
        stream.synchronize()
        got = {k: v.cpu().numpy() for k, v in outs.items()}
        for k in ref:
            if k != "best_p":
                assert torch.equal(outs[k], ref[k]), k
    for i, (F, D) in enumerate(zip(Fs, Ds)):
        n = F.shape[0]
        o = oracle.run_walks(F, D, W, seed=5, iters=200, tenure=(4, 12, 0), descend=True,
                             walk_ids=np.arange(W))
        rows = slice(i * W, (i + 1) * W)
        for k in FIELDS:
            assert np.array_equal(got[k][rows].astype(np.int64), o[k].astype(np.int64)), (i, k)
        assert np.array_equal(got["best_p"][rows, :n], o["best_p"]), (i, "best_p")
