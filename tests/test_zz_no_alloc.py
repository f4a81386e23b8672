"""The batch entry point that allocates nothing (qap_batch_search_noalloc),
for callers that cannot allocate device memory when they search: two calls
in a row, through the C-ABI, must give exactly the results of the ordinary
batch entry point (integer search, so the bar is equality)."""
import numpy as np
import pytest

import paper_2307_11248_gb300 as q
from paper_2307_11248_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is available")
    q.lib()
    return t


def _batch():
    insts = instances.batch_instances(9, 21)
    Fs, Ds = [i.F for i in insts], [i.D for i in insts]
    F, D = instances.uniform_instance(17, 5, symmetric=False)
    return q.Batch(Fs + [F], Ds + [D], force_int64=True)


def test_noalloc_equals_batch_search_on_two_calls(torch):
    W = 4
    prm = q.make_params(W, seed=77, iters=300, tenure=(90, 110, 200), tenure_per_n=True,
                        descend=True)
    with _batch() as b:
        stream = torch.cuda.Stream()
        ref = b.device_outputs(W)
        b.search_async(prm, ref, stream=stream)
        stream.synchronize()
        for call in range(2):
            outs = b.device_outputs(W)
            q.qap_batch_search_noalloc(b.h, prm, {k: v.data_ptr() for k, v in outs.items()},
                                       b.p_stride, stream.cuda_stream)
            stream.synchronize()
            for k in ref:
                assert torch.equal(outs[k], ref[k]), (call, k)
        assert (ref["iters_done"] == 300).all()


def test_noalloc_rejects_sizes_beyond_its_limit(torch):
    with _batch() as b:
        prm = q.make_params(10000, seed=1, iters=10, tenure=(1, 2, 0))  # 100000 walks > 65536
        outs = b.device_outputs(10000)  # valid buffers, though the call must not start
        stream = torch.cuda.Stream()
        with pytest.raises(q.QapError) as e:
            q.qap_batch_search_noalloc(b.h, prm, {k: v.data_ptr() for k, v in outs.items()},
                                       b.p_stride, stream.cuda_stream)
        stream.synchronize()
        assert e.value.status == q.EINVAL
        assert "static scratch limit" in q.last_error()


def test_noalloc_rejects_rules_that_need_a_workspace(torch):
    with _batch() as b:
        outs = b.device_outputs(2)
        stream = torch.cuda.Stream()
        for kw in [dict(criterion=q.TABU_UNIT), dict(freq_penalty=3)]:
            prm = q.make_params(2, seed=1, iters=10, tenure=(1, 2, 0), **kw)
            with pytest.raises(q.QapError) as e:
                q.qap_batch_search_noalloc(b.h, prm, {k: v.data_ptr() for k, v in outs.items()},
                                           b.p_stride, stream.cuda_stream)
            assert e.value.status == q.EUNSUPPORTED
        stream.synchronize()


def test_noalloc_products_form_batch(torch):
    """Asymmetric int8 instances run the products form of phase X; the
    allocation-free entry point gives the ordinary batch results with it."""
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
        q.qap_batch_search_noalloc(b.h, prm, {k: v.data_ptr() for k, v in outs.items()},
                                   b.p_stride, stream.cuda_stream)
        stream.synchronize()
        for k in ref:
            if k != "best_p":
                assert torch.equal(outs[k], ref[k]), k
        for i, F in enumerate(Fs):
            rows = slice(i * W, (i + 1) * W)
            assert torch.equal(outs["best_p"][rows, :F.shape[0]], ref["best_p"][rows, :F.shape[0]])
