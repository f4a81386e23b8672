"""GPU parity of the paper's own tenure rule and of its frequency memory.

Section 4.3 draws a tenure in [0.1 n, 0.33 n] for every applied move and
records each applied exchange (r, s) in the lower triangle of the tabu
array.  The kernel's frequency memory must equal the oracle's entry by
entry, for one instance and for a batch of uneven n, with and without a
2opt descent before the tabu phase (descent moves are not counted)."""
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


def oracle_freq(F, D, walk, *, seed, iters, tenure, descend=False, aspiration=True):
    """The oracle's frequency memory of one walk: its start permutation, the
    optional 2opt descent, then the tabu phase with the memory switched on."""
    n = F.shape[0]
    p = oracle.start_perm(seed, walk, n)
    if descend:
        p, _ = oracle.two_opt(F, D, p)
    *_, fq = oracle.tabu(F, D, p, iters, *tenure, aspiration, seed, walk, want_freq=True)
    return fq


def check_freq(fq, iters_done, F, D, walks, **kw):
    n = F.shape[0]
    for w, walk in enumerate(walks):
        ref = oracle_freq(F, D, walk, **kw)
        got = fq[w, :n, :n]
        assert np.array_equal(got, ref), (n, walk)
        assert not np.triu(got).any()             # lower triangle only
        assert got.sum() == iters_done[w]         # one count per applied move
        assert not fq[w, n:, :].any() and not fq[w, :, n:].any()


@pytest.mark.parametrize("n,sym", [(12, True), (50, False), (97, True), (181, False)])
def test_paper_tenure_mode_bit_exact(n, sym):
    """period 0: a tenure drawn from [0.1 n, 0.33 n] for every move."""
    F, D = instances.uniform_instance(n, 300 + n, symmetric=sym)
    tn = instances.paper_tenure(n)
    assert tn[2] == 0
    W, iters = 6, 400
    with q.Instance(F, D) as inst:
        g = inst.search(q.make_params(W, seed=77, iters=iters, tenure=tn))
    o = oracle.run_walks(F, D, W, seed=77, iters=iters, tenure=tn)
    for k in FIELDS + ["best_p"]:
        assert np.array_equal(g[k].astype(np.int64), o[k].astype(np.int64)), k


def test_paper_tenure_int64_lognormal():
    F, D = instances.lognormal_instance(64, 5, symmetric=False)
    tn = instances.paper_tenure(64)
    with q.Instance(F, D, force_int64=True) as one:
        g = one.search(q.make_params(4, seed=9, iters=600, tenure=tn, descend=True))
    o = oracle.run_walks(F, D, 4, seed=9, iters=600, tenure=tn, descend=True)
    for k in FIELDS + ["best_p"]:
        assert np.array_equal(g[k].astype(np.int64), o[k].astype(np.int64)), k


@pytest.mark.parametrize("tenure", ["paper", "baseline"])
def test_frequency_memory_single_instance(tenure):
    n = 50
    F, D = instances.uniform_instance(n, 11, symmetric=False)
    tn = instances.paper_tenure(n) if tenure == "paper" else instances.periodic_tenure(n)
    W, iters = 5, 500
    with q.Instance(F, D) as inst:
        g = inst.search(q.make_params(W, seed=21, iters=iters, tenure=tn), freq=True)
        plain = inst.search(q.make_params(W, seed=21, iters=iters, tenure=tn))
    assert g["freq"].shape == (W, n, n)
    for k in FIELDS:                              # the memory changes nothing else
        assert np.array_equal(g[k], plain[k]), k
    check_freq(g["freq"], g["iters_done"], F, D, range(W), seed=21, iters=iters, tenure=tn)


def test_frequency_memory_after_descent_and_stall():
    """Descent moves are not counted; a walk that stalls (every move tabu
    and none aspirated) counts only the moves it applied."""
    n = 9
    F, D = instances.uniform_instance(n, 4, symmetric=True)
    tn = (40, 40, 0)                              # 36 pairs: the walk stalls
    with q.Instance(F, D) as inst:
        g = inst.search(q.make_params(4, seed=2, iters=100, tenure=tn, descend=True,
                                      aspiration=False), freq=True)
    assert (g["status"] == 1).all() and (g["iters_done"] < 100).all()
    check_freq(g["freq"], g["iters_done"], F, D, range(4), seed=2, iters=100, tenure=tn,
               descend=True, aspiration=False)


def test_frequency_memory_large_n_workspace_plan():
    n = 230
    F, D = instances.uniform_instance(n, 12, symmetric=False)
    tn = instances.paper_tenure(n)
    with q.Instance(F, D) as inst:
        assert inst.plan(q.make_params(2, seed=3, iters=60, tenure=tn))["pairs_per_thread"] == 40
        g = inst.search(q.make_params(2, seed=3, iters=60, tenure=tn, walk_base=5), freq=True)
    check_freq(g["freq"], g["iters_done"], F, D, [5, 6], seed=3, iters=60, tenure=tn)


def test_frequency_memory_batch():
    Fs, Ds = [], []
    for k, n in enumerate([14, 40, 33, 71]):
        F, D = instances.uniform_instance(n, 600 + k, symmetric=(k % 2 == 1))
        Fs.append(F)
        Ds.append(D)
    W, iters = 3, 300
    with q.Batch(Fs, Ds) as b:
        m = b.p_stride
        g = b.search(q.make_params(W, seed=13, iters=iters, tenure=(10, 33, 0),
                                   tenure_per_n=True), freq=True)
    assert g["freq"].shape == (len(Fs) * W, m, m)
    for i in range(len(Fs)):
        n = Fs[i].shape[0]
        tn = instances.paper_tenure(n)
        rows = slice(i * W, (i + 1) * W)
        check_freq(g["freq"][rows], g["iters_done"][rows], Fs[i], Ds[i], range(W), seed=13,
                   iters=iters, tenure=tn)


def test_frequency_memory_async_device_buffer(gpu):
    torch = gpu
    n = 40
    F, D = instances.uniform_instance(n, 8, symmetric=False)
    tn = instances.paper_tenure(n)
    W = 4
    prm = q.make_params(W, seed=6, iters=250, tenure=tn)
    with q.Instance(F, D) as inst:
        outs = inst.device_outputs(W)
        outs["freq"] = torch.full((W, n, n), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()                  # the buffers are written
        s = torch.cuda.Stream()
        inst.search_async(prm, outs, stream=s)
        s.synchronize()
    fq = outs["freq"].cpu().numpy()
    check_freq(fq, outs["iters_done"].cpu().numpy(), F, D, range(W), seed=6, iters=250,
               tenure=tn)
