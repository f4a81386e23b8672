"""GPU parity of the other tabu criteria (Taillard's unit-location rule,
Zhu et al.'s unit marking of Section 3.1) and of the frequency penalty
(Section 7's long-term memory): every walk bit for bit equal to the
oracle's, for one instance, batches, large-n plans, the plain launch form
and the serving loop."""
import numpy as np
import pytest

import oracle
import paper_2307_11248_gb300 as q
from paper_2307_11248_gb300 import instances

pytestmark = pytest.mark.gpu

FIELDS = ["best_cost", "final_cost", "best_iter", "iters_done", "status", "descent_moves",
          "hash", "descent_hash"]
RULES = [(q.TABU_UNIT_LOC, 0), (q.TABU_UNIT, 0), (q.TABU_PAIR, 5), (q.TABU_UNIT_LOC, 2),
         (q.TABU_UNIT, 40)]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is available")
    oracle.build()
    q.lib()
    return torch


def check(g, o, rows=slice(None), n=None):
    for k in FIELDS:
        assert np.array_equal(g[k][rows].astype(np.int64), o[k].astype(np.int64)), k
    P = g["best_p"][rows]
    assert np.array_equal(P[:, :n] if n else P, o["best_p"])


@pytest.mark.parametrize("crit,lam", RULES)
@pytest.mark.parametrize("n,sym,tn", [(12, True, (2, 4, 0)), (50, False, (45, 55, 100)),
                                      (97, True, (3, 13, 0))])
def test_rules_single_instance_bit_exact(n, sym, tn, crit, lam):
    F, D = instances.uniform_instance(n, 800 + n, symmetric=sym)
    if crit == q.TABU_UNIT:  # Zhu et al.'s range [3, 3 + n/10]
        tn = (3, 3 + n // 10, 0)
    W, iters = 5, 400
    prm = q.make_params(W, seed=31, iters=iters, tenure=tn, criterion=crit, freq_penalty=lam)
    with q.Instance(F, D) as inst:
        g = inst.search(prm, freq=True)
    o = oracle.run_walks(F, D, W, seed=31, iters=iters, tenure=tn, criterion=crit, penalty=lam)
    check(g, o)
    for w in range(W):
        p0 = oracle.start_perm(31, w, n)
        *_, fq = oracle.tabu(F, D, p0, iters, *tn, True, 31, w, want_freq=True, criterion=crit,
                             penalty=lam)
        assert np.array_equal(g["freq"][w], fq)


@pytest.mark.parametrize("crit,lam", RULES)
def test_rules_int64_descend_no_aspiration(crit, lam):
    F, D = instances.lognormal_instance(40, 12, symmetric=False)
    tn = (2, 6, 0)
    prm = q.make_params(4, seed=5, iters=300, tenure=tn, descend=True, aspiration=False,
                        criterion=crit, freq_penalty=lam)
    with q.Instance(F, D, force_int64=True) as inst:
        g = inst.search(prm)
    o = oracle.run_walks(F, D, 4, seed=5, iters=300, tenure=tn, descend=True, aspiration=False,
                         criterion=crit, penalty=lam)
    check(g, o)


def test_rules_stall_like_the_oracle():
    """Unit marking with a long tenure and no aspiration stops after
    floor(n/2) moves on an instance whose every delta is zero."""
    n = 11
    F, _ = instances.uniform_instance(n, 3, symmetric=False)
    D = np.full((n, n), 5, dtype=np.int64)
    np.fill_diagonal(D, 0)
    prm = q.make_params(3, seed=1, iters=50, tenure=(100, 100, 0), aspiration=False,
                        criterion=q.TABU_UNIT)
    with q.Instance(F, D) as inst:
        g = inst.search(prm)
    assert (g["iters_done"] == n // 2).all() and (g["status"] == 1).all()
    o = oracle.run_walks(F, D, 3, seed=1, iters=50, tenure=(100, 100, 0), aspiration=False,
                         criterion=q.TABU_UNIT)
    check(g, o)


@pytest.mark.parametrize("threads", [128, 512, 1024])
def test_rules_every_thread_count(threads):
    n = 40
    F, D = instances.uniform_instance(n, 71, symmetric=False)
    tn = (6, 20, 0)
    for crit, lam in [(q.TABU_UNIT_LOC, 3), (q.TABU_UNIT, 1)]:
        prm = q.make_params(3, seed=2, iters=250, tenure=tn, criterion=crit, freq_penalty=lam,
                            threads_per_walk=threads)
        with q.Instance(F, D) as inst:
            g = inst.search(prm)
        o = oracle.run_walks(F, D, 3, seed=2, iters=250, tenure=tn, criterion=crit, penalty=lam)
        check(g, o)


def test_rules_plain_launch_form():
    n = 30
    F, D = instances.uniform_instance(n, 72, symmetric=True)
    prm = q.make_params(4, seed=6, iters=200, tenure=(3, 9, 0), criterion=q.TABU_UNIT_LOC,
                        freq_penalty=2, launch=q.LAUNCH_PLAIN)
    with q.Instance(F, D) as inst:
        g = inst.search(prm)
    o = oracle.run_walks(F, D, 4, seed=6, iters=200, tenure=(3, 9, 0),
                         criterion=q.TABU_UNIT_LOC, penalty=2)
    check(g, o)


@pytest.mark.parametrize("crit,lam", [(q.TABU_UNIT_LOC, 4), (q.TABU_UNIT, 0)])
def test_rules_large_n_workspace_plan(crit, lam):
    n = 220
    F, D = instances.uniform_instance(n, 73, symmetric=False)
    tn = instances.paper_tenure(n)
    prm = q.make_params(2, seed=9, iters=80, tenure=tn, criterion=crit, freq_penalty=lam)
    with q.Instance(F, D) as inst:
        assert inst.plan(prm)["pairs_per_thread"] == 40
        g = inst.search(prm)
    o = oracle.run_walks(F, D, 2, seed=9, iters=80, tenure=tn, criterion=crit, penalty=lam)
    check(g, o)


def test_rules_batch_uneven_n():
    Fs, Ds = [], []
    for k, n in enumerate([16, 45, 33, 90, 200]):
        F, D = instances.uniform_instance(n, 900 + k, symmetric=(k % 2 == 0))
        Fs.append(F)
        Ds.append(D)
    W, iters = 3, 150
    for crit, lam in [(q.TABU_UNIT_LOC, 2), (q.TABU_UNIT, 0), (q.TABU_PAIR, 9)]:
        prm = q.make_params(W, seed=17, iters=iters, tenure=(10, 33, 0), tenure_per_n=True,
                            criterion=crit, freq_penalty=lam)
        with q.Batch(Fs, Ds) as b:
            g = b.search(prm)
        for i, F in enumerate(Fs):
            n = F.shape[0]
            o = oracle.run_walks(F, Ds[i], W, seed=17, iters=iters,
                                 tenure=instances.paper_tenure(n), criterion=crit, penalty=lam)
            check(g, o, rows=slice(i * W, (i + 1) * W), n=n)


def test_rules_served_requests_equal_alone():
    reqs = instances.poisson_requests(4, seed=77, nmin=20, nmax=120)
    rules = [(q.TABU_UNIT_LOC, 0), (q.TABU_UNIT, 3), (q.TABU_PAIR, 2), (q.TABU_UNIT_LOC, 1)]
    with q.Server(slots=4, mem_bytes=128 << 20) as sv:
        tickets = []
        for r, (crit, lam) in zip(reqs, rules):
            prm = q.make_params(4, seed=r.rid, iters=150, tenure=(4, 12, 0), criterion=crit,
                                freq_penalty=lam)
            tickets.append((r, prm, sv.submit(r.inst.F, r.inst.D, prm)))
        for r, prm, t in tickets:
            res, _ = sv.wait(t)
            with q.Instance(r.inst.F, r.inst.D) as inst:
                alone = inst.search(prm)
            for k in FIELDS + ["best_p"]:
                assert np.array_equal(res[k], alone[k]), k


def test_penalty_overflow_is_reported():
    F, D = instances.uniform_instance(50, 1, symmetric=False)
    prm = q.make_params(2, seed=1, iters=1000, tenure=(3, 5, 0), freq_penalty=2**22)
    with q.Instance(F, D) as inst:
        assert inst.info["delta_bytes"] == 4
        with pytest.raises(q.QapError) as e:
            inst.search(prm)
        assert e.value.status == q.EOVERFLOW
    with q.Instance(F, D, force_int64=True) as inst:
        g = inst.search(q.make_params(2, seed=1, iters=100, tenure=(3, 5, 0),
                                      freq_penalty=2**22))
    o = oracle.run_walks(F, D, 2, seed=1, iters=100, tenure=(3, 5, 0), penalty=2**22)
    check(g, o)


def test_bad_rules_are_rejected():
    F, D = instances.uniform_instance(10, 1, symmetric=False)
    with q.Instance(F, D) as inst:
        for kw in [dict(criterion=3), dict(criterion=-1), dict(freq_penalty=-2)]:
            with pytest.raises(q.QapError) as e:
                inst.search(q.make_params(1, seed=1, iters=5, tenure=(1, 2, 0), **kw))
            assert e.value.status == q.EINVAL


def test_rules_int64_flows_in_global_memory():
    """Large n with int16 flows and int64 deltas: the workspace plan with F in
    global memory, under the unit-location criterion and the penalty."""
    F, D = instances.lognormal_instance(230, 31, symmetric=False)
    tn = (20, 60, 0)
    prm = q.make_params(2, seed=3, iters=60, tenure=tn, criterion=q.TABU_UNIT_LOC,
                        freq_penalty=3)
    with q.Instance(F, D, force_int64=True) as inst:
        pl = inst.plan(prm)
        assert pl["workspace"] == 1 and pl["products"] == 0
        g = inst.search(prm, freq=True)
    o = oracle.run_walks(F, D, 2, seed=3, iters=60, tenure=tn, criterion=q.TABU_UNIT_LOC,
                         penalty=3)
    check(g, o)
    for w in range(2):
        p0 = oracle.start_perm(3, w, 230)
        *_, fq = oracle.tabu(F, D, p0, 60, *tn, True, 3, w, want_freq=True,
                             criterion=q.TABU_UNIT_LOC, penalty=3)
        assert np.array_equal(g["freq"][w], fq)
