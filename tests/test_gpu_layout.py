"""GPU parity of the interleaved pair layout: with int16 flows and up to 512
threads per walk, thread j of row u owns the pairs (u, u + 1 + j + i c_u).
Every walk must equal the oracle's bit for bit, for int32 and int64 deltas,
each thread count, slot counts on both sides of the rescan's two forms (up
to 8 and above), the pair, unit-location and unit criteria (whose restamps
look up a pair's slot) and the frequency memory."""
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


def wide_flow_instance(n, seed, symmetric):
    """F in [0, 300] (its differences do not fit a byte, so the flows are
    int16), D in [0, 99]; the int32 bound holds up to n = 140."""
    F, _ = instances.uniform_instance(n, seed, symmetric=symmetric, lo=0, hi=300)
    _, D = instances.uniform_instance(n, seed + 1, symmetric=symmetric)
    return F, D


# (n, threads per walk, slots the plan is expected to take)
PLANS = [(30, 128, 4), (40, 128, 12), (30, 256, 6), (50, 512, 4), (70, 512, 8),
         (120, 512, 16), (140, 512, 24)]
RULES = [(q.TABU_PAIR, 0), (q.TABU_UNIT_LOC, 2), (q.TABU_UNIT, 0)]


@pytest.mark.parametrize("int64", [False, True])
@pytest.mark.parametrize("n,threads,slots", PLANS)
def test_interleaved_layout_bit_exact(n, threads, slots, int64):
    F, D = wide_flow_instance(n, 40 + n, symmetric=(n % 20 == 10))
    W, iters = 3, 250
    with q.Instance(F, D, force_int64=int64) as inst:
        assert inst.info["delta_bytes"] == (8 if int64 else 4)
        for k, (crit, lam) in enumerate(RULES):
            tn = (3, 3 + n // 10, 0) if crit == q.TABU_UNIT else (n // 10, n // 3, 0)
            descend = k == 1
            prm = q.make_params(W, seed=11 + k, iters=iters, tenure=tn, descend=descend,
                                criterion=crit, freq_penalty=lam, threads_per_walk=threads)
            pl = inst.plan(prm)
            assert (pl["threads_per_walk"], pl["pairs_per_thread"]) == (threads, slots)
            g = inst.search(prm, freq=True)
            o = oracle.run_walks(F, D, W, seed=11 + k, iters=iters, tenure=tn, descend=descend,
                                 criterion=crit, penalty=lam)
            for f in FIELDS:
                assert np.array_equal(g[f].astype(np.int64), o[f].astype(np.int64)), (f, crit)
            assert np.array_equal(g["best_p"], o["best_p"])
            if not descend:
                for w in range(W):
                    p0 = oracle.start_perm(11 + k, w, n)
                    *_, fq = oracle.tabu(F, D, p0, iters, *tn, True, 11 + k, w, want_freq=True,
                                         criterion=crit, penalty=lam)
                    assert np.array_equal(g["freq"][w], fq), (crit, w)
