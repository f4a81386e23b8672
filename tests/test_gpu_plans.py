"""GPU parity at the launch shapes that full-size launches take.

A launch with walks enough for two CTAs on every SM (at least 2 x SMs walks)
lets the automatic plan take 256 threads per walk with 8, 12, 16 or 24 pair
slots per thread, two walks per SM.  Those plans are what the n = 100 grid
workload (1024 walks x (2opt + 10^4 tabu iterations), Sections 4.1-4.4) and
every many-walk launch of n = 54..100 run.  Here each of them is reached by
the automatic choice itself, the plan is asserted, and sampled walks of the
launch are compared with the CPU oracle bit for bit: best permutation, best
and final cost, best iteration, iteration count, status, 2opt move count and
both trajectory hashes.
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


def sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def check_rows(g, F, D, rows, **kw):
    o = oracle.run_walks(F, D, len(rows), walk_ids=np.asarray(rows), **kw)
    for k in FIELDS:
        a = g[k][rows].astype(np.int64)
        b = o[k].astype(np.int64)
        assert np.array_equal(a, b), (k, rows)


def test_grid100_full_launch_on_its_own_plan():
    """The whole n = 100 grid workload in the launch its benchmark times
    (1024 walks, 2opt to a local minimum, then 10^4 tabu iterations): the
    automatic plan is 256 threads x 24 slots, two CTAs per SM, with phase X
    from the maintained products; sampled walks equal the oracle's."""
    w = instances.workload_grid100()
    W = w["walks"]
    assert W >= 2 * sms()
    with q.Instance(w["F"], w["D"]) as inst:
        prm = q.make_params(W, seed=w["seed"], iters=w["iters"], tenure=w["tenure"],
                            descend=True)
        plan = inst.plan(prm)
        assert (plan["threads_per_walk"], plan["pairs_per_thread"]) == (256, 24), plan
        assert plan["ctas_per_sm"] == 2 and plan["products"] == 1, plan
        g = inst.search(prm)
    assert (g["iters_done"] == w["iters"]).all()
    check_rows(g, w["F"], w["D"], [0, 1, 511, 700, 1022, 1023], seed=w["seed"],
               iters=w["iters"], tenure=w["tenure"], descend=True)
    # every walk: its best permutation's Eq. 1 cost is its best cost
    with q.Instance(w["F"], w["D"]) as inst:
        assert np.array_equal(inst.cost(g["best_p"]), g["best_cost"])


# (n, symmetric, expected slots): every int8 plan with 256 threads that a
# many-walk launch selects, on symmetric and asymmetric instances, each with
# phase X from the maintained products (the automatic form) and by dot
# products (asked for)
PLANS_256 = [(50, False, 6), (52, True, 6), (58, False, 8), (60, True, 8),
             (70, False, 12), (66, True, 12), (80, False, 16), (78, True, 16),
             (96, False, 24), (90, True, 24)]


@pytest.mark.parametrize("phase_x", [q.PHASE_X_AUTO, q.PHASE_X_DOTS])
@pytest.mark.parametrize("n,sym,slots", PLANS_256)
def test_many_walk_plans_int8(n, sym, slots, phase_x):
    W = 2 * sms()
    F, D = instances.uniform_instance(n, 600 + n, symmetric=sym)
    tn = instances.periodic_tenure(n)
    iters = 400
    products = int(phase_x == q.PHASE_X_AUTO)
    with q.Instance(F, D) as inst:
        assert inst.info["delta_bytes"] == 4
        prm = q.make_params(W, seed=31, iters=iters, tenure=tn, descend=True, phase_x=phase_x)
        plan = inst.plan(prm)
        assert plan["threads_per_walk"] == 256 and plan["pairs_per_thread"] == slots, plan
        assert plan["products"] == products and plan["ctas_per_sm"] >= 2, plan
        g = inst.search(prm)
    check_rows(g, F, D, [0, 5, W // 2 + 1, W - 1], seed=31, iters=iters, tenure=tn,
               descend=True)


@pytest.mark.parametrize("phase_x", [q.PHASE_X_AUTO, q.PHASE_X_DOTS])
# (n, symmetric, slots, int64 deltas, products form in the automatic choice):
# at n = 96 asymmetric M fits beside two walks per SM only without the
# transposed copies of F and P (form 2)
@pytest.mark.parametrize("n,sym,slots,int64,prod", [
    (58, False, 8, False, 1), (70, False, 12, False, 1), (80, True, 16, False, 1),
    (92, True, 24, False, 1), (96, False, 24, False, 2), (52, True, 6, True, 1),
    (66, False, 12, True, 1), (90, True, 24, True, 1)])
def test_many_walk_plans_int16_flows(n, sym, slots, int64, prod, phase_x):
    """Flows beyond a byte take the int16 element path (interleaved slots),
    with int32 or int64 deltas, phase X from the maintained products (the
    automatic form, when they fit shared memory) or by dot products."""
    W = 2 * sms()
    F, D = instances.uniform_instance(n, 700 + n, symmetric=sym, hi=99)
    F = F * 20  # up to 1980: int16 flows, still int32 deltas
    tn = instances.periodic_tenure(n)
    with q.Instance(F, D, force_int64=int64) as inst:
        assert inst.info["delta_bytes"] == (8 if int64 else 4)
        assert inst.info["flow_bytes"] == 2
        prm = q.make_params(W, seed=32, iters=300, tenure=tn, phase_x=phase_x)
        plan = inst.plan(prm)
        assert plan["threads_per_walk"] == 256 and plan["pairs_per_thread"] == slots, plan
        assert plan["products"] == (prod if phase_x == q.PHASE_X_AUTO else 0), plan
        g = inst.search(prm)
    check_rows(g, F, D, [1, W // 3, W - 2], seed=32, iters=300, tenure=tn)


@pytest.mark.parametrize("n,slots", [(58, 8), (70, 12), (80, 16)])
def test_fewer_walks_same_plan_by_request(n, slots):
    """The same 256-thread plans asked for explicitly with a few walks (one
    per SM at most): the launch shape does not change the walks."""
    F, D = instances.uniform_instance(n, 800 + n, symmetric=False)
    tn = instances.periodic_tenure(n)
    with q.Instance(F, D) as inst:
        prm = q.make_params(5, seed=33, iters=500, tenure=tn, threads_per_walk=256)
        plan = inst.plan(prm)
        assert plan["pairs_per_thread"] == slots, plan
        g = inst.search(prm)
    check_rows(g, F, D, list(range(5)), seed=33, iters=500, tenure=tn)


@pytest.mark.parametrize("n,sym,scale,int64", [(150, False, 1, False), (148, True, 1, False),
                                               (151, False, 90, True), (147, True, 90, True)])
def test_512x26_plan(n, sym, scale, int64):
    """n = 147-151 on 512 threads takes 26 slots per thread (the largest batch
    class's plan, in place of 1024 threads at 64 registers), with int8 or
    int16 flows and int32 or int64 deltas."""
    F, D = instances.uniform_instance(n, 990 + n, symmetric=sym)
    F = F * scale
    tn = instances.periodic_tenure(n)
    with q.Instance(F, D, force_int64=int64) as inst:
        prm = q.make_params(3, seed=34, iters=300, tenure=tn, descend=True,
                            threads_per_walk=512)
        plan = inst.plan(prm)
        assert (plan["threads_per_walk"], plan["pairs_per_thread"]) == (512, 26), plan
        g = inst.search(prm)
    check_rows(g, F, D, [0, 1, 2], seed=34, iters=300, tenure=tn, descend=True)


@pytest.mark.parametrize("phase_x", [q.PHASE_X_AUTO, q.PHASE_X_DOTS])
@pytest.mark.parametrize("n,sym,slots", [(104, False, 12), (110, True, 16), (127, False, 20),
                                         (131, True, 20), (139, False, 24), (144, True, 24)])
def test_512_thread_plans_int8(n, sym, slots, phase_x):
    """The 512-thread int8 plans of n = 101-146 (one walk per SM), with phase
    X from the maintained products (the automatic form, up to 24 slots) and
    by dot products: sampled walks equal the oracle's."""
    F, D = instances.uniform_instance(n, 1100 + n, symmetric=sym)
    tn = instances.periodic_tenure(n)
    with q.Instance(F, D) as inst:
        assert inst.info["delta_bytes"] == 4
        prm = q.make_params(4, seed=35, iters=300, tenure=tn, descend=True,
                            threads_per_walk=512, phase_x=phase_x)
        plan = inst.plan(prm)
        assert (plan["threads_per_walk"], plan["pairs_per_thread"]) == (512, slots), plan
        assert plan["products"] == int(phase_x == q.PHASE_X_AUTO), plan
        g = inst.search(prm)
    check_rows(g, F, D, [0, 1, 2, 3], seed=35, iters=300, tenure=tn, descend=True)


@pytest.mark.parametrize("n,fscale,int64", [(140, 20, True), (146, 1, False), (146, 20, False)])
def test_products_without_transposed_copies(n, fscale, int64):
    """Large asymmetric instances whose M fits shared memory only without the
    transposed copies of F and P (products form 2: their entries read from
    columns) on 512 x 24, int8 or int16 flows, int32 or int64 deltas: sampled
    walks equal the oracle's."""
    F, D = instances.uniform_instance(n, 1200 + n, symmetric=False)
    F = F * fscale
    tn = instances.periodic_tenure(n)
    with q.Instance(F, D, force_int64=int64) as inst:
        assert inst.info["flow_bytes"] == (2 if fscale > 1 or int64 else 1)
        prm = q.make_params(3, seed=36, iters=300, tenure=tn, descend=True,
                            threads_per_walk=512)
        plan = inst.plan(prm)
        assert (plan["threads_per_walk"], plan["pairs_per_thread"]) == (512, 24), plan
        assert plan["products"] == 2, plan
        g = inst.search(prm)
    check_rows(g, F, D, [0, 1, 2], seed=36, iters=300, tenure=tn, descend=True)


@pytest.mark.parametrize("n,sym,int64", [(60, False, False), (90, True, True), (130, False, True)])
def test_products_int16_flows_with_wide_differences(n, sym, int64):
    """int16 flows spanning more than 2^15 (differences of two entries need
    17 bits): the products form updates M by int32 multiply-adds instead of
    dp2a; sampled walks equal the oracle's."""
    F, D = instances.uniform_instance(n, 1300 + n, symmetric=sym, lo=-20000, hi=20000)
    _, D = instances.uniform_instance(n, 1400 + n, symmetric=sym)
    np.fill_diagonal(F, 0)
    tn = instances.periodic_tenure(n)
    W = 2 * sms() if n <= 100 else 4
    with q.Instance(F, D, force_int64=int64) as inst:
        assert inst.info["flow_bytes"] == 2
        prm = q.make_params(W, seed=37, iters=300, tenure=tn, descend=True)
        assert inst.plan(prm)["products"] in (1, 2)
        g = inst.search(prm)
    check_rows(g, F, D, [0, 1, W - 1], seed=37, iters=300, tenure=tn, descend=True)
