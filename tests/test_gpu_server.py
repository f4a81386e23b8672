"""The serving loop: requests of different n admitted by slots and device
memory, running on the device together.  Each request's results must be
those of the same search run alone (qap_search) and of the oracle."""
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


def request_params(n, rid, iters=120, walks=8):
    return q.make_params(walks, seed=rid, iters=iters, tenure=instances.periodic_tenure(n))


def alone(F, D, prm):
    with q.Instance(F, D) as inst:
        return inst.search(prm)


def same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in FIELDS)


def test_requests_equal_oracle_and_alone():
    reqs = instances.poisson_requests(6, seed=42, nmin=12, nmax=256)
    with q.Server(slots=4, mem_bytes=256 << 20) as sv:
        tickets = [(r, sv.submit(r.inst.F, r.inst.D, request_params(r.inst.n, r.rid)))
                   for r in reqs]
        for r, t in tickets:
            res, times = sv.wait(t)
            n = r.inst.n
            prm = request_params(n, r.rid)
            assert same(res, alone(r.inst.F, r.inst.D, prm)), (r.rid, n)
            o = oracle.run_walks(r.inst.F, r.inst.D, prm.starts, seed=r.rid, iters=prm.iters,
                                 tenure=instances.periodic_tenure(n))
            for k in FIELDS:
                assert np.array_equal(res[k].astype(np.int64), o[k].astype(np.int64)), (r.rid, k)
            assert times["total_us"] >= times["device_us"] > 0


def overlaps(a, b):
    """Kernel intervals (device clock) of two requests share some time."""
    return a["kernel_start_us"] < b["kernel_end_us"] and b["kernel_start_us"] < a["kernel_end_us"]


def test_result_is_the_same_alone_and_in_the_mix():
    """One request served alone, then the same request among 40 others that
    were admitted before and after it: identical results, and the request's
    kernel ran on the device at the same time as another request's."""
    probe = instances.poisson_requests(1, seed=7, nmin=60, nmax=60)[0]
    prm = request_params(probe.inst.n, 999, iters=300, walks=16)
    mix = instances.poisson_requests(40, seed=8, nmin=12, nmax=200)
    with q.Server(slots=16, mem_bytes=512 << 20) as sv:
        t0 = sv.submit(probe.inst.F, probe.inst.D, prm)
        solo, solo_t = sv.wait(t0)
        tickets = []
        for k, r in enumerate(mix):
            tickets.append(sv.submit(r.inst.F, r.inst.D, request_params(r.inst.n, r.rid)))
            if k == 20:
                t_mid = sv.submit(probe.inst.F, probe.inst.D, prm)
        in_mix, mid_t = sv.wait(t_mid)
        others = [sv.wait(t)[1] for t in tickets]
        stats = sv.stats()
    assert stats["submitted"] == 42 and stats["completed"] == 42
    assert same(solo, in_mix)
    # the device clock orders each request's kernel interval
    for t in [solo_t, mid_t] + others:
        assert 0 <= t["kernel_start_us"] < t["kernel_end_us"]
    assert any(overlaps(mid_t, t) for t in others), "the probe ran alone on the device"
    assert stats["peak_in_flight"] >= 2
    # more than one request's kernel at once, at some moment of the mix
    ev = sorted([(t["kernel_start_us"], 1) for t in others] +
                [(t["kernel_end_us"], -1) for t in others])
    depth = peak = 0
    for _, d in ev:
        depth += d
        peak = max(peak, depth)
    assert peak >= 2


def test_admission_by_memory_budget():
    """An arena that holds only a few requests at a time still serves every
    request, in arrival order, with correct results."""
    reqs = instances.poisson_requests(12, seed=3, nmin=150, nmax=250)
    with q.Server(slots=12, mem_bytes=24 << 20) as sv:
        tickets = [sv.submit(r.inst.F, r.inst.D, request_params(r.inst.n, r.rid, iters=40))
                   for r in reqs]
        for _ in range(50):
            st = sv.stats()
            assert st["arena_used"] <= st["arena_bytes"]
        for r, t in zip(reqs, tickets):
            res, _ = sv.wait(t)
            assert same(res, alone(r.inst.F, r.inst.D, request_params(r.inst.n, r.rid, iters=40)))
        st = sv.stats()
        assert st["completed"] == 12
        # the arena holds a few of these requests at a time, not all twelve
        assert 2 <= st["peak_in_flight"] < 12


def test_wait_is_bounded_and_tickets_are_checked():
    F, D = instances.uniform_instance(120, 1, symmetric=False)
    prm = q.make_params(32, seed=1, iters=100000, tenure=(100, 130, 240))
    with q.Server(slots=2, mem_bytes=64 << 20) as sv:
        t = sv.submit(F, D, prm)
        with pytest.raises(q.QapError) as e:
            sv.wait(t, timeout_ms=0)
        assert e.value.status == q.ETIMEOUT
        res, _ = sv.wait(t, timeout_ms=600000)  # the ticket is still valid
        assert (res["iters_done"] == 100000).all()
        with pytest.raises(q.QapError) as e:
            q.qap_server_wait(sv.h, 12345, 120, 32, 0)
        assert e.value.status == q.EINVAL


def test_submit_rejects_requests_that_cannot_fit():
    F, D = instances.uniform_instance(256, 2, symmetric=False)
    with q.Server(slots=1, mem_bytes=2 << 20) as sv:
        with pytest.raises(q.QapError) as e:
            sv.submit(F, D, q.make_params(32, seed=1, iters=10, tenure=(1, 2, 0)))
        assert e.value.status == q.ENOMEM
