"""Seeded random configurations across plan boundaries: n from 2 to 256,
symmetric or not, signed or unsigned values (int8 / int16 flows, int32 /
int64 deltas), 2opt descent or not, every tabu criterion, with and without
the frequency penalty.  Every walk must equal the oracle's, bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2307_11248_gb300 as q

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


def case(k):
    rng = np.random.default_rng(5000 + k)
    n = int(rng.choice([2, 3, 4, 7, 12, 16, 17, 31, 33, 48, 64, 65, 90, 101, 127, 150, 181,
                        182, 200, 256]))
    sym = bool(rng.integers(2))
    kind = int(rng.integers(3))
    if kind == 0:      # byte range: int8 flows
        lo, hi, dlo, dhi = 0, 99, 0, 99
    elif kind == 1:    # signed bytes with a wide range: int16 flows, int32 deltas
        lo, hi, dlo, dhi = -120, 120, -60, 60
    else:              # large flows: int16 flows, int64 deltas
        lo, hi, dlo, dhi = 0, 20000, 0, 100
    F = rng.integers(lo, hi + 1, size=(n, n)).astype(np.int64)
    D = rng.integers(dlo, dhi + 1, size=(n, n)).astype(np.int64)
    if sym:
        F = np.triu(F) + np.triu(F, 1).T
        D = np.triu(D) + np.triu(D, 1).T
    if rng.integers(2):
        np.fill_diagonal(F, 0)
        np.fill_diagonal(D, 0)
    crit = int(rng.integers(3))
    lam = int(rng.choice([0, 0, 2, 17]))
    descend = bool(rng.integers(2))
    tmin = int(rng.integers(1, max(2, n // 3) + 1))
    tn = (tmin, tmin + int(rng.integers(0, 5)), int(rng.choice([0, 0, 7, 2 * n])))
    iters = int(rng.integers(20, 120))
    asp = bool(rng.integers(4) > 0)
    return n, F, D, crit, lam, descend, tn, iters, asp


@pytest.mark.parametrize("k", range(28))
def test_random_configurations_bit_exact(k):
    n, F, D, crit, lam, descend, tn, iters, asp = case(k)
    W = 3
    prm = q.make_params(W, seed=90 + k, iters=iters, tenure=tn, aspiration=asp, descend=descend,
                        criterion=crit, freq_penalty=lam)
    try:
        inst = q.Instance(F, D)
    except q.QapError as e:  # values outside the supported ranges are refused up front
        assert e.status == q.EUNSUPPORTED
        return
    with inst:
        try:
            g = inst.search(prm)
        except q.QapError as e:  # a penalty that int32 deltas cannot hold
            assert e.status == q.EOVERFLOW and lam > 0
            return
    o = oracle.run_walks(F, D, W, seed=90 + k, iters=iters, tenure=tn, aspiration=asp,
                         descend=descend, criterion=crit, penalty=lam)
    for f in FIELDS:
        assert np.array_equal(g[f].astype(np.int64), o[f].astype(np.int64)), (k, f)
