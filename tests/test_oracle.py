"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: published
known-answer vectors, brute force over all permutations, cost differences
(Eq. 1) instead of the delta formula (Eq. 2), closed forms, invariances and
hand-computed cases.  None of them re-types the oracle's own formulas.
"""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_instance(rng, n, lo=-20, hi=20, diag=True):
    F = rng.integers(lo, hi + 1, size=(n, n)).astype(np.int64)
    D = rng.integers(lo, hi + 1, size=(n, n)).astype(np.int64)
    if not diag:
        np.fill_diagonal(F, 0)
        np.fill_diagonal(D, 0)
    return F, D


def swapped(p, r, s):
    q = np.array(p, copy=True)
    q[r], q[s] = q[s], q[r]
    return q


# ---------------------------------------------------------------------------
# Philox4x32-10 and the draws built on it
# ---------------------------------------------------------------------------

def load_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = load_kat()
    assert len(rows) >= 3
    for ctr, key, want in rows:
        got = orc.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_draw_layout(orc):
    # draw idx uses counter (walk, stream, idx // 4, 0) and output word idx % 4
    seed = (0x12345678 << 32) | 0x9abcdef0
    for walk, stream, idx in [(0, 0, 0), (7, 1, 5), (123, 0, 11), (2**31, 1, 2**20 + 3)]:
        blk = orc.philox4x32_10([walk, stream, idx >> 2, 0], [0x9abcdef0, 0x12345678])
        assert orc.draw(seed, walk, stream, idx) == int(blk[idx & 3])


def test_bounded_range(orc):
    for m in [1, 2, 3, 7, 100, 2**31 + 5]:
        assert orc.bounded(0, m) == 0
        assert orc.bounded(0xFFFFFFFF, m) == m - 1
        for x in [1, 12345, 2**31, 2**32 - 2]:
            assert 0 <= orc.bounded(x, m) < m
            assert orc.bounded(x, m) == (x * m) >> 32


def test_start_perm_is_uniform_permutation(orc):
    n = 4
    counts = {}
    trials = 4800
    for w in range(trials):
        p = orc.start_perm(99, w, n)
        assert sorted(p.tolist()) == list(range(n))
        counts[tuple(p.tolist())] = counts.get(tuple(p.tolist()), 0) + 1
    assert len(counts) == 24
    expect = trials / 24
    chi2 = sum((c - expect) ** 2 / expect for c in counts.values())
    assert chi2 < 60  # 23 dof; p ~ 1e-4 threshold
    assert orc.start_perm(5, 0, 1).tolist() == [0]


def test_start_perm_fisher_yates_steps(orc):
    # the first draw (index 0) picks which element lands in the last slot
    n = 9
    for w in range(50):
        p = orc.start_perm(3, w, n)
        j = orc.bounded(orc.draw(3, w, 0, 0), n)
        assert p[n - 1] == j


def test_tenure_rules(orc):
    tmin, tmax = 45, 55
    # period 100: constant within a period, redrawn at it = 1, 101, 201 ...
    vals = [orc.tenure(tmin, tmax, 100, 77, 3, it) for it in range(1, 401)]
    assert all(tmin <= v <= tmax for v in vals)
    for k in range(4):
        assert len(set(vals[100 * k:100 * (k + 1)])) == 1
    assert len(set(vals[::100])) > 1
    # period 0: one draw per move, draw index it - 1
    for it in range(1, 50):
        x = orc.draw(77, 3, 1, it - 1)
        assert orc.tenure(5, 16, 0, 77, 3, it) == 5 + orc.bounded(x, 12)


# ---------------------------------------------------------------------------
# Eq. 1: cost
# ---------------------------------------------------------------------------

def test_cost_hand_n2(orc):
    a, b, c, d = 3, 5, 7, 11
    F = np.array([[0, a], [b, 0]])
    D = np.array([[0, c], [d, 0]])
    assert orc.cost(F, D, [0, 1]) == a * c + b * d
    assert orc.cost(F, D, [1, 0]) == a * d + b * c


def test_cost_rank_one_closed_form(orc):
    # F = u v^T, D = x y^T  =>  cost = (sum_i u_i x_{p_i}) (sum_j v_j y_{p_j})
    rng = np.random.default_rng(1)
    for n in [1, 2, 5, 9, 17]:
        u, v, x, y = (rng.integers(-9, 10, size=n) for _ in range(4))
        F, D = np.outer(u, v), np.outer(x, y)
        for _ in range(5):
            p = rng.permutation(n)
            assert orc.cost(F, D, p) == int(np.dot(u, x[p])) * int(np.dot(v, y[p]))


def test_cost_constant_distance(orc):
    # D = c off the diagonal, 0 on it  =>  cost = c * sum_{i != j} F[i][j] for every p
    rng = np.random.default_rng(2)
    n, c = 8, 13
    F = rng.integers(0, 50, size=(n, n))
    D = np.full((n, n), c)
    np.fill_diagonal(D, 0)
    want = c * int(F.sum() - np.trace(F))
    for _ in range(10):
        assert orc.cost(F, D, rng.permutation(n)) == want
    assert orc.cost(np.zeros((n, n)), D, np.arange(n)) == 0


def test_cost_relabelling_invariance(orc):
    # F' = F[s][:, s], D' = D[t][:, t], p' = t^-1 o p o s  => cost' == cost
    rng = np.random.default_rng(3)
    for n in [3, 6, 11]:
        F, D = rand_instance(rng, n)
        p = rng.permutation(n)
        sg, tu = rng.permutation(n), rng.permutation(n)
        tinv = np.argsort(tu)
        F2, D2, p2 = F[sg][:, sg], D[tu][:, tu], tinv[p[sg]]
        assert orc.cost(F2, D2, p2) == orc.cost(F, D, p)


def test_cost_transpose_and_linearity(orc):
    rng = np.random.default_rng(4)
    n = 7
    F, D = rand_instance(rng, n)
    G, _ = rand_instance(rng, n)
    p = rng.permutation(n)
    assert orc.cost(F.T, D.T, p) == orc.cost(F, D, p)
    assert orc.cost(F + G, D, p) == orc.cost(F, D, p) + orc.cost(G, D, p)


def test_cost_overflow_detected(orc):
    big = np.full((2, 2), 2**40, dtype=np.int64)
    with pytest.raises(OverflowError):
        orc.cost(big, big, [0, 1])


# ---------------------------------------------------------------------------
# Eq. 2: the swap delta
# ---------------------------------------------------------------------------

def test_delta_equals_cost_difference_exhaustive(orc):
    # asymmetric, signed, non-zero diagonals: every pair of several perms
    rng = np.random.default_rng(5)
    for n in range(2, 9):
        F, D = rand_instance(rng, n)
        for _ in range(3):
            p = rng.permutation(n)
            c0 = orc.cost(F, D, p)
            for r in range(n):
                for s in range(r + 1, n):
                    assert orc.delta(F, D, p, r, s) == orc.cost(F, D, swapped(p, r, s)) - c0


def paper_eq2(F, D, pi, i, j):
    """Eq. 2 as printed (Section 4.1): exchange of the units at locations i
    and j of pi (pi[loc] = unit), no diagonal term."""
    f, d = F, D
    n = len(pi)
    val = (d[j][i] - d[i][j]) * (f[pi[i]][pi[j]] - f[pi[j]][pi[i]])
    for k in range(n):
        if k in (i, j):
            continue
        val += ((d[j][k] - d[i][k]) * (f[pi[i]][pi[k]] - f[pi[j]][pi[k]])
                + (d[k][j] - d[k][i]) * (f[pi[k]][pi[i]] - f[pi[k]][pi[j]]))
    return val


def test_delta_matches_printed_eq2_on_zero_diagonals(orc):
    # The paper's pi is the inverse of p; its location pair (p[r], p[s]) is
    # the unit pair (r, s) here.
    rng = np.random.default_rng(6)
    for n in [3, 5, 8, 12]:
        F, D = rand_instance(rng, n, diag=False)
        p = rng.permutation(n)
        pi = np.argsort(p)
        for r in range(n):
            for s in range(r + 1, n):
                i, j = sorted((p[r], p[s]))
                assert orc.delta(F, D, p, r, s) == paper_eq2(F, D, pi, i, j)


def test_printed_eq2_misses_diagonal_term(orc):
    # With non-constant diagonals the printed formula is not the cost change;
    # the oracle's extra term makes it exact (reading of Eq. 2).
    rng = np.random.default_rng(7)
    n = 6
    F, D = rand_instance(rng, n, diag=True)
    p = rng.permutation(n)
    pi = np.argsort(p)
    c0 = orc.cost(F, D, p)
    differs = 0
    for r in range(n):
        for s in range(r + 1, n):
            truth = orc.cost(F, D, swapped(p, r, s)) - c0
            i, j = sorted((p[r], p[s]))
            differs += paper_eq2(F, D, pi, i, j) != truth
            assert orc.delta(F, D, p, r, s) == truth
    assert differs > 0


def test_delta_symmetric_is_twice_one_side(orc):
    rng = np.random.default_rng(8)
    n = 9
    A = rng.integers(0, 30, size=(n, n)); F = A + A.T; np.fill_diagonal(F, 0)
    B = rng.integers(0, 30, size=(n, n)); D = B + B.T; np.fill_diagonal(D, 0)
    p = rng.permutation(n)
    P = D[p][:, p]
    for r in range(n):
        for s in range(r + 1, n):
            one = sum((F[r][k] - F[s][k]) * (P[s][k] - P[r][k]) for k in range(n) if k not in (r, s))
            assert orc.delta(F, D, p, r, s) == 2 * one


def test_delta_constant_distance_is_zero(orc):
    rng = np.random.default_rng(9)
    n = 7
    F = rng.integers(0, 50, size=(n, n))
    D = np.full((n, n), 4); np.fill_diagonal(D, 0)
    p = rng.permutation(n)
    assert all(orc.delta(F, D, p, r, s) == 0 for r in range(n) for s in range(r + 1, n))


# ---------------------------------------------------------------------------
# The O(1) delta update (ORC_CHECK compares the table with fresh Eq. 2 after
# every move and raises on any difference)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,diag,sym", [(2, False, False), (3, True, False), (7, True, False),
                                        (10, False, True), (16, True, True), (23, False, False)])
def test_fast_update_equals_fresh_eq2(orc, n, diag, sym):
    rng = np.random.default_rng(100 + n)
    F, D = rand_instance(rng, n, diag=diag)
    if sym:
        F, D = F + F.T, D + D.T
    p0 = rng.permutation(n)
    tn = (max(1, n // 3), max(1, n // 2), 0)
    orc.tabu(F, D, p0, 200, *tn, True, 11, 0, mode=orc.CHECK)
    orc.two_opt(F, D, p0, mode=orc.CHECK)


def test_fast_and_ref_modes_agree(orc):
    rng = np.random.default_rng(10)
    for n in [5, 9, 14]:
        F, D = rand_instance(rng, n)
        p0 = rng.permutation(n)
        a = orc.tabu(F, D, p0, 150, 2, 5, 0, True, 5, 1, mode=orc.REF)
        b = orc.tabu(F, D, p0, 150, 2, 5, 0, True, 5, 1, mode=orc.FAST)
        assert a[2]["hash"] == b[2]["hash"] and a[2]["best_cost"] == b[2]["best_cost"]
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])
        c = orc.two_opt(F, D, p0, mode=orc.REF)
        d = orc.two_opt(F, D, p0, mode=orc.FAST)
        assert np.array_equal(c[0], d[0]) and c[1] == d[1]


# ---------------------------------------------------------------------------
# 2opt (Section 4.1)
# ---------------------------------------------------------------------------

def replay_2opt(orc, F, D, p0, moves):
    """Re-derive each 2opt move by brute force on Eq. 1 cost differences."""
    n = len(p0)
    p = np.array(p0)
    for (r, s) in moves:
        c0 = orc.cost(F, D, p)
        cand = [(orc.cost(F, D, swapped(p, a, b)) - c0, a, b)
                for a in range(n) for b in range(a + 1, n)]
        best = min(cand)
        assert best[0] < 0 and (best[1], best[2]) == (r, s)
        p = swapped(p, r, s)
    return p


def test_2opt_moves_are_best_improvements_and_end_at_local_min(orc):
    rng = np.random.default_rng(11)
    for n in [4, 7, 10]:
        F, D = rand_instance(rng, n, lo=0, hi=30, diag=False)
        for _ in range(3):
            p0 = rng.permutation(n)
            p, res = orc.two_opt(F, D, p0, moves_cap=10000)
            assert len(res["moves"]) == res["iters_done"]
            p_end = replay_2opt(orc, F, D, p0, res["moves"])
            assert np.array_equal(p_end, p)
            assert res["best_cost"] == orc.cost(F, D, p)
            c = orc.cost(F, D, p)
            assert all(orc.cost(F, D, swapped(p, a, b)) >= c
                       for a in range(n) for b in range(a + 1, n))
            assert res["hash"] == orc.hash_moves(res["moves"])


def test_2opt_from_optimum_makes_no_move(orc):
    rng = np.random.default_rng(12)
    n = 7
    F, D = rand_instance(rng, n, lo=0, hi=40, diag=False)
    opt, popt = orc.brute_force(F, D)
    p, res = orc.two_opt(F, D, popt)
    assert res["iters_done"] == 0 and res["best_cost"] == opt


def test_2opt_max_iters_cap(orc):
    rng = np.random.default_rng(13)
    F, D = rand_instance(rng, 12, lo=0, hi=99, diag=False)
    p0 = rng.permutation(12)
    _, full = orc.two_opt(F, D, p0)
    assert full["iters_done"] >= 2
    _, capped = orc.two_opt(F, D, p0, max_iters=1)
    assert capped["iters_done"] == 1 and capped["best_cost"] > full["best_cost"]


# ---------------------------------------------------------------------------
# brute force and closed-form optima
# ---------------------------------------------------------------------------

def test_brute_force_path_on_line(orc):
    # F = path adjacency, D = |a - b|: optimum 2(n-1), reached at the identity
    for n in range(2, 9):
        F = np.zeros((n, n), dtype=np.int64)
        for i in range(n - 1):
            F[i][i + 1] = F[i + 1][i] = 1
        D = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
        opt, p = orc.brute_force(F, D)
        assert opt == 2 * (n - 1)
        assert orc.cost(F, D, np.arange(n)) == opt


def test_brute_force_matches_itertools(orc):
    rng = np.random.default_rng(14)
    n = 6
    F, D = rand_instance(rng, n)
    best = min(int((F * D[np.array(q)][:, np.array(q)]).sum())
               for q in itertools.permutations(range(n)))
    assert orc.brute_force(F, D)[0] == best


# ---------------------------------------------------------------------------
# Tabu search (Sections 4.3, 4.4)
# ---------------------------------------------------------------------------

def replay_tabu(orc, F, D, p0, moves, iters, tn, aspiration, seed, walk):
    """Brute-force replay of the tabu rules on Eq. 1 cost differences: each
    applied move must be the admissible move of lowest (delta, r, s)."""
    n = len(p0)
    p = np.array(p0)
    cur = orc.cost(F, D, p)
    best, best_iter = cur, 0
    tabu_until = {}
    for it in range(1, iters + 1):
        cand = []
        for a in range(n):
            for b in range(a + 1, n):
                dlt = orc.cost(F, D, swapped(p, a, b)) - cur
                ok = tabu_until.get((a, b), 0) <= it or (aspiration and cur + dlt < best)
                if ok:
                    cand.append((dlt, a, b))
        if not cand:
            assert len(moves) == it - 1
            return best, best_iter, 1
        dlt, a, b = min(cand)
        assert tuple(moves[it - 1]) == (a, b), f"iteration {it}"
        p = swapped(p, a, b)
        cur += dlt
        tabu_until[(a, b)] = it + orc.tenure(*tn, seed, walk, it)
        if cur < best:
            best, best_iter = cur, it
    assert len(moves) == iters
    return best, best_iter, 0


@pytest.mark.parametrize("n,iters,tn,asp", [(5, 40, (1, 3, 0), True), (7, 60, (2, 4, 14), True),
                                            (8, 50, (3, 6, 0), False), (4, 30, (1, 1, 0), True)])
def test_tabu_moves_follow_rules(orc, n, iters, tn, asp):
    rng = np.random.default_rng(15 + n)
    F, D = rand_instance(rng, n, lo=0, hi=25, diag=False)
    seed, walk = 21, 4
    p0 = orc.start_perm(seed, walk, n)
    p, best_p, res = orc.tabu(F, D, p0, iters, *tn, asp, seed, walk)
    best, best_iter, status = replay_tabu(orc, F, D, p0, res["moves"], iters, tn, asp, seed, walk)
    assert (res["best_cost"], res["best_iter"], res["status"]) == (best, best_iter, status)
    assert orc.cost(F, D, best_p) == best
    assert res["final_cost"] == orc.cost(F, D, p)
    assert res["hash"] == orc.hash_moves(res["moves"])


def test_tabu_best_not_below_optimum_and_often_reaches_it(orc):
    rng = np.random.default_rng(16)
    n = 8
    F, D = rand_instance(rng, n, lo=0, hi=99, diag=False)
    opt, _ = orc.brute_force(F, D)
    out = orc.run_walks(F, D, 16, seed=5, iters=200, tenure=(2, 4, 16), aspiration=True)
    assert (out["best_cost"] >= opt).all()
    assert (out["best_cost"] == opt).sum() >= 8
    for w in range(16):
        assert orc.cost(F, D, out["best_p"][w]) == out["best_cost"][w]


def test_tabu_stalls_when_every_move_is_tabu(orc):
    # n = 3 has 3 moves; with tenure 100 and no aspiration each applied move
    # stays tabu, so the walk stops at iteration 4 with 3 moves applied.
    rng = np.random.default_rng(17)
    F, D = rand_instance(rng, 3, lo=0, hi=9, diag=False)
    p, best_p, res = orc.tabu(F, D, [0, 1, 2], 10, 100, 100, 0, False, 1, 0)
    assert res["status"] == 1 and res["iters_done"] == 3
    assert sorted(map(tuple, res["moves"].tolist())) == [(0, 1), (0, 2), (1, 2)]


def test_tabu_zero_iterations(orc):
    rng = np.random.default_rng(18)
    F, D = rand_instance(rng, 6)
    p0 = rng.permutation(6)
    p, best_p, res = orc.tabu(F, D, p0, 0, 1, 2, 0, True, 1, 0)
    assert res["best_cost"] == orc.cost(F, D, p0) and res["best_iter"] == 0
    assert res["iters_done"] == 0 and np.array_equal(best_p, p0)


def test_frequency_memory_counts_exchanges(orc):
    rng = np.random.default_rng(19)
    n = 9
    F, D = rand_instance(rng, n, lo=0, hi=40, diag=False)
    p, best_p, res, freq = orc.tabu(F, D, rng.permutation(n), 120, 2, 4, 0, True, 3, 2,
                                    want_freq=True)
    assert np.triu(freq).sum() == 0
    assert freq.sum() == res["iters_done"]
    for (r, s) in res["moves"]:
        assert freq[s][r] > 0


def test_run_walks_matches_single_walks(orc):
    rng = np.random.default_rng(20)
    n = 10
    F, D = rand_instance(rng, n, lo=0, hi=50, diag=False)
    out = orc.run_walks(F, D, 6, seed=9, iters=80, tenure=(2, 5, 20), aspiration=True,
                        descend=True)
    for w in range(6):
        p0 = orc.start_perm(9, w, n)
        p1, r1 = orc.two_opt(F, D, p0)
        assert out["descent_moves"][w] == r1["iters_done"]
        _, bp, r2 = orc.tabu(F, D, p1, 80, 2, 5, 20, True, 9, w)
        assert out["best_cost"][w] == r2["best_cost"] and out["hash"][w] == r2["hash"]
        assert np.array_equal(out["best_p"][w], bp)


# ---------------------------------------------------------------------------
# Other tabu criteria (Taillard's unit-location rule, Zhu et al.'s unit
# marking, Section 3.1) and the frequency penalty (Section 7's long-term
# memory).  Replayed by brute force on Eq. 1 differences with bookkeeping of
# their own, and pinned by hand-derived trajectories on instances whose
# every delta is zero (constant off-diagonal distances).
# ---------------------------------------------------------------------------

def replay_rules(orc, F, D, p0, moves, iters, tn, aspiration, seed, walk, criterion, penalty):
    n = len(p0)
    p = np.array(p0)
    cur = orc.cost(F, D, p)
    best = cur
    pair_until, barred, marked, count = {}, {}, {}, {}
    for it in range(1, iters + 1):
        cand = []
        for a in range(n):
            for b in range(a + 1, n):
                dlt = orc.cost(F, D, swapped(p, a, b)) - cur
                if criterion == orc.TABU_PAIR:
                    forbidden = pair_until.get((a, b), 0) > it
                elif criterion == orc.TABU_UNIT_LOC:
                    # a would move to b's location and b to a's
                    forbidden = (barred.get((a, p[b]), 0) > it and barred.get((b, p[a]), 0) > it)
                else:
                    forbidden = marked.get(a, 0) > it or marked.get(b, 0) > it
                if forbidden and not (aspiration and cur + dlt < best):
                    continue
                rank = dlt + penalty * count.get((a, b), 0) if dlt >= 0 else dlt
                cand.append((rank, a, b, dlt))
        if not cand:
            assert len(moves) == it - 1
            return best, 1
        _, a, b, dlt = min(cand)
        assert tuple(moves[it - 1]) == (a, b), f"iteration {it}"
        until = it + orc.tenure(*tn, seed, walk, it)
        pair_until[(a, b)] = until
        barred[(a, p[a])] = until
        barred[(b, p[b])] = until
        marked[a] = marked[b] = until
        count[(a, b)] = count.get((a, b), 0) + 1
        p = swapped(p, a, b)
        cur += dlt
        best = min(best, cur)
    assert len(moves) == iters
    return best, 0


@pytest.mark.parametrize("criterion", [1, 2])
@pytest.mark.parametrize("penalty,asp,tn", [(0, True, (1, 3, 0)), (0, False, (2, 2, 5)),
                                            (4, True, (1, 2, 0)), (50, False, (1, 3, 4))])
def test_rules_moves_follow_definitions(orc, criterion, penalty, asp, tn):
    rng = np.random.default_rng(30 + 7 * criterion + penalty)
    n, iters = 7, 50
    F, D = rand_instance(rng, n, lo=0, hi=12, diag=False)
    seed, walk = 8, 3
    p0 = orc.start_perm(seed, walk, n)
    p, best_p, res, freq = orc.tabu(F, D, p0, iters, *tn, asp, seed, walk, want_freq=True,
                                    criterion=criterion, penalty=penalty)
    best, status = replay_rules(orc, F, D, p0, res["moves"], iters, tn, asp, seed, walk,
                                criterion, penalty)
    assert (res["best_cost"], res["status"]) == (best, status)
    assert res["final_cost"] == orc.cost(F, D, p) and orc.cost(F, D, best_p) == best
    assert freq.sum() == res["iters_done"]


def test_penalty_moves_follow_definition_pair_criterion(orc):
    rng = np.random.default_rng(41)
    n, iters, tn = 6, 80, (1, 2, 0)
    F, D = rand_instance(rng, n, lo=-5, hi=9)
    p0 = orc.start_perm(2, 0, n)
    _, _, res = orc.tabu(F, D, p0, iters, *tn, True, 2, 0, penalty=7)
    best, status = replay_rules(orc, F, D, p0, res["moves"], iters, tn, True, 2, 0, 0, 7)
    assert (res["best_cost"], res["status"]) == (best, status)


def constant_distance_instance(rng, n, c=7):
    """Every permutation costs c * sum of off-diagonal F: every delta is 0."""
    F, _ = rand_instance(rng, n, lo=0, hi=9, diag=False)
    D = np.full((n, n), c, dtype=np.int64)
    np.fill_diagonal(D, 0)
    return F, D


def test_unit_marking_stops_after_disjoint_pairs(orc):
    # Every delta is 0, so the lowest free pair is taken.  With a long
    # tenure each move marks two fresh units: (0,1), (2,3), (4,5), then only
    # unit 6 is free and no move is allowed.
    F, D = constant_distance_instance(np.random.default_rng(42), 7)
    _, _, res = orc.tabu(F, D, np.arange(7), 20, 100, 100, 0, False, 1, 0,
                         criterion=orc.TABU_UNIT)
    assert res["moves"].tolist() == [[0, 1], [2, 3], [4, 5]]
    assert res["status"] == 1 and res["iters_done"] == 3


def test_unit_marking_tenure_two_alternates(orc):
    # A mark set at it lasts through it + 1, so (0,1) and (2,3) alternate.
    F, D = constant_distance_instance(np.random.default_rng(43), 6)
    _, _, res = orc.tabu(F, D, np.arange(6), 8, 2, 2, 0, False, 1, 0, criterion=orc.TABU_UNIT)
    assert res["moves"].tolist() == [[0, 1], [2, 3]] * 4 and res["status"] == 0


def test_unit_location_hand_trajectory(orc):
    # n = 3, identity start, every delta 0, long tenure, no aspiration.
    # it 1: (0,1); units 0, 1 barred from locations 0, 1.  it 2: (0,1) would
    # return both, (0,2) sends unit 0 to location 2: taken.  it 3: (0,1)
    # sends unit 1 to location 2, never left: taken.  it 4: (0,1) returns
    # both, (0,2) sends unit 2 to location 0: taken.  it 5: every move
    # returns both of its units: the walk stops.
    F, D = constant_distance_instance(np.random.default_rng(44), 3)
    _, _, res = orc.tabu(F, D, np.arange(3), 10, 100, 100, 0, False, 1, 0,
                         criterion=orc.TABU_UNIT_LOC)
    assert res["moves"].tolist() == [[0, 1], [0, 2], [0, 1], [0, 2]]
    assert res["status"] == 1


def test_frequency_penalty_round_robin(orc):
    # Every delta is 0 and a tenure of 1 forbids nothing, so with the
    # penalty the least-applied pair is taken, lowest first: a round robin
    # over the 6 pairs of n = 4 in lexicographic order.
    F, D = constant_distance_instance(np.random.default_rng(45), 4)
    pairs = [[a, b] for a in range(4) for b in range(a + 1, 4)]
    _, _, res, freq = orc.tabu(F, D, np.arange(4), 14, 1, 1, 0, True, 1, 0, want_freq=True,
                               penalty=1)
    assert res["moves"].tolist() == [pairs[k % 6] for k in range(14)]
    assert sorted(freq[np.tril_indices(4, -1)].tolist()) == [2, 2, 2, 2, 3, 3]
    # without the penalty the same search repeats the lowest pair
    _, _, res0 = orc.tabu(F, D, np.arange(4), 14, 1, 1, 0, True, 1, 0)
    assert res0["moves"].tolist() == [[0, 1]] * 14


def test_penalty_leaves_improving_moves_alone(orc):
    # Improving moves are ranked by their delta alone, so a heavy penalty
    # follows the unpenalised search for as long as that one improves.
    rng = np.random.default_rng(46)
    n = 12
    F, D = rand_instance(rng, n, lo=0, hi=50, diag=False)
    p0 = orc.start_perm(4, 1, n)
    _, _, plain = orc.tabu(F, D, p0, 60, 3, 5, 0, True, 4, 1)
    _, _, heavy = orc.tabu(F, D, p0, 60, 3, 5, 0, True, 4, 1, penalty=10**6)
    costs, p, k = [], np.array(p0), 0
    for (a, b) in plain["moves"]:
        q = swapped(p, a, b)
        if orc.cost(F, D, q) >= orc.cost(F, D, p):
            break
        p, k = q, k + 1
    assert k >= 3
    assert np.array_equal(heavy["moves"][:k], plain["moves"][:k])
    assert not np.array_equal(heavy["moves"], plain["moves"])


def test_rules_reject_bad_arguments(orc):
    F, D = constant_distance_instance(np.random.default_rng(47), 4)
    with pytest.raises(ValueError):
        orc.tabu(F, D, np.arange(4), 5, 1, 1, 0, True, 1, 0, criterion=3)
    with pytest.raises(ValueError):
        orc.tabu(F, D, np.arange(4), 5, 1, 1, 0, True, 1, 0, penalty=-1)


# ---------------------------------------------------------------------------
# stored oracle outputs (written by tests/golden/make_golden.py)
# ---------------------------------------------------------------------------

def test_golden_sym12_2opt(orc):
    from paper_2307_11248_gb300 import instances
    import json
    with open(os.path.join(GOLDEN, "sym12_2opt.json")) as f:
        g = json.load(f)
    w = instances.workload_sym12()
    assert int(w["F"].sum()) == g["F_sum"] and int(w["D"].sum()) == g["D_sum"]
    out = orc.run_walks(w["F"], w["D"], w["walks"], seed=w["seed"], descend=True)
    assert out["best_cost"].tolist() == g["best_cost"]
    assert out["descent_moves"].tolist() == g["moves"]
    assert [int(h) for h in out["descent_hash"]] == g["hash"]
    sub_opt, _ = orc.brute_force(w["F"][:9, :9], w["D"][:9, :9])
    assert sub_opt == g["sub9_optimum"]
