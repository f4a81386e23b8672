"""The algebra of the products form of phase X, checked in plain numpy on
random instances (no GPU, no library code).

For a permutation p of n units over n locations, Q = D[p][p] and

    M[x][k] = sum_j F[x][j] Q[k][j] + F[j][x] Q[j][k]

(the dot products Eq. 2 needs for the pairs touching a move).  The walk keeps
Q as the starting matrix Q0 and a label sigma[k] per location (the row of Q0
location k holds, so Q[i][j] = Q0[sigma[i]][sigma[j]]), and M with its
columns indexed by label, Mt[x][sigma[k]] = M[x][k].  Exchanging locations
r and s then changes Mt by one rank-2 update and moves no column:

    Mt'[x][u] = Mt[x][u] - a_x b_j - c_x e_j,   j the location of label u

with a_x = F[r][x] - F[s][x], c_x = F[x][r] - F[x][s], b_j = Q[r][j] -
Q[s][j], e_j = Q[j][r] - Q[j][s] (the move's update vectors, before it).
These tests check that identity and its bookkeeping over a sequence of
moves, and how a pair's delta follows from M."""
import numpy as np
import pytest


def products(F, Q):
    return F @ Q.T + F.T @ Q


def delta(F, Q, r, s):
    """Cost difference of exchanging locations r and s (Eq. 1 before and
    after, by brute force)."""
    Q2 = Q.copy()
    Q2[[r, s], :] = Q2[[s, r], :]
    Q2[:, [r, s]] = Q2[:, [s, r]]
    return int((F * Q2).sum() - (F * Q).sum())


@pytest.mark.parametrize("n,seed,sym", [(7, 1, False), (12, 2, False), (12, 3, True),
                                        (30, 4, False)])
def test_label_indexed_rank2_update(n, seed, sym):
    rng = np.random.default_rng(seed)
    F = rng.integers(-50, 51, (n, n)).astype(np.int64)
    D = rng.integers(-9, 10, (n, n)).astype(np.int64)
    if sym:
        F = np.triu(F) + np.triu(F, 1).T
        D = np.triu(D) + np.triu(D, 1).T
    p = rng.permutation(n)
    Q0 = D[np.ix_(p, p)]
    sigma = np.arange(n)
    Mt = products(F, Q0)  # sigma is the identity: Mt = M
    for _ in range(40):
        r, s = sorted(rng.choice(n, 2, replace=False))
        Q = Q0[np.ix_(sigma, sigma)]
        # before the move: Mt read through the labels is M
        assert np.array_equal(Mt[:, sigma], products(F, Q))
        a = F[r, :] - F[s, :]
        c = F[:, r] - F[:, s]
        b = Q[r, :] - Q[s, :]
        e = Q[:, r] - Q[:, s]
        loc = np.empty(n, dtype=np.int64)
        loc[sigma] = np.arange(n)  # location of each label before the move
        Mt = Mt - np.outer(a, b[loc]) - np.outer(c, e[loc])
        sigma[[r, s]] = sigma[[s, r]]
    Q = Q0[np.ix_(sigma, sigma)]
    assert np.array_equal(Mt[:, sigma], products(F, Q))


def test_a_pair_delta_from_the_products():
    """The swap delta of any pair {u, v} from M alone plus the pair's own
    entries: the dot-product sums of Eq. 2 over all j are
    M[u][v] + M[v][u] - M[u][u] - M[v][v]; removing their j = u, v terms and
    adding the exact change of the 2 x 2 block at rows and columns u, v gives
    the brute-force cost difference."""
    rng = np.random.default_rng(9)
    n = 11
    F = rng.integers(0, 20, (n, n)).astype(np.int64)
    Q = rng.integers(0, 20, (n, n)).astype(np.int64)
    M = products(F, Q)
    for u in range(n):
        for v in range(u + 1, n):
            full = M[u, v] + M[v, u] - M[u, u] - M[v, v]
            own = sum((F[u, j] - F[v, j]) * (Q[v, j] - Q[u, j]) +
                      (F[j, u] - F[j, v]) * (Q[j, v] - Q[j, u]) for j in (u, v))
            uv = np.ix_([u, v], [u, v])
            block = int((F[uv] * Q[np.ix_([v, u], [v, u])]).sum() - (F[uv] * Q[uv]).sum())
            assert delta(F, Q, u, v) == full - own + block, (u, v)
