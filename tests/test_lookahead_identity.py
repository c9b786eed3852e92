"""The walk-count identity behind the lookahead sweep's derived levels, pinned by enumeration.

A lookahead run guesses the next winners c_1..c_D and keeps, per vertex v and length i, the
walks ending at v that avoid S (phi^miss under S) and, for each guess c_j, the walks ending at v
that avoid T_{j-1} = S + {c_1..c_{j-1}} and visit c_j. A walk that avoids S either avoids all of
c_1..c_d or has a first guess c_j among them, so

    phi^miss_i(T_d)(v) = phi^miss_i(S)(v) - sum_{j <= d} z_{j,i}(v),

and z_j obeys the masked recurrence z_{j,i}(v) = [v not in T_{j-1}] sum_{u ~ v} z_{j,i-1}(u),
except at v = c_j, where every walk ending there visits c_j: z_{j,i}(c_j) = phi^miss_i(T_{j-1})(c_j).
The sweep epilogue computes the levels' phi^miss vectors, and c_j's own-row values, as these
differences. Here every term is counted by enumerating all walks of tiny graphs, and the
recurrences (unscaled integer counts, as with alpha = 1) are checked against those counts.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg


def _adj(g):
    A = np.zeros((g.n, g.n), dtype=np.int64)
    for v in range(g.n):
        A[v, g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]] = 1
    return A


def _walks(A, i):
    n = A.shape[0]
    for w in itertools.product(range(n), repeat=i + 1):
        if all(A[w[t], w[t + 1]] for t in range(i)):
            yield w


def _enumerated(A, S, cand, i):
    """phi^miss_i(T_d)(v) for d = 0..D and z_{j,i}(v) for j = 1..D, counted walk by walk."""
    n, D = A.shape[0], len(cand)
    miss = np.zeros((D + 1, n), dtype=np.int64)
    z = np.zeros((D + 1, n), dtype=np.int64)
    Sset = set(S)
    for w in _walks(A, i):
        if Sset & set(w):
            continue
        first = next((j for j, c in enumerate(cand, start=1) if c in w), None)  # first guess visited
        for d in range(D + 1):
            if first is None or first > d:
                miss[d, w[-1]] += 1
        if first is not None:
            z[first, w[-1]] += 1
    return miss, z


def _recurrence(A, S, cand, L):
    """The masked recurrences of the run: phi^miss under S and one column per guess."""
    n, D = A.shape[0], len(cand)
    inS = np.zeros(n, bool)
    inS[list(S)] = True
    T = [inS.copy()]
    for c in cand:
        t = T[-1].copy()
        t[c] = True
        T.append(t)
    m = (~inS).astype(A.dtype)  # integer counts, or weighted sums for a weighted matrix
    z = np.zeros((D + 1, n), dtype=A.dtype)
    for j, c in enumerate(cand, start=1):
        z[j, c] = 1
    out = []
    for _ in range(L):
        m_new = np.where(inS, 0, A @ m)
        z_new = np.zeros_like(z)
        for j, c in enumerate(cand, start=1):
            z_new[j] = np.where(T[j - 1], 0, A @ z[j])
            # c_j's own row: all walks ending there that avoid T_{j-1}, a difference of the columns
            z_new[j, c] = m_new[c] - z_new[1:j, c].sum()
        m, z = m_new, z_new
        levels = np.array([np.where(T[d], 0, m - z[1:d + 1].sum(axis=0)) for d in range(D + 1)])
        out.append((levels, z.copy()))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_levels_are_differences_of_the_guess_columns(seed):
    g = gg.random_graph_small(6, 0.55, seed)
    A = _adj(g)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n)
    S, cand = [int(perm[0])], [int(x) for x in perm[1:4]]
    L = 4
    rec = _recurrence(A, S, cand, L)
    for i in range(1, L + 1):
        miss, z = _enumerated(A, S, cand, i)
        levels, zr = rec[i - 1]
        # the identity itself, on enumerated counts
        for d in range(len(cand) + 1):
            assert np.array_equal(miss[d], miss[0] - z[1:d + 1].sum(axis=0)), (i, d)
        # the recurrences the sweeps run give the same counts
        assert np.array_equal(levels, miss), i
        assert np.array_equal(zr[1:], z[1:]), i


def test_guess_adjacent_to_earlier_guess_and_star_centre():
    # c_2 is a leaf behind c_1: every walk ending at c_2 (length >= 1) passes c_1 or starts at c_2
    g = gg.star(4)  # centre 0, leaves 1..4
    A = _adj(g)
    S, cand = [3], [0, 1, 2]
    rec = _recurrence(A, S, cand, 4)
    for i in range(1, 5):
        miss, z = _enumerated(A, S, cand, i)
        levels, zr = rec[i - 1]
        assert np.array_equal(levels, miss) and np.array_equal(zr[1:], z[1:]), i
        assert miss[1][1] == 0 and miss[1][2] == 0  # under S + {centre} no walk of length >= 1 remains


@pytest.mark.parametrize("seed", range(4))
def test_levels_of_weighted_walks(seed):
    # Section 5.4's weighted walks with w(v,u) = s_v s_u: a walk counts with the product of its
    # entry weights. The partition by the first guess visited is the same, so the identity and
    # the recurrences hold for the weighted sums; the sweeps apply them to true values.
    g = gg.random_graph_small(6, 0.6, 10 + seed)
    A = _adj(g)
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.2, 1.0, g.n)
    W = A * np.outer(s, s)
    perm = rng.permutation(g.n)
    S, cand = [int(perm[0])], [int(x) for x in perm[1:4]]
    n, D, L = g.n, len(cand), 4
    for i in range(1, L + 1):
        miss = np.zeros((D + 1, n))
        z = np.zeros((D + 1, n))
        for w in _walks(A, i):
            if set(S) & set(w):
                continue
            wt = np.prod([W[w[t], w[t + 1]] for t in range(i)])
            first = next((j for j, c in enumerate(cand, start=1) if c in w), None)
            for d in range(D + 1):
                if first is None or first > d:
                    miss[d, w[-1]] += wt
            if first is not None:
                z[first, w[-1]] += wt
        for d in range(D + 1):
            assert np.allclose(miss[d], miss[0] - z[1:d + 1].sum(axis=0), rtol=1e-12, atol=1e-15), (i, d)
    # the recurrence with weights as coefficients (W in place of A) gives the enumerated sums
    rec = _recurrence(W, S, cand, L)
    levels, zr = rec[L - 1]
    assert np.allclose(levels, miss, rtol=1e-12, atol=1e-15)
    assert np.allclose(zr[1:], z[1:], rtol=1e-12, atol=1e-15)
