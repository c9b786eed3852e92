"""Comparison of a GPU greedy sequence with the oracle's, under the tie rule of the parity tests.

The picks must be identical wherever the oracle's best gain is separated from the GPU's pick by
more than the tolerance. Where they differ, the GPU's pick must tie with the oracle's (the oracle's
gain of the GPU's pick, under the same prefix, within the tolerance of the best gain); from there
on the oracle continues from the GPU's own prefix, so every later pick is still compared.
"""
import numpy as np


def rel(a, b):
    return abs(float(a) - float(b)) / max(abs(float(b)), 1e-300)


def check_sequence(grp, gains, tol, ref_grp, ref_gains, gain_of, continue_from):
    """grp, gains: the GPU's picks and gains. ref_grp, ref_gains: the oracle's sequence from the
    same start. gain_of(prefix, v): the oracle's gain of v after prefix. continue_from(prefix, count):
    the oracle's next `count` picks and gains after prefix. Returns the number of divergences."""
    k = len(grp)
    ref_grp = [int(v) for v in ref_grp]
    ref_gains = [float(x) for x in ref_gains]
    parted = 0
    for j in range(k):
        v, want_v, want_g = int(grp[j]), ref_grp[j], ref_gains[j]
        if v == want_v:
            assert gains[j] == want_g == 0.0 or rel(gains[j], want_g) < tol, (j, v, gains[j], want_g)
            continue
        mine = gain_of([int(x) for x in grp[:j]], v)
        assert abs(mine - want_g) <= tol * abs(want_g), ("pick differs without a tie", j, v, mine, want_v, want_g)
        assert mine == gains[j] == 0.0 or rel(gains[j], mine) < tol, (j, v, gains[j], mine)
        parted += 1
        if j + 1 < k:
            cg, cgains = continue_from([int(x) for x in grp[: j + 1]], k - j - 1)
            ref_grp[j + 1:] = [int(x) for x in cg]
            ref_gains[j + 1:] = [float(x) for x in cgains]
    return parted


def oracle_greedy_checker(oracle, g, alpha, L, w=None, directed=False, long_double=False):
    """gain_of / continue_from for the oracle's fixed-length greedy on graph g."""

    def gain_of(prefix, v):
        return oracle.gain(g, prefix, v, alpha, L, w=w, long_double=long_double)

    def continue_from(prefix, count):
        cg, cgains, _ = oracle.greedy(g, count, alpha, L, "lazy", init=prefix, w=w, directed=directed)
        if long_double:
            cgains = [oracle.gain(g, list(prefix) + [int(x) for x in cg[:i]], int(cg[i]), alpha, L, w=w,
                                  long_double=True) for i in range(len(cg))]
        return cg, np.asarray(cgains)

    return gain_of, continue_from


def oracle_stochastic_checker(oracle, g, alpha, L, k, eta, seed, w=None):
    """gain_of / continue_from for stochastic greedy (Appendix D): the step-j sample is drawn by the
    oracle's counter-based hash (vertex v outside S when hash(seed, j, v) < p 2^64, p = m / |V \\ S|,
    m = ceil((n/k) ln(1/eta)); all of V \\ S when nothing is drawn), and within it the oracle's best
    exact gain wins, the lowest id among equal gains."""
    import math

    n = g.n
    m = math.ceil(n / k * math.log(1.0 / eta))

    def gain_of(prefix, v):
        return oracle.gain(g, prefix, v, alpha, L, w=w)

    def continue_from(prefix, count):
        S = [int(x) for x in prefix]
        out_v, out_g = [], []
        for j in range(len(S), len(S) + count):
            inS = set(S)
            p = m / (n - j)
            rest = [v for v in range(n) if v not in inS]
            cand = rest if p >= 1.0 else [v for v in rest if oracle.sample_hash(seed, j, v) < int(p * 2.0 ** 64)]
            if not cand:
                cand = rest
            best_v, best_g = -1, -1.0
            for v in cand:
                gv = oracle.gain(g, S, v, alpha, L, w=w)
                if gv > best_g:
                    best_v, best_g = v, gv
            out_v.append(best_v)
            out_g.append(best_g)
            S.append(best_v)
        return np.asarray(out_v), np.asarray(out_g)

    return gain_of, continue_from
