"""Weighted GED-Walk (Section 5.4) on the GPU against the CPU oracle, through the C ABI.

A walk of length i contributes alpha^i times the product of its edge weights. The library takes
vertex-separable weights w(v, u) = s_v s_u: the symmetrically normalised adjacency
D^{-1/2} A D^{-1/2} (no scales given) or caller scales. The oracle receives the same weights as
one value per CSR entry. Tolerances as for the unweighted path: FP64 1e-12, FP32 1e-5 relative.
Both sides use the oracle's alpha, so that the comparison does not hinge on the last bit of
alpha = 1/(1 + delta).
"""
import functools

import numpy as np
import pytest

import graphgen as gg
import oracle
from seqcheck import check_sequence, oracle_greedy_checker, oracle_stochastic_checker

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@functools.lru_cache(maxsize=None)
def case(name):
    """(host graph, vertex scales or None, entry weights for the oracle)."""
    if name == "er1000":
        g = gg.erdos_renyi(1000, 10, 1)
    elif name == "ba5000":
        g = gg.barabasi_albert(5000, 4, 2)
    elif name in ("rmat14", "rmat14_scaled"):
        g = gg.rmat(14, 16, seed=3)  # heavy rows split across warps, and isolated vertices
    elif name == "isolated":
        g = gg.from_edges(30, [(0, 1), (1, 2), (2, 0), (5, 6), (6, 7), (7, 8), (8, 5), (5, 7)])
    else:
        raise KeyError(name)
    if name.endswith("_scaled"):
        scale = np.random.default_rng(7).uniform(0.2, 1.0, size=g.n)
        rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        return g, scale, scale[rows] * scale[g.col_idx]
    return g, None, oracle.normalized_weights(g)


_dev = {}


def dev(name):
    from paper_1910_13874_gb300 import gedwalk

    if name not in _dev:
        g, scale, _ = case(name)
        _dev[name] = gedwalk.Graph.from_host(g, weighted=True, vertex_scale=scale)
    return _dev[name]


NAMES = ["er1000", "ba5000", "rmat14", "rmat14_scaled", "isolated"]


@pytest.mark.parametrize("name", NAMES)
def test_weighted_delta_alpha_and_truncation(cuda_device, name):
    g, _, w = case(name)
    G = dev(name)
    assert G.weighted
    assert rel(G.delta, oracle.delta(g, w)) < 1e-14
    assert rel(G.alpha_default, oracle.default_alpha(g, w)) < 1e-14
    alpha = oracle.default_alpha(g, w)
    # At alpha = 1/(1 + delta) the bound's factor alpha delta / (1 - alpha delta) amplifies the last-bit
    # difference of delta (summed in another order on each side) by about 1 + delta.
    tol_b = 1e-12 + (1.0 + G.delta) * 1e-14
    for eps in (1e-3, 1e-6):
        L, B = G.truncation(alpha, eps)
        Lo, Bo = oracle.select_L(g, alpha, eps, w=w)
        assert L == Lo and rel(B, Bo) < tol_b


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weighted_score_matches_oracle(cuda_device, name, prec):
    g, _, w = case(name)
    G = dev(name)
    alpha = oracle.default_alpha(g, w)
    off, mem = gg.random_groups(g.n, 6, 1, min(40, g.n), 13)
    for j in range(6):
        S = mem[off[j]:off[j + 1]]
        s, L, _ = G.score(S, alpha=alpha, precision=prec, epsilon=1e-5)
        want = oracle.score(g, S, alpha, L, w=w)
        assert rel(s, want) < TOL[prec], (j, s, want)


@pytest.mark.parametrize("name", ["ba5000", "rmat14", "rmat14_scaled", "isolated"])
def test_weighted_batch_matches_oracle(cuda_device, name):
    # first-visit form with scaled vectors and the scaled walk-total table
    g, _, w = case(name)
    G = dev(name)
    alpha = oracle.default_alpha(g, w)
    off, mem = gg.random_groups(g.n, 40, 1, min(30, g.n), 17)
    scores, L = G.score_batch(off, mem, alpha=alpha, epsilon=1e-5)
    for j in range(40):
        S = mem[off[j]:off[j + 1]]
        assert rel(scores[j], oracle.score(g, S, alpha, L, w=w)) < 1e-5, j


@pytest.mark.parametrize("name", ["er1000", "rmat14_scaled", "isolated"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weighted_gains_match_oracle(cuda_device, name, prec):
    g, _, w = case(name)
    G = dev(name)
    alpha = oracle.default_alpha(g, w)
    S = [0, 2, 7]
    gains, L = G.gains(S, alpha=alpha, precision=prec, epsilon=1e-4)
    rng = np.random.default_rng(3)
    for x in list(rng.choice(g.n, size=min(25, g.n), replace=False)) + S:
        want = oracle.gain(g, S, int(x), alpha, L, w=w)
        assert gains[x] == want == 0.0 or rel(gains[x], want) < TOL[prec], (x, gains[x], want)


@pytest.mark.parametrize("name,k", [("er1000", 6), ("ba5000", 12), ("rmat14", 12), ("rmat14_scaled", 10)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weighted_maximize_matches_oracle(cuda_device, name, k, prec):
    g, _, w = case(name)
    G = dev(name)
    alpha = oracle.default_alpha(g, w)
    grp, gains, score, L = G.maximize(k, alpha=alpha, precision=prec, epsilon=1e-4)
    ogrp, ogains, _ = oracle.greedy(g, k, alpha, L, "lazy", w=w)
    tol = TOL[prec]
    # only a tie inside the tolerance may part the sequences; the oracle then continues from the
    # GPU's own prefix
    check_sequence(grp, gains, tol, ogrp, ogains, *oracle_greedy_checker(oracle, g, alpha, L, w=w))
    assert rel(score, oracle.score(g, grp, alpha, L, w=w)) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weighted_adaptive_and_stochastic(cuda_device, prec):
    g, _, w = case("ba5000")
    G = dev("ba5000")
    alpha = oracle.default_alpha(g, w)
    tol = TOL[prec]
    k, eps = 8, 1e-4
    grp, gains, score, L = G.maximize(k, alpha=alpha, precision=prec, epsilon=eps, adaptive=True)
    ell, _ = G.maximize_lengths()
    ref = oracle.greedy_adaptive(g, k, alpha, eps / k, w=w)
    for j in range(k):  # validity at every step: the pick's exact gain at its length
        want = oracle.gain(g, list(grp[:j]), int(grp[j]), alpha, int(ell[j]), w=w)
        assert rel(gains[j], want) < tol, j
    assert grp[0] == ref["group"][0] and ell[0] == ref["ell"][0]
    grp, gains, score, L = G.maximize(k, alpha=alpha, precision=prec, epsilon=eps, stochastic=True, eta=0.2, seed=3)
    ogrp, ogains, _ = oracle.greedy_stochastic(g, k, alpha, L, 0.2, 3, w=w)
    check_sequence(grp, gains, tol, ogrp, ogains,
                   *oracle_stochastic_checker(oracle, g, alpha, L, k, 0.2, 3, w=w))


def test_weighted_rejects_bad_scales(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    g = gg.cycle(5)
    for bad in ([1, 1, 0, 1, 1], [1, 1, -2, 1, 1], [1, 1, float("nan"), 1, 1]):
        with pytest.raises(gedwalk.GedWalkError):
            gedwalk.Graph.from_host(g, vertex_scale=np.array(bad, dtype=np.float64))
