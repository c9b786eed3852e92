"""Directed graphs (Section 2) on the GPU against the CPU oracle, through the C ABI.

The rows are successor lists. Scores and gains run on them; the Lemma-initialize bound also
needs the S-avoiding walks of the other orientation (psi^miss, computed on the reverse CSR), and
batched scoring takes its walk-total table from the reverse CSR. The combinatorial bound uses
d = min(max out-degree, max in-degree). Tolerances as for undirected graphs.
"""
import functools

import numpy as np
import pytest

import graphgen as gg
import oracle
from seqcheck import check_sequence, oracle_greedy_checker

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@functools.lru_cache(maxsize=None)
def host(name):
    if name == "rmat14d":
        return gg.rmat(14, 16, seed=3, directed=True)  # heavy rows in both orientations, isolated vertices
    if name == "rmat12d":
        return gg.rmat(12, 8, seed=6, directed=True)
    if name == "digraph":
        return gg.random_digraph(600, 0.01, 4)
    if name == "outstar":  # hub with out-degree 1500 (sliced), in-degree 0; leaves point on along a chain
        arcs = [(0, v) for v in range(1, 1501)] + [(v, v + 1) for v in range(1, 1500)] + [(1600, 3)]
        return gg.from_arcs(1700, arcs)
    raise KeyError(name)


_dev = {}


def dev(name):
    from paper_1910_13874_gb300 import gedwalk

    if name not in _dev:
        _dev[name] = gedwalk.Graph.from_host(host(name), directed=True)
    return _dev[name]


NAMES = ["rmat14d", "rmat12d", "digraph", "outstar"]


@pytest.mark.parametrize("name", NAMES)
def test_directed_alpha_and_truncation(cuda_device, name):
    g = host(name)
    G = dev(name)
    assert G.directed
    assert G.delta == oracle.delta(g, directed=True)
    alpha = oracle.default_alpha(g, directed=True)
    assert G.alpha_default == alpha
    for eps in (1e-3, 1e-6):
        L, B = G.truncation(0.0, eps)
        Lo, Bo = oracle.select_L(g, alpha, eps, directed=True)
        assert L == Lo and rel(B, Bo) < 1e-12


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_directed_score_matches_oracle(cuda_device, name, prec):
    g = host(name)
    G = dev(name)
    alpha = oracle.default_alpha(g, directed=True)
    off, mem = gg.random_groups(g.n, 6, 1, 40, 21)
    for j in range(6):
        S = mem[off[j]:off[j + 1]]
        s, L, _ = G.score(S, precision=prec, epsilon=1e-5)
        want = oracle.score(g, S, alpha, L)
        assert rel(s, want) < TOL[prec], (j, s, want)
    s, L, _ = G.score([0], precision=prec, epsilon=1e-5)
    assert rel(s, oracle.score(g, [0], alpha, L)) < TOL[prec]


@pytest.mark.parametrize("name", NAMES)
def test_directed_batch_matches_oracle(cuda_device, name):
    # first-visit form: F from the successor lists, the walk totals K from the reverse CSR
    g = host(name)
    G = dev(name)
    alpha = oracle.default_alpha(g, directed=True)
    off, mem = gg.random_groups(g.n, 40, 1, 30, 23)
    scores, L = G.score_batch(off, mem, epsilon=1e-5)
    for j in range(40):
        S = mem[off[j]:off[j + 1]]
        assert rel(scores[j], oracle.score(g, S, alpha, L)) < 1e-5, j


@pytest.mark.parametrize("name", ["rmat12d", "outstar"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_directed_gains_match_oracle(cuda_device, name, prec):
    g = host(name)
    G = dev(name)
    alpha = oracle.default_alpha(g, directed=True)
    S = [0, 5, 9]
    gains, L = G.gains(S, precision=prec, epsilon=1e-4)
    rng = np.random.default_rng(5)
    for x in list(rng.choice(g.n, size=25, replace=False)) + S + [1, 2]:
        want = oracle.gain(g, S, int(x), alpha, L)
        assert gains[x] == want == 0.0 or rel(gains[x], want) < TOL[prec], (x, gains[x], want)


@pytest.mark.parametrize("name,k", [("rmat14d", 12), ("rmat12d", 10), ("digraph", 8), ("outstar", 5)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_directed_maximize_matches_oracle(cuda_device, name, k, prec):
    # certification relies on the two-orientation bound: a wrong psi would let a bound undercut a gain
    g = host(name)
    G = dev(name)
    alpha = oracle.default_alpha(g, directed=True)
    grp, gains, score, L = G.maximize(k, precision=prec, epsilon=1e-4)
    ogrp, ogains, _ = oracle.greedy(g, k, alpha, L, "lazy", directed=True)
    tol = TOL[prec]
    # only a tie inside the tolerance may part the sequences; the oracle then continues from the
    # GPU's own prefix
    check_sequence(grp, gains, tol, ogrp, ogains,
                   *oracle_greedy_checker(oracle, g, alpha, L, directed=True))
    assert rel(score, oracle.score(g, grp, alpha, L)) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_directed_adaptive(cuda_device, prec):
    g = host("rmat12d")
    G = dev("rmat12d")
    alpha = oracle.default_alpha(g, directed=True)
    k, eps = 6, 1e-4
    grp, gains, score, L = G.maximize(k, precision=prec, epsilon=eps, adaptive=True)
    ell, _ = G.maximize_lengths()
    ref = oracle.greedy_adaptive(g, k, alpha, eps / k, directed=True)
    for j in range(k):
        want = oracle.gain(g, list(grp[:j]), int(grp[j]), alpha, int(ell[j]))
        assert rel(gains[j], want) < TOL[prec], j
    assert grp[0] == ref["group"][0] and ell[0] == ref["ell"][0]


def test_directed_rejects_weighted_and_checks_rows(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    g = host("digraph")
    with pytest.raises(gedwalk.GedWalkError):
        gedwalk.Graph.from_host(g, directed=True, weighted=True)
    bad = gg.Graph(np.array([0, 2, 2, 2], np.int32), np.array([1, 1], np.int32))  # repeated arc
    with pytest.raises(gedwalk.GedWalkError):
        gedwalk.Graph.from_host(bad, directed=True)
