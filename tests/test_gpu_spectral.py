"""Spectral bound (Lemma spectral-bound) and sigma_max on the GPU, through the C ABI.

sigma_max comes from a sparse eigen/singular value solver (scipy) here, independent of the
library; for the normalised adjacency of a connected graph it is exactly 1. The library's value
is a certified upper bound (Collatz-Wielandt) that must not fall below the solver's and must
come close to it after enough power iterations. With alpha = delta / sigma_max (Appendix E) the
truncation lengths and the scores must match the oracle's at the solver's sigma.
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
def case(name):
    """(graph, directed, weights for the oracle or None)."""
    if name == "er1000":
        return gg.erdos_renyi(1000, 10, 1), False, None
    if name == "ba5000":
        return gg.barabasi_albert(5000, 4, 2), False, None
    if name == "rmat12":
        return gg.rmat(12, 16, seed=8), False, None
    if name == "rmat12d":
        return gg.rmat(12, 8, seed=6, directed=True), True, None
    if name == "ba5000w":
        g = gg.barabasi_albert(5000, 4, 2)
        return g, False, oracle.normalized_weights(g)
    raise KeyError(name)


@functools.lru_cache(maxsize=None)
def sigma_true(name):
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    g, directed, w = case(name)
    if w is not None:
        return 1.0  # D^{-1/2} A D^{-1/2} of a connected graph: largest eigenvalue exactly 1
    A = sp.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    if directed:
        return float(sla.svds(A, k=1, return_singular_vectors=False, tol=1e-14)[0])
    return float(sla.eigsh(A, k=1, which="LA", return_eigenvectors=False, tol=1e-14)[0])


_dev = {}


def dev(name):
    from paper_1910_13874_gb300 import gedwalk

    if name not in _dev:
        g, directed, w = case(name)
        G = gedwalk.Graph.from_host(g, directed=directed, weighted=w is not None)
        G.sigma_max(4000)
        _dev[name] = G
    return _dev[name]


NAMES = ["er1000", "ba5000", "rmat12", "rmat12d", "ba5000w"]


@pytest.mark.parametrize("name", NAMES)
def test_sigma_max_is_certified_and_tight(cuda_device, name):
    G = dev(name)
    s = sigma_true(name)
    up, lo = G.sigma_max(10)  # a few more iterations never loosen the kept value
    assert up >= s * (1 - 1e-12), (up, s)
    assert lo <= s * (1 + 1e-9), (lo, s)
    assert up <= s * (1 + 1e-7), (up, s)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("delta", [0.3, 0.6])
def test_spectral_truncation_matches_oracle(cuda_device, name, delta):
    g, directed, w = case(name)
    G = dev(name)
    s = sigma_true(name)
    alpha = delta / s
    for eps in (1e-2, 1e-5):
        L, B = G.truncation(alpha, eps, bound="spectral")
        Lo, Bo = oracle.select_L_spectral(g, alpha, eps, s, w=w)
        # B_l depends on sigma through alpha sigma / (1 - alpha sigma): a relative sigma excess e moves
        # it by about e / (1 - delta)
        assert L == Lo and rel(B, Bo) < 1e-6, (L, Lo, B, Bo)


def test_spectral_reaches_beyond_the_combinatorial_bound(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    G = dev("rmat12")
    alpha = 0.5 / sigma_true("rmat12")
    assert alpha * G.dmax >= 1.0
    with pytest.raises(gedwalk.GedWalkError):
        G.truncation(alpha, 1e-4)  # combinatorial: not convergent
    with pytest.raises(gedwalk.GedWalkError):
        G.truncation(1.01 / sigma_true("rmat12"), 1e-4, bound="spectral")


@pytest.mark.parametrize("name", ["rmat12", "rmat12d", "ba5000w"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_spectral_score_and_maximize_match_oracle(cuda_device, name, prec):
    g, directed, w = case(name)
    G = dev(name)
    alpha = 0.5 / sigma_true(name)
    off, mem = gg.random_groups(g.n, 4, 1, 30, 29)
    for j in range(4):
        S = mem[off[j]:off[j + 1]]
        sc, L, _ = G.score(S, alpha=alpha, precision=prec, epsilon=1e-4, bound="spectral")
        assert L == oracle.select_L_spectral(g, alpha, 1e-4, sigma_true(name), w=w)[0]
        assert rel(sc, oracle.score(g, S, alpha, L, w=w)) < TOL[prec], j
    k = 5
    grp, gains, score, L = G.maximize(k, alpha=alpha, precision=prec, epsilon=1e-3, bound="spectral")
    ogrp, ogains, _ = oracle.greedy(g, k, alpha, L, "lazy", w=w, directed=directed)
    check_sequence(grp, gains, TOL[prec], ogrp, ogains,
                   *oracle_greedy_checker(oracle, g, alpha, L, w=w, directed=directed))
