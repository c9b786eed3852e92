"""Parity at the configured sizes, in the launch configuration bench.py times.

The whole k = 100 greedy sequences of the benchmarked configurations (R-MAT scale 22 in FP32; the
Barabasi-Albert graph with n = 10^6 in FP32 and FP64) are compared pick by pick and gain by gain
with the oracle's sequences in tests/golden/, written once by tests/golden/make_greedy_goldens.py
from the CPU oracle alone. A pick may differ only where the two gains tie within the tolerance;
the oracle then continues from the GPU's own prefix (here, on the CPU) and the comparison goes on
(tests/seqcheck.py). FP64 gains at n = 10^6 are compared with the long-double oracle: the FP64
oracle's own sequential sums carry rounding near the FP64 tolerance there. Batched scoring is
checked on sampled groups the oracle scores one by one.
"""
import functools
import importlib.util
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from seqcheck import check_sequence, oracle_greedy_checker

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@functools.lru_cache(maxsize=None)
def rmat22():
    return gg.rmat(22, 16, 0.57, 0.19, 0.19, seed=1)


@functools.lru_cache(maxsize=None)
def ba1m():
    return gg.barabasi_albert(1_000_000, 8, seed=1)


def golden(name):
    """(alpha, L, group, gains, long-double gains or None) of the oracle's k = 100 sequence."""
    path = os.path.join(os.path.dirname(__file__), "golden", "make_greedy_goldens.py")
    spec = importlib.util.spec_from_file_location("make_greedy_goldens", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.read(name)


def test_rmat22_greedy_k100_fp32(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    g = rmat22()
    alpha, Lg, ref_grp, ref_gains, _ = golden("rmat22")
    assert alpha == oracle.default_alpha(g)
    G = gedwalk.Graph.from_host(g)
    grp, gains, score, L = G.maximize(100, precision="fp32", epsilon=1e-4)  # the bench configuration
    assert L == Lg
    assert len(set(grp.tolist())) == 100
    check_sequence(grp, gains, TOL32, ref_grp, ref_gains, *oracle_greedy_checker(oracle, g, alpha, L))
    # the gains add up to the score of the final group (FP64 oracle, same L)
    want = oracle.score(g, grp, alpha, L)
    assert rel(score, want) < TOL32
    assert rel(gains.sum(), want) < TOL32
    G.free()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_ba1m_greedy_k100(cuda_device, prec):
    from paper_1910_13874_gb300 import gedwalk

    g = ba1m()
    alpha, Lg, ref_grp, ref_gains, ref_ld = golden("ba1m")
    assert alpha == oracle.default_alpha(g) and ref_ld is not None
    G = gedwalk.Graph.from_host(g)
    grp, gains, score, L = G.maximize(100, precision=prec, epsilon=1e-4)
    assert L == Lg
    fp64 = prec == "fp64"
    tol = TOL64 if fp64 else TOL32
    check_sequence(grp, gains, tol, ref_grp, ref_ld if fp64 else ref_gains,
                   *oracle_greedy_checker(oracle, g, alpha, L, long_double=fp64))
    assert rel(score, oracle.score(g, grp, alpha, L, long_double=fp64)) < tol
    G.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ba1m_greedy_k10(cuda_device, prec):
    from paper_1910_13874_gb300 import gedwalk

    g = ba1m()
    G = gedwalk.Graph.from_host(g)
    alpha = oracle.default_alpha(g)
    grp, gains, score, L = G.maximize(10, precision=prec, epsilon=1e-4)
    tol = TOL64 if prec == "fp64" else TOL32
    fp64 = prec == "fp64"
    ogrp, _, _ = oracle.greedy(g, 10, alpha, L, "lazy")
    ref = [oracle.gain(g, list(ogrp[:j]), int(ogrp[j]), alpha, L, long_double=fp64) for j in range(10)]
    check_sequence(grp, gains, tol, ogrp, ref, *oracle_greedy_checker(oracle, g, alpha, L, long_double=fp64))
    assert rel(score, oracle.score(g, grp, alpha, L, long_double=True)) < tol
    G.free()


def test_ba1m_batch_4096_groups(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    g = ba1m()
    G = gedwalk.Graph.from_host(g)
    alpha = oracle.default_alpha(g)
    off, mem = gg.random_groups(g.n, 4096, 1, 100, 42)  # the batched-scoring configuration
    scores, L = G.score_batch(off, mem, epsilon=1e-4)
    rng = np.random.default_rng(0)
    for j in rng.choice(4096, size=12, replace=False):
        S = mem[off[j]:off[j + 1]]
        assert rel(scores[j], oracle.score(g, S, alpha, L)) < TOL32, j
    # the per-group FP64 path agrees as well (long-double oracle: see test_ba1m_greedy_k10)
    for j in (0, 4095):
        s64, _, _ = G.score(mem[off[j]:off[j + 1]], precision="fp64", epsilon=1e-4)
        assert rel(s64, oracle.score(g, mem[off[j]:off[j + 1]], alpha, L, long_double=True)) < TOL64
        assert rel(scores[j], s64) < TOL32
    G.free()
