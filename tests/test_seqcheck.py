"""The sequence checker of the GPU parity tests (tests/seqcheck.py), on the CPU with the oracle."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from seqcheck import check_sequence, oracle_greedy_checker, oracle_stochastic_checker


def test_identical_sequence_passes_without_divergence():
    g = gg.erdos_renyi(200, 6, 3)
    alpha = oracle.default_alpha(g)
    grp, gains, _ = oracle.greedy(g, 8, alpha, 6, "lazy")
    assert check_sequence(grp, gains, 1e-12, grp, gains, *oracle_greedy_checker(oracle, g, alpha, 6)) == 0


def test_tie_may_part_the_sequences_and_the_rest_is_still_checked():
    # K_n: every vertex outside S has the same gain, so any order is a valid greedy sequence
    g = gg.complete(7)
    alpha, L = 0.1, 4
    ref, refg, _ = oracle.greedy(g, 4, alpha, L, "all")
    mine = [int(ref[1]), int(ref[0]), int(ref[2]), int(ref[3])]
    mg = [oracle.gain(g, mine[:j], mine[j], alpha, L) for j in range(4)]
    parted = check_sequence(mine, mg, 1e-12, ref, refg, *oracle_greedy_checker(oracle, g, alpha, L))
    assert parted >= 1
    # a wrong gain after the tie is still caught
    bad = list(mg)
    bad[3] *= 1.01
    with pytest.raises(AssertionError):
        check_sequence(mine, bad, 1e-12, ref, refg, *oracle_greedy_checker(oracle, g, alpha, L))


def test_a_pick_that_is_not_a_tie_fails():
    g = gg.star(6)  # the centre's gain is far above every leaf's
    alpha, L = 0.1, 4
    ref, refg, _ = oracle.greedy(g, 2, alpha, L, "all")
    assert int(ref[0]) == 0
    mine = [1, 0]
    mg = [oracle.gain(g, mine[:j], mine[j], alpha, L) for j in range(2)]
    with pytest.raises(AssertionError):
        check_sequence(mine, mg, 1e-5, ref, refg, *oracle_greedy_checker(oracle, g, alpha, L))


@pytest.mark.parametrize("seed,eta", [(1, 0.1), (7, 0.3)])
def test_stochastic_continuation_equals_the_oracle_routine(seed, eta):
    # the checker's restatement of one stochastic step, from the empty prefix, reproduces the
    # oracle's own stochastic greedy (same counter-based draws, same argmax)
    g = gg.barabasi_albert(600, 3, 5)
    alpha = oracle.default_alpha(g)
    k, L = 10, 5
    ogrp, ogains, _ = oracle.greedy_stochastic(g, k, alpha, L, eta, seed)
    _, cont = oracle_stochastic_checker(oracle, g, alpha, L, k, eta, seed)
    cg, cgains = cont([], k)
    assert list(cg) == list(ogrp)
    assert np.allclose(cgains, ogains, rtol=1e-14, atol=0)
