"""CUDA library vs the CPU oracle, element by element, through the C ABI.

Tolerances (stated by the specification this library follows): FP64 walk vectors match the
FP64 oracle to relative error 1e-12 per score and gain; FP32 walk vectors (FP64 sums) to 1e-5.
The selected greedy sequence must be identical wherever the top two oracle gains differ by
more than the tolerance; elsewhere the chosen vertex's oracle gain must be within the
tolerance of the best one. Gains that are exactly zero (members of S, isolated vertices) must
be exactly zero.

Graphs: the 1000-vertex Erdos-Renyi graph of the small configuration (average degree 10),
Barabasi-Albert and R-MAT graphs large enough to have rows split across several CTAs
(degree > 1024) and many light units, plus the special graphs with closed forms.
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@functools.lru_cache(maxsize=None)
def host_graph(name):
    if name == "er1000":
        return gg.erdos_renyi(1000, 10, 1)
    if name == "ba5000":
        return gg.barabasi_albert(5000, 4, 2)
    if name == "rmat14":
        return gg.rmat(14, 16, seed=3)
    if name == "rmat15":
        return gg.rmat(15, 16, seed=4)
    if name == "k8":
        return gg.complete(8)
    if name == "star":
        return gg.star(40)
    if name == "path":
        return gg.path(50)
    if name == "isolated":
        return gg.from_edges(30, [(0, 1), (1, 2), (2, 0), (5, 6), (6, 7), (7, 8), (8, 5), (5, 7)])
    raise KeyError(name)


_dev = {}


def dev_graph(name):
    from paper_1910_13874_gb300 import gedwalk

    if name not in _dev:
        _dev[name] = gedwalk.Graph.from_host(host_graph(name))
    return _dev[name]


def groups(n, count, lo, hi, seed):
    off, mem = gg.random_groups(n, count, lo, hi, seed)
    return [mem[off[j]:off[j + 1]] for j in range(count)]


# ------------------------------------------------------------------ truncation length
@pytest.mark.parametrize("name,eps", [("er1000", 1e-6), ("er1000", 1e-3), ("ba5000", 1e-4), ("rmat14", 1e-4)])
def test_truncation_length_matches_oracle(cuda_device, name, eps):
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    assert G.alpha_default == alpha
    L, B = G.truncation(0.0, eps)
    Lo, Bo = oracle.select_L(g, alpha, eps)
    assert L == Lo
    assert rel(B, Bo) < 1e-12


def _golden_truncations():
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "comb_bound.txt")
    return [tuple(x.strip() for x in ln.split(";")) for ln in open(path)
            if ln.strip() and not ln.startswith("#") and ln.startswith("L ")]


@pytest.mark.parametrize("rec", _golden_truncations(), ids=lambda r: "-".join(r[1:4]))
def test_truncation_length_matches_hand_values(cuda_device, rec):
    # Eq. comb-bound and Algorithm 1's strict stop test against values derived by hand
    # (tests/golden/comb_bound.txt), independent of the oracle: the device's walk totals and
    # its first-crossing test must give the same L and B_L.
    from fractions import Fraction

    from paper_1910_13874_gb300 import gedwalk

    cube = gg.from_edges(8, [(u, v) for u in range(8) for v in range(u + 1, 8) if bin(u ^ v).count("1") == 1])
    g = {"K4": gg.complete(4), "C5": gg.cycle(5), "star3": gg.star(3), "Q3": cube}[rec[1]]
    G = gedwalk.Graph.from_host(g)
    L, B = G.truncation(float(Fraction(rec[2])), float(rec[3]))
    assert L == int(rec[4])
    assert rel(B, float(Fraction(rec[5]))) < 1e-14
    G.free()


# ------------------------------------------------------------------ scoring one group
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_score_small_config_16_groups(cuda_device, prec):
    # the small configuration: 16 random groups of 5 vertices, epsilon 1e-6
    g = host_graph("er1000")
    G = dev_graph("er1000")
    alpha = oracle.default_alpha(g)
    for S in groups(g.n, 16, 5, 5, 42):
        s, L, B = G.score(S, precision=prec, epsilon=1e-6)
        Lo, Bo = oracle.select_L(g, alpha, 1e-6)
        assert L == Lo
        want = oracle.score(g, S, alpha, L)
        assert rel(s, want) < TOL[prec], (S, s, want)
        assert rel(B, Bo) < 1e-12


@pytest.mark.parametrize("name", ["ba5000", "rmat14", "rmat15", "star", "path", "isolated"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_score_graphs(cuda_device, name, prec):
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    rng = np.random.default_rng(7)
    for size in (1, 2, 17, 60):
        size = min(size, g.n)
        S = rng.choice(g.n, size=size, replace=False)
        L = 6
        s, Lu, _ = G.score(S, precision=prec, L=L)
        assert Lu == L
        want = oracle.score(g, S, alpha, L)
        assert rel(s, want) < TOL[prec], (name, size, s, want)
    # the highest-degree vertex (a row split over several CTAs in the R-MAT graphs)
    hub = int(np.argmax(g.degrees))
    s, _, _ = G.score([hub], precision=prec, L=5)
    assert rel(s, oracle.score(g, [hub], alpha, 5)) < TOL[prec]


def test_score_closed_forms_and_edge_cases(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    G = dev_graph("k8")
    # K_n: phi_i = n(n-1)^i - (n-s)(n-s-1)^i; alpha = 1/8 keeps the arithmetic exact
    n, s_, L = 8, 3, 5
    want = sum(0.125 ** i * (n * (n - 1) ** i - (n - s_) * (n - s_ - 1) ** i) for i in range(1, L + 1))
    for prec in ("fp64", "fp32"):
        got, _, _ = G.score([0, 1, 2], precision=prec, alpha=0.125, L=L)
        assert got == want
        # duplicates are a set
        assert G.score([2, 1, 0, 1, 2], precision=prec, alpha=0.125, L=L)[0] == want
        assert G.score([], precision=prec, alpha=0.125, L=L)[0] == 0.0
    # S = V gives GED_{<=L}(V) = sum_x Katz_{<=L}(x) (Prop. katz-relation)
    gi = host_graph("isolated")
    Gi = dev_graph("isolated")
    alpha = oracle.default_alpha(gi)
    _, Wa = oracle.walk_totals(gi, alpha, 6)
    assert rel(Gi.score(np.arange(gi.n), precision="fp64", L=6)[0], Wa[1:].sum()) < 1e-12
    # isolated vertices score exactly 0
    assert Gi.score([20, 25], precision="fp32", L=6)[0] == 0.0
    with pytest.raises(gedwalk.GedWalkError) as e:
        Gi.score([0, 30], L=3)
    assert e.value.status == gedwalk.ERR_INVALID
    with pytest.raises(gedwalk.GedWalkError) as e:
        Gi.score([0], alpha=0.5, epsilon=1e-4)  # alpha * d_max >= 1
    assert e.value.status == gedwalk.ERR_NOT_CONVERGENT
    assert Gi.score([0], alpha=0.5, L=3)[0] == pytest.approx(oracle.score(gi, [0], 0.5, 3), rel=1e-12)


def test_upload_rejects_malformed_graphs(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    g = gg.from_edges(4, [(0, 1), (1, 2)])
    bad_sym = g.col_idx.copy()
    bad_sym[0] = 3  # row 0 now lists 3, row 3 does not list 0
    for rp, ci in [(g.row_ptr, bad_sym), (g.row_ptr, np.array([1, 0, 2, 1], np.int32) * 9),
                   (np.array([0, 1, 1, 3, 3], np.int32), np.array([0, 1, 2], np.int32))]:
        with pytest.raises(gedwalk.GedWalkError) as e:
            gedwalk.Graph(rp, ci)
        assert e.value.status == gedwalk.ERR_INVALID
    # A missing mirror is found from the endpoint of smaller (degree, id) (row 0 above), or, when
    # only the up/down entry counts disagree, by the full pass: here vertex 4 lists the hub 0, which
    # does not list 4 back.
    rp = np.array([0, 3, 4, 5, 6, 7], np.int32)
    ci = np.array([1, 2, 3, 0, 0, 0, 0], np.int32)
    with pytest.raises(gedwalk.GedWalkError) as e:
        gedwalk.Graph(rp, ci)
    assert e.value.status == gedwalk.ERR_INVALID and "row 4" in str(e.value) and "symmetric" in str(e.value)
    with pytest.raises(gedwalk.GedWalkError) as e:
        gedwalk.Graph(g.row_ptr, bad_sym)
    assert "row 0" in str(e.value) and "symmetric" in str(e.value)
    # row pointers that decrease are caught before any entry is read
    with pytest.raises(gedwalk.GedWalkError) as e:
        gedwalk.Graph(np.array([0, 2, 1, 3], np.int32), np.array([1, 2, 0], np.int32))
    assert "row 1" in str(e.value) and "row_ptr decreases" in str(e.value)
    # the same lists pass when declared directed, and a symmetric star passes undirected
    gedwalk.Graph(rp, ci, directed=True).free()
    st = gg.star(40)
    gedwalk.Graph(st.row_ptr, st.col_idx).free()


# ------------------------------------------------------------------ exact gains of every vertex
@pytest.mark.parametrize("name", ["er1000", "rmat14", "isolated"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_all_vertex_gains(cuda_device, name, prec):
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    L = 5
    S = [int(np.argmax(g.degrees)), 3, 7]
    gains, Lu = G.gains(S, precision=prec, L=L)
    assert Lu == L
    xs = range(g.n) if g.n <= 1000 else np.random.default_rng(1).choice(g.n, 300, replace=False)
    for x in xs:
        want = oracle.gain(g, S, int(x), alpha, L)
        if want == 0.0:
            assert gains[x] == 0.0, x
        else:
            assert rel(gains[x], want) < TOL[prec], (x, gains[x], want)


# ------------------------------------------------------------------ greedy maximisation
def check_greedy(g, grp, gains, alpha, L, tol, init=()):
    """Each pick is the oracle's best next vertex for the GPU's own prefix, or within tol of it.

    With a tie inside the tolerance the sequences may part; from then on every GPU pick is
    still compared with the oracle's best continuation of the GPU's prefix.
    """
    S = list(init)
    for step, v in enumerate(grp):
        v = int(v)
        ob, obg, _ = oracle.greedy(g, 1, alpha, L, "lazy", init=S or None)
        gv = oracle.gain(g, S, v, alpha, L)
        if gv == 0.0:
            assert gains[step] == 0.0, step
        else:
            assert rel(gains[step], gv) < tol, (step, gains[step], gv)
        if v != int(ob[0]):
            assert gv >= obg[0] * (1 - tol), (step, v, gv, int(ob[0]), obg[0])
        S.append(v)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_maximize_small_config_all_gains(cuda_device, prec):
    # the small configuration: greedy k=5 with every vertex's exact gain compared at every step
    g = host_graph("er1000")
    G = dev_graph("er1000")
    alpha = oracle.default_alpha(g)
    grp, gains, score, L = G.maximize(5, precision=prec, epsilon=1e-6, gains_all=True)
    L_o, _ = oracle.select_L(g, alpha, 1e-6 / 5)
    assert L == L_o
    ogrp, ogains, _ = oracle.greedy(g, 5, alpha, L, "all")
    assert list(grp) == list(ogrp)
    assert np.all(rel(gains, ogains) < TOL[prec])
    assert rel(score, oracle.score(g, grp, alpha, L)) < TOL[prec]
    # the pruned path chooses the same group
    grp2, gains2, _, _ = G.maximize(5, precision=prec, epsilon=1e-6)
    assert list(grp2) == list(grp)
    assert np.all(rel(gains2, ogains) < TOL[prec])


@pytest.mark.parametrize("name,k", [("ba5000", 25), ("rmat14", 25), ("rmat15", 12), ("er1000", 12)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_maximize_graphs(cuda_device, name, k, prec):
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    grp, gains, score, L = G.maximize(k, precision=prec, epsilon=1e-4)
    assert len(set(grp.tolist())) == k
    check_greedy(g, grp, gains, alpha, L, TOL[prec])
    assert rel(score, oracle.score(g, grp, alpha, L)) < TOL[prec]


def test_maximize_ties_go_to_lowest_id(cuda_device):
    G = dev_graph("k8")
    for prec in ("fp64", "fp32"):
        grp, gains, _, _ = G.maximize(5, precision=prec, alpha=0.125, L=4)
        assert list(grp) == [0, 1, 2, 3, 4]
    # star: the centre first, then every gain is 0 and the lowest leaf follows
    Gs = dev_graph("star")
    grp, gains, _, _ = Gs.maximize(3, precision="fp32", L=5)
    assert list(grp) == [0, 1, 2] and gains[1] == 0.0 and gains[2] == 0.0


def test_maximize_isolated_and_resume(cuda_device):
    g = host_graph("isolated")
    G = dev_graph("isolated")
    alpha = oracle.default_alpha(g)
    # more picks than vertices with positive gain: zeros go to the lowest ids
    grp, gains, _, L = G.maximize(12, precision="fp64", L=6)
    ogrp, ogains, _ = oracle.greedy(g, 12, alpha, 6, "all")
    assert list(grp) == list(ogrp)
    assert np.all(rel(gains, ogains) < 1e-12)
    # resuming from a prefix reproduces the rest
    g2 = host_graph("rmat14")
    G2 = dev_graph("rmat14")
    full, fg, _, L = G2.maximize(10, precision="fp32", L=6)
    rest, rg, _, _ = G2.maximize(6, precision="fp32", L=6, init=full[:4])
    assert list(rest) == list(full[4:])
    assert np.all(rel(rg, fg[4:]) < 1e-5)


def test_determinism(cuda_device):
    G = dev_graph("rmat15")
    a = G.maximize(8, precision="fp32", epsilon=1e-4)
    b = G.maximize(8, precision="fp32", epsilon=1e-4)
    assert list(a[0]) == list(b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    S = list(range(0, 3000, 37))
    assert G.score(S, precision="fp32", L=7)[0] == G.score(S, precision="fp32", L=7)[0]


# ------------------------------------------------------------------ batched scoring
@pytest.mark.parametrize("name", ["er1000", "ba5000", "rmat15"])
def test_score_batch(cuda_device, name):
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    off, mem = gg.random_groups(g.n, 70, 1, 100, 11)
    scores, L = G.score_batch(off, mem, epsilon=1e-4)
    for j in range(70):
        S = mem[off[j]:off[j + 1]]
        assert rel(scores[j], oracle.score(g, S, alpha, L)) < 1e-5, j
    # batch invariance: each column alone gives bitwise the same value
    for j in (0, 33, 69):
        one, _ = G.score_batch([0, off[j + 1] - off[j]], mem[off[j]:off[j + 1]], epsilon=1e-4)
        assert one[0] == scores[j]
    # empty groups and duplicate members
    s2, _ = G.score_batch([0, 0, 4], [5, 5, 6, 5], epsilon=1e-4)
    assert s2[0] == 0.0 and rel(s2[1], oracle.score(g, [5, 6], alpha, L)) < 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_maximize_past_the_positive_gains(cuda_device, prec):
    # 7 vertices have edges, 23 are isolated (caller ids 3, 4, 9..29). After 4 picks every gain is
    # exactly 0 (vertex 2's neighbours are both in S) and the picks go by increasing caller id,
    # isolated or not (the bound pass leaves the isolated rows to the host, which tracks the
    # smallest such id outside S)
    g = host_graph("isolated")
    G = dev_graph("isolated")
    alpha = oracle.default_alpha(g)
    grp, gains, score, L = G.maximize(12, precision=prec, epsilon=1e-4)
    ogrp, ogains, _ = oracle.greedy(g, 12, alpha, L, "all")
    check_sequence(grp, gains, TOL[prec], ogrp, ogains, *oracle_greedy_checker(oracle, g, alpha, L))
    assert list(grp[4:]) == [2, 3, 4, 6, 8, 9, 10, 11] and np.all(gains[4:] == 0.0)
    # resuming from a prefix that already holds isolated vertices skips them
    grp2, gains2, _, _ = G.maximize(3, precision=prec, epsilon=1e-4, init=[0, 1, 2, 5, 6, 7, 8, 3, 9])
    assert list(grp2) == [4, 10, 11] and np.all(gains2 == 0.0)


# ------------------------------------------------------------------ stochastic greedy (Appendix D)
@pytest.mark.parametrize("name,k,eta,seed", [("ba5000", 20, 0.1, 1), ("rmat14", 20, 0.2, 5), ("er1000", 8, 0.3, 9)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stochastic_maximize_matches_oracle(cuda_device, name, k, eta, seed, prec):
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    grp, gains, score, L = G.maximize(k, precision=prec, epsilon=1e-4, stochastic=True, eta=eta, seed=seed)
    ogrp, ogains, _ = oracle.greedy_stochastic(g, k, alpha, L, eta, seed)
    tol = TOL[prec]
    # sequences may part only at a tie inside the tolerance; the oracle then continues from the
    # GPU's own prefix with the same draws
    check_sequence(grp, gains, tol, ogrp, ogains,
                   *oracle_stochastic_checker(oracle, g, alpha, L, k, eta, seed))
    # every pick lies in its step's sample (the oracle's own draw)
    import math

    m = math.ceil(g.n / k * math.log(1.0 / eta))
    for j in range(k):
        p = m / (g.n - j)
        if p < 1.0:
            assert oracle.sample_hash(seed, j, int(grp[j])) < int(p * 2.0 ** 64)
    assert rel(score, oracle.score(g, grp, alpha, L)) < tol


# ------------------------------------------------------------------ lazy greedy with l-doubling (Algorithm 2)
@pytest.mark.parametrize("name,k,eps", [("er1000", 5, 1e-6), ("er1000", 12, 1e-4), ("ba5000", 20, 1e-4),
                                        ("rmat14", 16, 1e-4), ("star", 4, 1e-4), ("isolated", 6, 1e-3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adaptive_maximize_matches_oracle(cuda_device, name, k, eps, prec):
    # Identical picks, walk lengths and separation failures as long as no separation test of the
    # oracle lies within the tolerance of its threshold; after such a test only validity is checked.
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    sep = eps / k
    ref = oracle.greedy_adaptive(g, k, alpha, sep)
    grp, gains, score, L = G.maximize(k, precision=prec, epsilon=eps, adaptive=True)
    ell, fails = G.maximize_lengths()
    tol = TOL[prec]
    assert len(ell) == k and L == ell[-1]
    assert all(int(l) & (int(l) - 1) == 0 for l in ell) and np.all(np.diff(ell) >= 0)
    gu, gv, B = ref["att_gu"], ref["att_gv"], ref["att_B"]
    close = np.abs(gu - (gv + B - sep)) <= 10 * tol * np.maximum(np.maximum(gu, B), 1e-300)
    close &= gv >= 0
    upto = int(ref["att_step"][np.argmax(close)]) if close.any() else k  # steps decided far from the threshold
    for j in range(upto):
        assert ell[j] == ref["ell"][j], (j, list(ell), list(ref["ell"]))
        if grp[j] != ref["group"][j]:  # an exact tie of gains (symmetric vertices) may part the sequences
            assert abs(gains[j] - ref["gains"][j]) <= tol * max(ref["gains"][j], 1e-300), j
            upto = j
            break
        assert gains[j] == ref["gains"][j] == 0.0 or rel(gains[j], ref["gains"][j]) < tol, j
    if upto == k:
        n_fail = int(np.sum((gv >= 0) & ~(gu > gv + B - sep)))
        assert fails == n_fail
    # every pick is the exact gain of that vertex at its step's length
    for j in range(k):
        want = oracle.gain(g, list(grp[:j]), int(grp[j]), alpha, int(ell[j]))
        assert gains[j] == want == 0.0 or rel(gains[j], want) < tol, j
    L_fixed = oracle.select_L(g, alpha, sep)[0]
    assert rel(score, oracle.score(g, grp, alpha, L_fixed)) < tol
    assert ell[-1] < 2 * L_fixed


def test_adaptive_maximize_rejects_bad_combinations(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    G = dev_graph("er1000")
    for kw in ({"L": 8}, {"gains_all": True}, {"stochastic": True}):
        with pytest.raises(gedwalk.GedWalkError):
            G.maximize(3, adaptive=True, **kw)
    with pytest.raises(gedwalk.GedWalkError):
        G.maximize(3, adaptive=True, init=[1, 2])
    # the fixed-length run reports its L for every step
    grp, gains, score, L = G.maximize(3)
    ell, fails = G.maximize_lengths()
    assert list(ell) == [L] * 3 and fails == 0


# ------------------------------------------------------------------ lookahead sweeps (several steps per run)
@pytest.mark.parametrize("name,k", [("ba5000", 24), ("rmat14", 24), ("er1000", 10)])
@pytest.mark.parametrize("levels", [1, 3, 7])
def test_lookahead_levels_match_oracle(cuda_device, name, k, levels):
    # A lookahead run's rows hold phi^miss under S and, for each guess c_j, the walks through c_j
    # that avoid S + {c_1..c_{j-1}}; level d's phi^miss is their difference. Whatever the number of
    # levels, every pick is certified against the bounds of the current S.
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    grp, gains, score, L = G.maximize(k, precision="fp32", epsilon=1e-4, lookahead=int(levels))
    ogrp, ogains, _ = oracle.greedy(g, k, alpha, L, "lazy")
    # only a tie inside the tolerance may part the sequences; after one the oracle continues from
    # the GPU's own prefix
    check_sequence(grp, gains, 1e-5, ogrp, ogains, *oracle_greedy_checker(oracle, g, alpha, L))
    assert rel(score, oracle.score(g, grp, alpha, L)) < 1e-5
    st = G.maximize_stats()
    if levels != 1:  # steps whose winner was guessed run no sweep of their own
        assert st["sweeps"] < (k + 1) * L


@pytest.mark.parametrize("name,k,levels,prec,init", [
    ("ba5000", 24, 7, "fp32", ()), ("rmat14", 24, 3, "fp32", ()), ("er1000", 10, 3, "fp64", ()),
    ("rmat15", 40, 3, "fp64", ()), ("isolated", 12, 7, "fp32", ()), ("isolated", 3, 3, "fp64", (0, 1, 2, 5, 6)),
    ("star", 6, 7, "fp32", ()), ("path", 9, 3, "fp32", (4,))])
def test_device_loop_matches_host_loop(cuda_device, name, k, levels, prec, init):
    # The device-resident loop (conditional graph nodes) and the host-driven loop run the same
    # kernels on the same tables: identical picks, gains equal to the last bit, same counters.
    g = host_graph(name)
    G = dev_graph(name)
    alpha = oracle.default_alpha(g)
    kw = dict(precision=prec, epsilon=1e-4, lookahead=levels, init=list(init) or None)
    grp_h, gains_h, score_h, L_h = G.maximize(k, **kw)
    st_h = G.maximize_stats()
    grp_d, gains_d, score_d, L_d = G.maximize(k, device_loop=True, **kw)
    st_d = G.maximize_stats()
    assert L_h == L_d
    assert list(grp_d) == list(grp_h)
    assert np.array_equal(gains_d, gains_h)
    assert score_d == score_h
    assert st_d["evaluations"] == st_h["evaluations"] and st_d["spec_misses"] == st_h["spec_misses"]
    # and the oracle agrees with both (from the same init group)
    ini = [int(x) for x in init]
    ogrp, ogains, _ = oracle.greedy(g, k, alpha, L_d, "lazy", init=ini or None)

    def gain_of(prefix, v):
        return oracle.gain(g, ini + list(prefix), v, alpha, L_d)

    def continue_from(prefix, count):
        cg, cgains, _ = oracle.greedy(g, count, alpha, L_d, "lazy", init=ini + list(prefix))
        return cg, np.asarray(cgains)

    check_sequence(grp_d, gains_d, TOL[prec], ogrp, ogains, gain_of, continue_from)
    # the loop's graph is reused by the next call with the same configuration
    grp_r, gains_r, _, _ = G.maximize(k, device_loop=True, **kw)
    assert list(grp_r) == list(grp_d) and np.array_equal(gains_r, gains_d)


def _relabel_case(kind):
    # Graphs that take the device relabelling through one, two and three 8-bit radix passes
    # (d_max < 256, < 65536, >= 65536), with vertices of equal degree far apart, rows cut into
    # 1024-entry sorting pieces, and isolated vertices spread over the caller ids (their rows must
    # stay in increasing caller id, the order the zero-gain picks rely on).
    rng = np.random.default_rng({"one": 11, "two": 12, "three": 13}[kind])
    n = {"one": 5000, "two": 9000, "three": 85_000}[kind]
    hub_deg = {"one": 200, "two": 3000, "three": 70_000}[kind]
    iso = set(range(3, n, 7))
    live = [v for v in range(n) if v not in iso and v != 5]
    edges = set()
    for u in rng.choice(live, size=hub_deg, replace=False):  # hub 5
        edges.add((5, int(u)))
    a = rng.choice(live, size=2 * n)  # sparse random edges among the others
    b = rng.choice(live, size=2 * n)
    for x, y in zip(a.tolist(), b.tolist()):
        if x != y:
            edges.add((min(x, y), max(x, y)))
    return gg.from_edges(n, sorted(edges))


@pytest.mark.parametrize("kind", ["one", "two", "three"])
def test_device_relabel_radix_passes(cuda_device, kind):
    from paper_1910_13874_gb300 import gedwalk

    g = _relabel_case(kind)
    G = gedwalk.Graph.from_host(g)
    alpha = oracle.default_alpha(g)
    deg = np.diff(g.row_ptr)
    assert G.dmax == int(deg.max())
    S = np.array([5, 1, 2, 8, 13], dtype=np.int32)
    score, L, _ = G.score(S, precision="fp64", epsilon=1e-6)
    assert rel(score, oracle.score(g, S, alpha, L)) < 1e-12
    k = 6
    grp, gains, _, L = G.maximize(k, precision="fp64", epsilon=1e-4)
    ogrp, ogains, _ = oracle.greedy(g, k, alpha, L, "lazy")
    check_sequence(grp, gains, 1e-12, ogrp, ogains, *oracle_greedy_checker(oracle, g, alpha, L))
    # every isolated vertex has gain 0
    all_g, _ = G.gains([], precision="fp64", epsilon=1e-4)
    assert np.all(all_g[deg == 0] == 0.0)
    # with every vertex that has an edge in S, only isolated vertices are left: the picks are the
    # lowest caller ids among them (the isolated rows keep increasing caller ids)
    live = np.flatnonzero(deg > 0).astype(np.int32)
    grp2, gains2, _, _ = G.maximize(3, precision="fp32", epsilon=1e-4, init=live)
    assert list(grp2) == [int(x) for x in np.flatnonzero(deg == 0)[:3]] and np.all(gains2 == 0.0)
    G.free()
