"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

None of these compare the oracle with itself: brute-force walk enumeration, hand-derived
walk counts (tests/golden/hand_walks.txt), closed forms, Prop. katz-relation evaluated by
dense matrix powers, Prop. ged_submod, Lemma initialize, exhaustive optima and the
long-double build bound each routine from outside.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_walks.txt")


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _small_graphs():
    out = []
    for seed in range(8):
        n = 5 + seed % 5
        out.append(gg.random_graph_small(n, 0.45, seed))
    out += [gg.complete(5), gg.star(4), gg.path(6), gg.cycle(5)]
    return out


def _parse_golden():
    recs = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [x.strip() for x in line.split(";")]
        n = int(f[2])
        edges = [tuple(int(v) for v in e.split("-")) for e in f[3].split(",")]
        S = [int(v) for v in f[4].split(",")]
        if f[0] == "phi":
            recs.append(("phi", f[1], n, edges, S, None, [int(v) for v in f[5].split()]))
        else:
            recs.append(("gain", f[1], n, edges, S, int(f[5]), [int(v) for v in f[6].split()]))
    return recs


@pytest.mark.parametrize("rec", _parse_golden(), ids=lambda r: f"{r[0]}-{r[1]}-{r[4]}")
def test_hand_enumerated_counts(rec):
    kind, _, n, edges, S, x, want = rec
    g = gg.from_edges(n, edges)
    alpha = 0.5  # a power of two keeps alpha^i * count exact in binary floating point
    for i, w in enumerate(want, start=1):
        if kind == "phi":
            assert oracle.brute_phi(g, S, i)[0] == w
            _, terms = oracle.score(g, S, alpha, i, terms=True)
            assert terms[i] == alpha ** i * w
        else:
            assert oracle.brute_gain(g, S, x, i) == w
    if kind == "gain":
        L = len(want)
        assert oracle.gain(g, S, x, alpha, L) == sum(alpha ** i * w for i, w in enumerate(want, start=1))


@pytest.mark.parametrize("gi", range(12))
def test_two_state_recurrence_matches_brute_force(gi):
    g = _small_graphs()[gi]
    rng = np.random.default_rng(100 + gi)
    alpha = 0.5
    for _ in range(4):
        s = int(rng.integers(0, g.n + 1))
        S = sorted(rng.choice(g.n, size=s, replace=False).tolist())
        L = 5
        _, terms = oracle.score(g, S, alpha, L, terms=True)
        for i in range(1, L + 1):
            phi, _ = oracle.brute_phi(g, S, i)
            assert terms[i] == alpha ** i * phi, (S, i)


@pytest.mark.parametrize("n,s", [(4, 1), (6, 2), (7, 3), (9, 0), (9, 9)])
def test_complete_graph_closed_form(n, s):
    # walks avoiding S on K_n are exactly the walks of K_{n-s}: phi_i = n(n-1)^i - (n-s)(n-s-1)^i
    g = gg.complete(n)
    alpha = 0.125
    L = 6
    _, terms = oracle.score(g, list(range(s)), alpha, L, terms=True)
    for i in range(1, L + 1):
        want = n * (n - 1) ** i - (n - s) * max(n - s - 1, 0) ** i
        assert terms[i] == alpha ** i * want


def test_walk_total_closed_forms():
    L = 8
    # complete graph: n (n-1)^i
    _, Wa = oracle.walk_totals(gg.complete(6), 1.0, L)
    assert [round(w) for w in Wa[1:]] == [6 * 5 ** i for i in range(1, L + 1)]
    # star K_{1,m}: m^ceil(i/2) + m^(floor(i/2)+1)
    m = 5
    _, Wa = oracle.walk_totals(gg.star(m), 1.0, L)
    assert [round(w) for w in Wa[1:]] == [m ** math.ceil(i / 2) + m ** (i // 2 + 1) for i in range(1, L + 1)]
    # cycle C_n: n 2^i
    _, Wa = oracle.walk_totals(gg.cycle(7), 1.0, L)
    assert [round(w) for w in Wa[1:]] == [7 * 2 ** i for i in range(1, L + 1)]
    # path P_n: sum_k (1^T u_k)^2 (2 cos(k pi/(n+1)))^i with u_k the normalised sine eigenvectors
    n = 6
    _, Wa = oracle.walk_totals(gg.path(n), 1.0, L)
    j = np.arange(1, n + 1)
    for i in range(1, L + 1):
        tot = 0.0
        for k in range(1, n + 1):
            u = np.sin(j * k * np.pi / (n + 1)) * math.sqrt(2.0 / (n + 1))
            tot += u.sum() ** 2 * (2 * math.cos(k * math.pi / (n + 1))) ** i
        assert abs(Wa[i] - tot) < 1e-9 * max(1.0, tot)


@pytest.mark.parametrize("gi", range(12))
def test_katz_relation(gi):
    # Prop. katz-relation (1): GED(V) = sum_x KC(x); truncated at L both sides, with the Katz
    # terms alpha^i (A^i 1)(x) taken from dense integer matrix powers
    g = _small_graphs()[gi]
    A = g.to_dense()
    alpha = 1.0 / (1 + max(g.d_max, 1))
    L = 7
    katz = 0.0
    Ai = np.eye(g.n, dtype=np.int64)
    for i in range(1, L + 1):
        Ai = Ai @ A
        katz += alpha ** i * float(Ai.sum())
    ged = oracle.score(g, list(range(g.n)), alpha, L)
    assert _rel(ged, katz) < 1e-13


def test_two_forms_and_long_double_agree():
    g = gg.erdos_renyi(1000, 10, 1)
    alpha = oracle.default_alpha(g)
    L, _ = oracle.select_L(g, alpha, 1e-6)
    rng = np.random.default_rng(42)
    for _ in range(4):
        S = rng.choice(g.n, size=5, replace=False)
        a = oracle.score(g, S, alpha, L)
        b = oracle.score(g, S, alpha, L, long_double=True)
        c = oracle.score_by_complement(g, S, alpha, L)
        assert _rel(a, b) < 1e-13
        # the complement form cancels; its error is ~u * GED(V) / GED(S)
        gv = oracle.score(g, np.arange(g.n), alpha, L)
        assert abs(c - b) < 64 * 2.2e-16 * gv * L


@pytest.mark.parametrize("gi", range(12))
def test_gain_matches_brute_force_and_difference(gi):
    g = _small_graphs()[gi]
    rng = np.random.default_rng(7 + gi)
    alpha = 0.25
    L = 5
    for _ in range(3):
        s = int(rng.integers(0, g.n))
        S = sorted(rng.choice(g.n, size=s, replace=False).tolist())
        for x in range(g.n):
            want = sum(alpha ** i * oracle.brute_gain(g, S, x, i) for i in range(1, L + 1))
            got = oracle.gain(g, S, x, alpha, L)
            assert got == want or _rel(got, want) < 1e-14
            if x not in S:
                diff = oracle.score(g, S + [x], alpha, L) - oracle.score(g, S, alpha, L)
                assert abs(diff - got) <= 1e-13 * max(1.0, oracle.score(g, S + [x], alpha, L))
            else:
                assert got == 0.0


@pytest.mark.parametrize("seed", range(6))
def test_monotone_and_submodular(seed):
    # Prop. ged_submod on random triples S subset T, x outside T
    g = gg.erdos_renyi(40, 4, seed)
    alpha = oracle.default_alpha(g)
    L = 6
    rng = np.random.default_rng(seed)
    for _ in range(30):
        t = int(rng.integers(1, 10))
        T = rng.choice(g.n, size=t, replace=False).tolist()
        S = T[: int(rng.integers(0, t + 1))]
        rest = [v for v in range(g.n) if v not in T]
        x = int(rng.choice(rest))
        assert oracle.score(g, T, alpha, L) >= oracle.score(g, S, alpha, L) - 1e-15
        assert oracle.gain(g, S, x, alpha, L) >= oracle.gain(g, T, x, alpha, L) - 1e-15


@pytest.mark.parametrize("gi", range(12))
def test_upper_bound_lemma_initialize(gi):
    g = _small_graphs()[gi]
    alpha = 1.0 / (1 + g.d_max)
    rng = np.random.default_rng(gi)
    S = sorted(rng.choice(g.n, size=int(rng.integers(0, g.n // 2 + 1)), replace=False).tolist())
    for L in (1, 3, 6):
        ub = oracle.upper_bounds(g, S, alpha, L)
        for x in range(g.n):
            gx = oracle.gain(g, S, x, alpha, L)
            assert ub[x] >= gx * (1 - 1e-14)
            if L == 1:  # P_1 counts each 1-walk through x once when there are no self-loops
                assert abs(ub[x] - gx) <= 1e-15 * max(gx, 1e-300)
            if x in S:
                assert ub[x] == 0.0


def test_upper_bound_brute_multiplicity():
    # P_i counts walks through x weighted by the number of visits of x (proof of Lemma initialize)
    g = gg.random_graph_small(6, 0.6, 3)
    S = [0]
    alpha = 1.0
    for i in range(1, 5):
        ub_i = oracle.upper_bounds(g, S, alpha, i) - (oracle.upper_bounds(g, S, alpha, i - 1) if i > 1 else 0)
        inS = np.zeros(g.n, bool)
        inS[S] = True
        for x in range(g.n):
            if inS[x]:
                continue
            cnt = 0
            for walk in itertools.product(range(g.n), repeat=i + 1):
                if any(inS[v] for v in walk):
                    continue
                if all(walk[j + 1] in g.col_idx[g.row_ptr[walk[j]]:g.row_ptr[walk[j] + 1]] for j in range(i)):
                    cnt += walk.count(x)
            assert round(ub_i[x]) == cnt


@pytest.mark.parametrize("seed", range(4))
def test_tail_bound_holds(seed):
    # Eq. comb-bound: GED_{>l}(S) <= B_l; the true tail is taken from a long FP64 run
    g = gg.erdos_renyi(60, 5, seed)
    alpha = oracle.default_alpha(g)
    S = list(range(0, 60, 7))
    _, Wa = oracle.walk_totals(g, alpha, 12)
    full = oracle.score(g, S, alpha, 400)
    for l in range(1, 12):
        tail = full - oracle.score(g, S, alpha, l)
        assert tail <= oracle.comb_bound(g, alpha, Wa[l]) * (1 + 1e-12)
    # and the whole-graph tail equals sum_{i>l} alpha^i W_i, also below the bound
    fullV = oracle.score(g, list(range(60)), alpha, 400)
    for l in range(1, 12):
        tailV = fullV - oracle.score(g, list(range(60)), alpha, l)
        assert tailV <= oracle.comb_bound(g, alpha, Wa[l]) * (1 + 1e-12)


def test_select_L_is_first_crossing_and_monotone():
    g = gg.erdos_renyi(1000, 10, 1)
    alpha = oracle.default_alpha(g)
    _, Wa = oracle.walk_totals(g, alpha, 60)
    prev = 0
    for eps in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10):
        L, B = oracle.select_L(g, alpha, eps)
        assert L >= prev
        prev = L
        assert oracle.comb_bound(g, alpha, Wa[L]) < eps
        assert L == 1 or oracle.comb_bound(g, alpha, Wa[L - 1]) >= eps
    # alpha*dmax >= 1 voids the combinatorial bound
    assert oracle.select_L(g, 1.0 / g.d_max, 1e-4)[0] == -1


BOUND_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "comb_bound.txt")


def _cube3():
    return gg.from_edges(8, [(u, v) for u in range(8) for v in range(u + 1, 8) if bin(u ^ v).count("1") == 1])


def _petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    return gg.from_edges(10, outer + inner + spokes)


_NAMED = {"K4": lambda: gg.complete(4), "C5": lambda: gg.cycle(5), "star3": lambda: gg.star(3), "Q3": _cube3}


def _parse_bound_golden():
    recs = []
    for line in open(BOUND_GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [x.strip() for x in line.split(";")]
        recs.append(tuple(f))
    return recs


@pytest.mark.parametrize("rec", _parse_bound_golden(), ids=lambda r: "-".join(r[:4]))
def test_comb_bound_hand_values(rec):
    # Eq. comb-bound and Algorithm 1's stop test against values derived by hand
    # (tests/golden/comb_bound.txt): a dropped alpha, alpha^l for alpha^{l+1}, a wrong
    # d/(1 - alpha d), an average degree for d_max or an off-by-one in l all change them.
    from fractions import Fraction

    g = _NAMED[rec[1]]()
    alpha = float(Fraction(rec[2]))
    if rec[0] == "B":
        l, want = int(rec[3]), float(Fraction(rec[4]))
        _, Wa = oracle.walk_totals(g, alpha, l)
        assert _rel(oracle.comb_bound(g, alpha, Wa[l]), want) < 1e-14
    else:
        L, B = oracle.select_L(g, alpha, float(rec[3]))
        assert L == int(rec[4])
        assert _rel(B, float(Fraction(rec[5]))) < 1e-14


def _dense_tail(g, alpha, upto=4000):
    """alpha^i W_i for i = 1..upto from dense powers of the adjacency matrix (numpy)."""
    A = g.to_dense().astype(float)
    v, terms = np.ones(g.n), [0.0]
    for _ in range(upto):
        v = alpha * (A @ v)
        terms.append(float(v.sum()))
        if terms[-1] < 1e-30 * max(terms):
            break
    return np.array(terms)


@pytest.mark.parametrize("name,d", [("C7", 2), ("K6", 5), ("Q3", 3), ("petersen", 3)])
@pytest.mark.parametrize("frac", [None, 0.5, 0.9])
def test_comb_bound_is_tight_on_regular_graphs(name, d, frac):
    # On a d-regular graph W_{l+j} = d^j W_l, so the whole-graph tail sum_{i>l} alpha^i W_i equals
    # the bound of Eq. comb-bound exactly: the pin holds from both sides, not only tail <= B_l.
    g = {"C7": lambda: gg.cycle(7), "K6": lambda: gg.complete(6), "Q3": _cube3, "petersen": _petersen}[name]()
    assert oracle.dmax(g) == d and np.all(np.diff(g.row_ptr) == d)
    alpha = 1.0 / (d + 1) if frac is None else frac / d
    terms = _dense_tail(g, alpha)
    _, Wa = oracle.walk_totals(g, alpha, 8)
    for l in range(1, 9):
        tail = terms[l + 1:].sum()
        closed = g.n * (alpha * d) ** (l + 1) / (1.0 - alpha * d)  # geometric series of n (alpha d)^i
        assert _rel(tail, closed) < 1e-11
        assert _rel(oracle.comb_bound(g, alpha, Wa[l]), tail) < 1e-11
        # the oracle's own two-state score at S = V gives the same tail (GED_{>l}(V))
        if frac is None:
            fullV = oracle.score(g, list(range(g.n)), alpha, 600)
            partV = oracle.score(g, list(range(g.n)), alpha, l)
            assert _rel(fullV - partV, tail) < 1e-9
        # Lemma spectral-bound with sigma_max = d is sqrt(|V|) times the true tail
        assert _rel(oracle.spectral_bound(g, alpha, Wa[l], float(d)), math.sqrt(g.n) * tail) < 1e-11


@pytest.mark.parametrize("name,d", [("C7", 2), ("K6", 5), ("Q3", 3)])
@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-7])
def test_select_L_matches_closed_form_on_regular_graphs(name, d, eps):
    # L = min{l >= 1 : n (alpha d)^{l+1} / (1 - alpha d) < eps}, evaluated in exact rationals
    from fractions import Fraction

    g = {"C7": lambda: gg.cycle(7), "K6": lambda: gg.complete(6), "Q3": _cube3}[name]()
    a = Fraction(1, d + 1)
    e = Fraction(eps)
    l = 1
    while g.n * (a * d) ** (l + 1) / (1 - a * d) >= e:
        l += 1
    B = g.n * (a * d) ** (l + 1) / (1 - a * d)
    # the crossing is far from a rounding boundary at these parameters
    assert abs(float(B / e) - 1) > 1e-6 and abs(float(B / (a * d) / e) - 1) > 1e-6
    L, BL = oracle.select_L(g, float(a), eps)
    assert L == l
    assert _rel(BL, float(B)) < 1e-13


@pytest.mark.parametrize("kind,seed", [("er", 1), ("er", 2), ("ba", 3), ("ba", 4), ("rmat", 5)])
def test_greedy_all_vertex_equals_lazy(kind, seed):
    if kind == "er":
        g = gg.erdos_renyi(300, 6, seed)
    elif kind == "ba":
        g = gg.barabasi_albert(300, 3, seed)
    else:
        g = gg.rmat(9, 8, seed=seed)
    alpha = oracle.default_alpha(g)
    L = 6
    a = oracle.greedy(g, 8, alpha, L, "all")
    b = oracle.greedy(g, 8, alpha, L, "lazy")
    assert list(a[0]) == list(b[0])
    assert np.allclose(a[1], b[1], rtol=1e-14, atol=0)
    assert b[2] < a[2]  # the lazy mode evaluates fewer vertices


def test_greedy_gains_are_score_differences_and_resume():
    g = gg.erdos_renyi(200, 8, 3)
    alpha = oracle.default_alpha(g)
    L = 7
    grp, gains, _ = oracle.greedy(g, 6, alpha, L, "lazy")
    for j in range(6):
        d = oracle.score(g, grp[: j + 1], alpha, L) - oracle.score(g, grp[:j], alpha, L)
        assert _rel(gains[j], d) < 1e-12
    # resuming from a prefix reproduces the rest
    grp2, gains2, _ = oracle.greedy(g, 3, alpha, L, "lazy", init=grp[:3])
    assert list(grp2) == list(grp[3:])


@pytest.mark.parametrize("seed", range(5))
def test_greedy_against_exhaustive_optimum(seed):
    g = gg.random_graph_small(9, 0.35, 50 + seed)
    alpha = 1.0 / (1 + max(g.d_max, 1))
    L = 6
    for k in (1, 2, 3):
        grp, _, _ = oracle.greedy(g, k, alpha, L, "all")
        best = max(oracle.score(g, list(c), alpha, L) for c in itertools.combinations(range(g.n), k))
        got = oracle.score(g, list(grp), alpha, L)
        # Prop. greedy_approx applies to the truncated objective (itself monotone submodular)
        assert got >= (1 - 1 / math.e) * best - 1e-12
        if k == 1:
            assert abs(got - best) <= 1e-12 * best


def test_greedy_tie_break_lowest_id():
    # K_n: all gains tie exactly (alpha a power of two keeps the arithmetic exact)
    g = gg.complete(7)
    for mode in ("all", "lazy"):
        grp, _, _ = oracle.greedy(g, 4, 0.125, 4, mode)
        assert list(grp) == [0, 1, 2, 3]


def test_greedy_small_alpha_follows_group_degree():
    # Thm. hardness: for tiny alpha GED degrades to group degree, so every greedy pick covers the
    # largest number of still-uncovered edges (ties among those are settled by the alpha^2 terms)
    g = gg.erdos_renyi(50, 4, 9)
    alpha = 1.0 / (g.n ** 3 + g.n + 1)
    grp, _, _ = oracle.greedy(g, 6, alpha, 4, "all")
    A = g.to_dense().astype(bool)
    covered = np.zeros_like(A)
    for v in grp:
        new = lambda u: int((A[u] & ~covered[u]).sum())
        assert new(v) == max(new(u) for u in range(g.n) if u not in grp[: list(grp).index(v)])
        covered[v, :] = True
        covered[:, v] = True


def test_star_first_pick_is_centre():
    g = gg.star(9)
    grp, gains, _ = oracle.greedy(g, 2, 1.0 / 10, 5, "lazy")
    assert grp[0] == 0
    # with the centre in S every remaining gain is 0; the lowest id (leaf 1) follows
    assert grp[1] == 1 and gains[1] == 0.0


def test_empty_group_and_isolated_vertices():
    g = gg.from_edges(6, [(0, 1), (1, 2)])  # vertices 3,4,5 isolated
    alpha = 0.25
    assert oracle.score(g, [], alpha, 5) == 0.0
    assert oracle.score(g, [4], alpha, 5) == 0.0
    assert oracle.gain(g, [], 3, alpha, 5) == 0.0
    assert oracle.upper_bounds(g, [], alpha, 5)[3] == 0.0


# ---------------------------------------------------------------- stochastic greedy (Appendix D)
def test_sample_hash_is_splitmix64():
    # splitmix64 started from state 0 first outputs 0xE220A8397B1DCDAF (its published reference value)
    assert oracle.sample_hash(0, 0, 0) == 0xE220A8397B1DCDAF
    # the state is seed ^ (step << 32) ^ v: for a fixed seed every (step, v) gives its own draw,
    # and the draws of one step are uniform (mean of u/2^64 near 1/2)
    outs = {oracle.sample_hash(7, t, v) for t in range(4) for v in range(64)}
    assert len(outs) == 256
    u = np.array([oracle.sample_hash(7, 3, v) for v in range(4000)], dtype=np.float64) / 2.0 ** 64
    assert abs(u.mean() - 0.5) < 0.02 and abs((u < 0.25).mean() - 0.25) < 0.03


def _stochastic_threshold(n, k, step, eta):
    m = math.ceil(n / k * math.log(1.0 / eta))
    p = m / (n - step)
    return None if p >= 1.0 else int(p * 2.0 ** 64)


def test_stochastic_greedy_with_full_samples_is_greedy():
    # with (n/k) ln(1/eta) >= n every vertex is sampled and the algorithm is plain greedy
    g = gg.erdos_renyi(120, 6, 2)
    alpha = oracle.default_alpha(g)
    grp, gains, _ = oracle.greedy_stochastic(g, 4, alpha, 6, 1e-9, 3)
    full, fgains, _ = oracle.greedy(g, 4, alpha, 6, "all")
    assert list(grp) == list(full) and np.allclose(gains, fgains, rtol=1e-15, atol=0)


def test_stochastic_greedy_picks_the_best_sampled_vertex():
    g = gg.barabasi_albert(400, 3, 4)
    alpha = oracle.default_alpha(g)
    k, eta, seed, L = 8, 0.3, 11, 6
    grp, gains, evals = oracle.greedy_stochastic(g, k, alpha, L, eta, seed)
    S = []
    sizes = []
    for step in range(k):
        thr = _stochastic_threshold(g.n, k, step, eta)
        sample = [v for v in range(g.n) if v not in S and (thr is None or oracle.sample_hash(seed, step, v) < thr)]
        sizes.append(len(sample))
        assert int(grp[step]) in sample
        best = max(oracle.gain(g, S, v, alpha, L) for v in sample)
        assert gains[step] == best
        S.append(int(grp[step]))
    # the samples have about (n/k) ln(1/eta) members
    m = g.n / k * math.log(1 / eta)
    assert 0.6 * m < np.mean(sizes) < 1.4 * m
    assert evals == sum(sizes)


def test_stochastic_greedy_approximation_in_expectation():
    # E[f(S)] >= (1 - 1/e - eta) f(S*) (Appendix D); checked on the mean over seeds
    g = gg.random_graph_small(10, 0.4, 21)
    alpha = 1.0 / (1 + g.d_max)
    L, k, eta = 6, 3, 0.2
    best = max(oracle.score(g, list(c), alpha, L) for c in itertools.combinations(range(g.n), k))
    vals = [oracle.score(g, list(oracle.greedy_stochastic(g, k, alpha, L, eta, s)[0]), alpha, L) for s in range(40)]
    assert np.mean(vals) >= (1 - 1 / math.e - eta) * best


# ---------------------------------------------------------------- lazy greedy with l-doubling (Algorithm 2)
def _bound(g, alpha, l):
    _, Wa = oracle.walk_totals(g, alpha, l)
    return oracle.comb_bound(g, alpha, Wa[l])


def _all_gains(g, S, alpha, l):
    return np.array([oracle.gain(g, S, x, alpha, l) if x not in S else -np.inf for x in range(g.n)])


def _top2(gv):
    order = sorted(range(len(gv)), key=lambda x: (-gv[x], x))
    return order[0], (order[1] if len(order) > 1 and np.isfinite(gv[order[1]]) else None)


@pytest.mark.parametrize("kind,eps", [("er", 1e-4), ("er", 1e-2), ("ba", 1e-5), ("small", 1e-3)])
def test_adaptive_greedy_separation_and_doubling(kind, eps):
    # Every pick is the argmax of L_l(S, .) at the step's l and is eps/k-separated from the runner-up
    # (Def. separation with U_l = L_l + B_l); every smaller power of two that l passed through on
    # that step failed the test. Gains come from the independent per-vertex routine.
    g = {"er": lambda: gg.erdos_renyi(150, 6, 3), "ba": lambda: gg.barabasi_albert(200, 3, 4),
         "small": lambda: gg.random_graph_small(11, 0.4, 7)}[kind]()
    alpha = oracle.default_alpha(g)
    k = 6
    sep = eps / k
    r = oracle.greedy_adaptive(g, k, alpha, sep)
    ell = r["ell"]
    assert all(int(l) & (int(l) - 1) == 0 for l in ell) and np.all(np.diff(ell) >= 0)
    L_fixed = oracle.select_L(g, alpha, sep)[0]
    assert ell[-1] < 2 * L_fixed  # B_l < eps/k forces separation once l >= L(eps/k)
    prev = 1
    for j in range(k):
        S = list(r["group"][:j])
        # the levels tried and failed on this step
        l = prev
        while l < ell[j]:
            gv = _all_gains(g, S, alpha, l)
            u, v = _top2(gv)
            assert v is not None and gv[u] <= gv[v] + _bound(g, alpha, l) - sep + 1e-12 * gv[u]
            l *= 2
        gv = _all_gains(g, S, alpha, int(ell[j]))
        u, v = _top2(gv)
        assert abs(gv[u] - r["gains"][j]) <= 1e-12 * max(gv[u], 1e-300)
        assert abs(gv[r["group"][j]] - gv[u]) <= 1e-12 * max(gv[u], 1e-300)  # an argmax (ties: any)
        if v is not None:
            assert gv[r["group"][j]] > gv[v] + _bound(g, alpha, int(ell[j])) - sep - 1e-12 * gv[u]
        prev = int(ell[j])


def test_adaptive_greedy_additive_guarantee():
    # Separation at eps/k makes each pick's true gain within eps/k of the best true gain
    # (Prop. additive-greedy); "true" here is a truncation far beyond the bound.
    g = gg.erdos_renyi(120, 5, 11)
    alpha = oracle.default_alpha(g)
    k, eps = 5, 1e-3
    r = oracle.greedy_adaptive(g, k, alpha, eps / k)
    Lbig = 120
    for j in range(k):
        S = list(r["group"][:j])
        gv = _all_gains(g, S, alpha, Lbig)
        assert gv[r["group"][j]] >= gv[np.isfinite(gv)].max() - eps / k


def test_adaptive_greedy_at_l1_is_remaining_degree_greedy():
    # With eps/k above B_1 the separation test always passes at l = 1, where L_1(S, x) counts the
    # two orientations of every edge from x to V \ S: 2 alpha |N(x) \ S|. So the picks follow the
    # largest remaining degree (lowest id among equals), computed here from the adjacency matrix.
    g = gg.erdos_renyi(80, 6, 5)
    alpha = oracle.default_alpha(g)
    k = 8
    sep = 2 * _bound(g, alpha, 1)
    r = oracle.greedy_adaptive(g, k, alpha, sep)
    assert list(r["ell"]) == [1] * k
    A = g.to_dense().astype(bool)
    S = []
    for j in range(k):
        rem = np.ones(g.n, dtype=bool)
        rem[S] = False
        deg = np.where(rem, (A & rem[None, :]).sum(axis=1), -1)
        want = int(np.argmax(deg))
        assert r["group"][j] == want
        assert abs(r["gains"][j] - 2 * alpha * deg[want]) <= 1e-14
        S.append(want)


@pytest.mark.parametrize("seed", range(4))
def test_adaptive_greedy_against_exhaustive_optimum(seed):
    # (1 - 1/e) OPT - eps for the untruncated objective (Lemma after Algorithm 2); OPT by exhaustion
    g = gg.random_graph_small(9, 0.35, 70 + seed)
    alpha = oracle.default_alpha(g)
    Lbig, eps = 80, 1e-3
    for k in (1, 2, 3):
        r = oracle.greedy_adaptive(g, k, alpha, eps / k)
        best = max(oracle.score(g, list(c), alpha, Lbig) for c in itertools.combinations(range(g.n), k))
        assert oracle.score(g, list(r["group"]), alpha, Lbig) >= (1 - 1 / math.e) * best - eps


def test_adaptive_greedy_records_and_star():
    g = gg.star(9)
    alpha = 1.0 / 10
    r = oracle.greedy_adaptive(g, 3, alpha, 1e-4)
    assert r["group"][0] == 0  # the centre first
    # after the centre joins, every gain is 0: no l separates 0 from 0 until B_l < eps, so l grows
    assert r["gains"][1] == 0.0 and _bound(g, alpha, int(r["ell"][1])) < 1e-4
    # each failed test is followed by a test of the same step at twice the length
    st, el, gu, gv, B = r["att_step"], r["att_ell"], r["att_gu"], r["att_gv"], r["att_B"]
    for i in range(len(st)):
        sep_ok = gv[i] < 0 or gu[i] > gv[i] + B[i] - 1e-4
        if not sep_ok:
            assert st[i + 1] == st[i] and el[i + 1] == 2 * el[i]
        elif i + 1 < len(st):
            assert st[i + 1] == st[i] + 1 and el[i + 1] == el[i]


def test_adaptive_greedy_rejects_bad_input():
    g = gg.complete(5)
    with pytest.raises(ValueError):
        oracle.greedy_adaptive(g, 2, 0.3, 1e-3)  # alpha * d_max >= 1: no bound
    with pytest.raises(ValueError):
        oracle.greedy_adaptive(g, 2, 0.1, 1e-30, lcap=4)  # l would pass the cap


# ---------------------------------------------------------------- weighted walks (Section 5.4)
def _scaled_weights(g, scale):
    """w(v, u) = scale[v] * scale[u] per CSR entry (input construction for the weighted tests)."""
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return np.asarray(scale, dtype=np.float64)[rows] * np.asarray(scale, dtype=np.float64)[g.col_idx]


def _weighted_dense(g, w):
    M = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    M[rows, g.col_idx] = w
    return M


def test_normalized_weights_are_sym_normalised_adjacency():
    g = gg.erdos_renyi(40, 5, 3)
    A = g.to_dense().astype(float)
    d = A.sum(axis=1)
    with np.errstate(divide="ignore"):
        Dm = np.where(d > 0, 1.0 / np.sqrt(d), 0.0)
    N = Dm[:, None] * A * Dm[None, :]
    assert np.allclose(_weighted_dense(g, oracle.normalized_weights(g)), N, rtol=1e-15, atol=0)


@pytest.mark.parametrize("g", [gg.cycle(7), gg.complete(6)], ids=["cycle7", "k6"])
def test_weighted_regular_graph_rescales_alpha(g):
    # On a d-regular graph D^{-1/2} A D^{-1/2} = A / d: every i-walk weighs d^{-i}, so the weighted
    # objective at alpha is the unweighted one at alpha / d.
    d = g.d_max
    w = oracle.normalized_weights(g)
    alpha, L = 0.3, 7
    for S in ([0], [1, 3], [0, 2, 4]):
        assert _rel(oracle.score(g, S, alpha, L, w=w), oracle.score(g, S, alpha / d, L)) < 1e-14
        assert _rel(oracle.gain(g, S, 5, alpha, L, w=w), oracle.gain(g, S, 5, alpha / d, L)) < 1e-14
    _, Wa_w = oracle.walk_totals(g, alpha, L, w=w)
    _, Wa = oracle.walk_totals(g, alpha / d, L)
    assert np.allclose(Wa_w, Wa, rtol=1e-14, atol=0)


def _brute_weighted(g, S, wmat, i, x=None):
    """Sum over i-walks (exhaustive) of the product of their edge weights: the walks that contain a
    vertex of S, or (x given) the walks that avoid S and visit x."""
    from fractions import Fraction

    A = g.to_dense().astype(bool)
    Sset = set(S)
    tot = Fraction(0)
    for walk in itertools.product(range(g.n), repeat=i + 1):
        if not all(A[walk[j], walk[j + 1]] for j in range(i)):
            continue
        if x is None and not (Sset & set(walk)):
            continue
        if x is not None and (Sset & set(walk) or x not in walk):
            continue
        p = Fraction(1)
        for j in range(i):
            p *= wmat[walk[j]][walk[j + 1]]
        tot += p
    return tot


@pytest.mark.parametrize("gi", range(4))
def test_weighted_score_and_gain_match_brute_force(gi):
    from fractions import Fraction

    g = gg.random_graph_small(6 + gi % 2, 0.5, 30 + gi)
    rng = np.random.default_rng(gi)
    num = rng.integers(1, 9, size=g.n)
    scale = [Fraction(int(a), 8) for a in num]  # rational scales keep the brute force exact
    wmat = [[scale[v] * scale[u] for u in range(g.n)] for v in range(g.n)]
    w = _scaled_weights(g, [float(s) for s in scale])
    alpha = Fraction(1, 5)
    S = [0, g.n - 1]
    L = 4
    val, terms = oracle.score(g, S, float(alpha), L, terms=True, w=w)
    for i in range(1, L + 1):
        want = float(alpha ** i * _brute_weighted(g, S, wmat, i))
        assert abs(terms[i] - want) <= 1e-14 * max(want, 1e-300), i
    x = 2
    want = float(sum(alpha ** i * _brute_weighted(g, S, wmat, i, x) for i in range(1, L + 1)))
    assert abs(oracle.gain(g, S, x, float(alpha), L, w=w) - want) <= 1e-14 * max(want, 1e-300)
    # the complement form and the two-state form agree with weights as well
    assert _rel(oracle.score_by_complement(g, S, float(alpha), L, w=w), val) < 1e-12


def test_weighted_katz_relation_and_tail_bound():
    # GED(V) = sum_i alpha^i 1^T N^i 1 (Prop. katz-relation with weights) by dense powers, and the
    # weighted combinatorial bound with delta = max weighted degree covers the true tail.
    g = gg.barabasi_albert(60, 3, 5)
    w = oracle.normalized_weights(g)
    N = _weighted_dense(g, w)
    delta = N.sum(axis=1).max()
    assert abs(oracle.delta(g, w) - delta) <= 1e-14 * delta
    alpha = 0.9 / delta
    one = np.ones(g.n)
    Ls = 12
    katz, v = [], one.copy()
    for i in range(1, 400):
        v = N @ v
        katz.append(alpha ** i * v.sum())
    assert _rel(oracle.score(g, list(range(g.n)), alpha, Ls, w=w), sum(katz[:Ls])) < 1e-12
    _, Wa = oracle.walk_totals(g, alpha, Ls, w=w)
    for l in range(1, Ls):
        assert sum(katz[l:]) <= oracle.comb_bound(g, alpha, Wa[l], w=w) * (1 + 1e-12)
    L, B = oracle.select_L(g, alpha, 1e-3, w=w)
    assert B < 1e-3 and oracle.comb_bound(g, alpha, Wa[L - 1], w=w) >= 1e-3


def test_weighted_bounds_submodularity_and_greedy():
    g = gg.erdos_renyi(60, 5, 8)
    w = oracle.normalized_weights(g)
    alpha = oracle.default_alpha(g, w)
    L = 6
    S = [1, 7, 20]
    ub = oracle.upper_bounds(g, S, alpha, L, w=w)
    ub1 = oracle.upper_bounds(g, S, alpha, 1, w=w)
    for x in range(0, g.n, 3):
        gx = oracle.gain(g, S, x, alpha, L, w=w)
        assert gx <= ub[x] * (1 + 1e-12)
        assert abs(oracle.gain(g, S, x, alpha, 1, w=w) - ub1[x]) <= 1e-15  # Lemma initialize, L = 1
        assert gx <= oracle.gain(g, S[:1], x, alpha, L, w=w) * (1 + 1e-12) or x in S  # submodular
    grp_a, gains_a, _ = oracle.greedy(g, 5, alpha, L, "all", w=w)
    grp_l, gains_l, _ = oracle.greedy(g, 5, alpha, L, "lazy", w=w)
    assert list(grp_a) == list(grp_l) and np.allclose(gains_a, gains_l, rtol=1e-12)
    r = oracle.greedy_adaptive(g, 3, alpha, 1e-4, w=w)
    assert r["group"][0] == grp_a[0]


# ---------------------------------------------------------------- directed graphs (Section 2; Lemma initialize's psi)
def _digraph(seed, n=7, p=0.35):
    return gg.random_digraph(n, p, seed)


def _transposed_graph(g):
    rpt, cit, _ = oracle.transpose(g)
    return gg.Graph(rpt, cit)


@pytest.mark.parametrize("seed", range(4))
def test_directed_score_and_gain_match_brute_force(seed):
    # the CSR rows are successor lists; the brute force follows them, so both count directed walks
    g = _digraph(seed)
    alpha = 0.2
    S = [0, 3]
    val, terms = oracle.score(g, S, alpha, 5, terms=True)
    for i in range(1, 6):
        phi, _ = oracle.brute_phi(g, S, i)
        assert abs(terms[i] - alpha ** i * phi) <= 1e-14 * max(terms[i], 1e-300)
    for x in (1, 4, 6):
        want = sum(alpha ** i * oracle.brute_gain(g, S, x, i) for i in range(1, 6))
        assert abs(oracle.gain(g, S, x, alpha, 5) - want) <= 1e-14 * max(want, 1e-300)
    # reversing every walk is a bijection that keeps its vertex set: GED is the same on the reverse graph
    gt = _transposed_graph(g)
    assert _rel(oracle.score(gt, S, alpha, 5), val) < 1e-14


def _brute_psi_phi(g, S, x, i):
    """(S-avoiding i-walks ending at x, S-avoiding i-walks starting at x), by enumeration."""
    A = g.to_dense().astype(bool)
    end = start = 0
    for walk in itertools.product(range(g.n), repeat=i + 1):
        if any(v in S for v in walk) or not all(A[walk[j], walk[j + 1]] for j in range(i)):
            continue
        end += walk[-1] == x
        start += walk[0] == x
    return end, start


@pytest.mark.parametrize("seed", range(3))
def test_directed_upper_bound_uses_walks_from_and_to_x(seed):
    # Lemma initialize on a digraph: P_i = sum_j phi^miss_{i-j}(x) psi^miss_j(x), phi ending at x and
    # psi starting at x. Built here from enumerated counts; the oracle must take psi from the reverse.
    g = _digraph(10 + seed)
    alpha, L = 0.25, 4
    S = [2]
    ub = oracle.upper_bounds(g, S, alpha, L, directed=True)
    for x in range(g.n):
        if x in S:
            assert ub[x] == 0.0
            continue
        cnt = [_brute_psi_phi(g, S, x, i) for i in range(L + 1)]
        want = sum(alpha ** i * sum(cnt[i - j][1] * cnt[j][0] for j in range(i + 1)) for i in range(1, L + 1))
        # orientation: the oracle's rows are successor lists, so its phi^miss counts walks that
        # start at x and psi those that end there; the product is symmetric in the two
        assert abs(ub[x] - want) <= 1e-13 * max(want, 1e-300), x
        gain = oracle.gain(g, S, x, alpha, L)
        assert gain <= ub[x] * (1 + 1e-12)
    ub1 = oracle.upper_bounds(g, S, alpha, 1, directed=True)
    for x in range(g.n):
        assert abs(oracle.gain(g, S, x, alpha, 1) - ub1[x]) <= 1e-15  # P_1 is exact without self-loops


def test_directed_greedy_all_equals_lazy_and_adaptive_separates():
    g = gg.rmat(8, 8, seed=5, directed=True)
    alpha = oracle.default_alpha(g, directed=True)
    L = 6
    a, ga, _ = oracle.greedy(g, 6, alpha, L, "all")
    b, gb, _ = oracle.greedy(g, 6, alpha, L, "lazy", directed=True)
    assert list(a) == list(b) and np.allclose(ga, gb, rtol=1e-12)
    k, eps = 4, 1e-3
    r = oracle.greedy_adaptive(g, k, alpha, eps / k, directed=True)
    for j in range(k):
        S = list(r["group"][:j])
        gv = _all_gains(g, S, alpha, int(r["ell"][j]))
        u, v = _top2(gv)
        assert abs(gv[r["group"][j]] - gv[u]) <= 1e-12 * gv[u]
        assert gv[u] > gv[v] + oracle.comb_bound(g, alpha, oracle.walk_totals(g, alpha, int(r["ell"][j]))[1][-1],
                                                  directed=True) - eps / k - 1e-12 * gv[u]


def test_directed_delta_and_tail_bound():
    # out-star: the centre has out-degree n-1 but every in-degree is <= 1, so walks cannot grow
    g = gg.from_arcs(6, [(0, v) for v in range(1, 6)])
    assert oracle.delta(g, directed=True) == 1.0 and oracle.delta(g) == 5.0
    # random digraph: the bound with delta = min(max in, max out) covers the true tail (dense powers)
    g = gg.rmat(7, 8, seed=9, directed=True)
    A = g.to_dense().astype(float)
    d = min(A.sum(axis=0).max(), A.sum(axis=1).max())
    assert oracle.delta(g, directed=True) == d
    alpha = 0.95 / d
    terms, v = [], np.ones(g.n)
    for i in range(1, 600):
        v = alpha * (A @ v)  # alpha-scaled, so that nothing overflows
        terms.append(v.sum())
    _, Wa = oracle.walk_totals(g, alpha, 10)
    for l in range(1, 10):
        assert sum(terms[l:]) <= oracle.comb_bound(g, alpha, Wa[l], directed=True) * (1 + 1e-12)


# ---------------------------------------------------------------- spectral bound (Lemma spectral-bound, Appendix E)
@pytest.mark.parametrize("kind", ["ba", "er", "digraph"])
def test_spectral_bound_covers_the_tail_up_to_one_over_sigma(kind):
    # sigma_max from a dense SVD; alpha = delta / sigma_max up to 0.9, beyond the reach of the
    # combinatorial bound (alpha < 1/d_max) on these graphs
    g = {"ba": lambda: gg.barabasi_albert(80, 3, 2), "er": lambda: gg.erdos_renyi(70, 6, 4),
         "digraph": lambda: gg.rmat(6, 6, seed=2, directed=True)}[kind]()
    A = g.to_dense().astype(float)
    sigma = np.linalg.norm(A, 2)
    assert sigma <= oracle.dmax(g)
    for delta in (0.3, 0.6, 0.9):
        alpha = delta / sigma
        terms, v = [], np.ones(g.n)
        for i in range(1, 3000):
            v = alpha * (A @ v)
            terms.append(v.sum())
        _, Wa = oracle.walk_totals(g, alpha, 30)
        for l in range(1, 30):
            assert sum(terms[l:]) <= oracle.spectral_bound(g, alpha, Wa[l], sigma) * (1 + 1e-12)
        L, B = oracle.select_L_spectral(g, alpha, 1e-4, sigma)
        _, WaL = oracle.walk_totals(g, alpha, L)
        assert B < 1e-4 and oracle.spectral_bound(g, alpha, WaL[L - 1], sigma) >= 1e-4 and sum(terms[L:]) < 1e-4


def test_spectral_bound_on_regular_graph_is_sqrt_n_times_combinatorial():
    # d-regular: sigma_max = d, so the two bounds differ exactly by the factor sqrt(|V|)
    g = gg.cycle(9)
    alpha = 0.2
    _, Wa = oracle.walk_totals(g, alpha, 6)
    for l in range(1, 7):
        assert _rel(oracle.spectral_bound(g, alpha, Wa[l], 2.0), 3.0 * oracle.comb_bound(g, alpha, Wa[l])) < 1e-15
    assert oracle.select_L_spectral(g, 0.6, 1e-3, 2.0)[0] == -1  # alpha * sigma >= 1: no bound


# ---------------------------------------------------------------- threads
def test_threads_leave_every_result_bitwise_unchanged():
    # The row loops may run on several threads; each row's sum keeps its order and every sum over
    # vertices stays serial, so the results are bitwise those of one thread.
    g = gg.rmat(15, 8, seed=9)  # more rows than the parallel threshold
    alpha = oracle.default_alpha(g)
    S = list(range(0, 3000, 37))
    out = {}
    for t in (1, 4):
        oracle.set_threads(t)
        out[t] = (oracle.score(g, S, alpha, 7, terms=True)[1].tolist(),
                  oracle.score(g, S, alpha, 7, long_double=True),
                  oracle.walk_totals(g, alpha, 6)[1].tolist(),
                  oracle.upper_bounds(g, S, alpha, 6).tolist(),
                  [oracle.gain(g, S, x, alpha, 6) for x in (1, 5, 4000)],
                  [list(a) for a in oracle.greedy(g, 4, alpha, 6, "lazy")[:2]])
    oracle.set_threads(1)
    assert out[1] == out[4]
