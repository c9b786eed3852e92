"""GED-Walk CPU oracle: a ctypes front-end to oracle.c (double and long double).

TEST INFRASTRUCTURE ONLY. The oracle restates the paper's definitions in plain, slow
C so that the CUDA library can be checked against it. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it; the
library never does, and the oracle never imports the library.

Graphs are any object with ``row_ptr`` (int32[n+1]) and ``col_idx`` (int32[nnz]) numpy
arrays describing an undirected CSR. Every routine cites the passage it follows in
oracle_impl.inc / oracle.c.

Parity status: every routine here is pinned by tests/test_oracle.py (brute force,
closed forms, propositions, long-double agreement); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle_impl.inc")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no vendor code, portable to x86 and Arm).

    With OpenMP where gcc has it: the row loops may then run on several threads (set_threads),
    with bitwise the same results; without it the build is single-threaded.
    """
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRCS[0], "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            G = [ctypes.c_int32, _i32p, _i32p]
            GW = G + [_f64p]  # graph with optional entry weights (NULL: unweighted)
            lib.orc_set_threads.restype = None
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_threads.argtypes = []
            lib.orc_set_threads(1)  # single-threaded unless asked: test runs stay light
            lib.orc_dmax.restype = ctypes.c_int32
            lib.orc_dmax.argtypes = [ctypes.c_int32, _i32p]
            lib.orc_walk_totals_d.restype = ctypes.c_int
            lib.orc_walk_totals_d.argtypes = GW + [ctypes.c_double, ctypes.c_int32, _f64p, _f64p]
            lib.orc_select_L_d.restype = ctypes.c_int32
            lib.orc_select_L_d.argtypes = GW + [_i32p, _f64p, ctypes.c_double, ctypes.c_double, ctypes.c_int32, _f64p]
            lib.orc_comb_bound_d.restype = ctypes.c_double
            lib.orc_comb_bound_d.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.orc_spectral_bound_d.restype = ctypes.c_double
            lib.orc_spectral_bound_d.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.orc_select_L_spectral_d.restype = ctypes.c_int32
            lib.orc_select_L_spectral_d.argtypes = GW + [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                         ctypes.c_int32, _f64p]
            lib.orc_delta.restype = ctypes.c_double
            lib.orc_delta.argtypes = [ctypes.c_int32, _i32p, _f64p]
            lib.orc_delta2.restype = ctypes.c_double
            lib.orc_delta2.argtypes = [ctypes.c_int32, _i32p, _f64p, _i32p, _f64p]
            lib.orc_transpose.restype = None
            lib.orc_transpose.argtypes = G + [_f64p, _i32p, _i32p, _f64p]
            lib.orc_normalized_weights.restype = None
            lib.orc_normalized_weights.argtypes = G + [_f64p]
            lib.orc_score_d.restype = ctypes.c_double
            lib.orc_score_d.argtypes = GW + [_i32p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _f64p]
            lib.orc_score_ld_as_d.restype = ctypes.c_double
            lib.orc_score_ld_as_d.argtypes = GW + [_i32p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32]
            lib.orc_score_by_complement_d.restype = ctypes.c_double
            lib.orc_score_by_complement_d.argtypes = GW + [_i32p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32]
            lib.orc_gain_d.restype = ctypes.c_double
            lib.orc_gain_d.argtypes = GW + [_i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32]
            lib.orc_gain_ld_as_d.restype = ctypes.c_double
            lib.orc_gain_ld_as_d.argtypes = GW + [_i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                 ctypes.c_int32]
            lib.orc_upper_bounds_d.restype = ctypes.c_int
            lib.orc_upper_bounds_d.argtypes = GW + [_i32p, _i32p, _f64p, _i32p, ctypes.c_int32, ctypes.c_double,
                                                   ctypes.c_int32, _f64p]
            lib.orc_greedy_d.restype = ctypes.c_int
            lib.orc_greedy_d.argtypes = GW + [_i32p, _i32p, _f64p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                             _i32p, ctypes.c_int32, _i32p, _f64p, _i64p]
            lib.orc_greedy_stochastic_d.restype = ctypes.c_int
            lib.orc_greedy_stochastic_d.argtypes = GW + [ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                                        ctypes.c_double, ctypes.c_uint64, _i32p, _f64p, _i64p]
            lib.orc_greedy_adaptive_d.restype = ctypes.c_int
            lib.orc_greedy_adaptive_d.argtypes = GW + [_i32p, _i32p, _f64p, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_int32, _i32p, _f64p, _i32p, _i64p, ctypes.c_int32,
                                                      _i32p, _i32p, _f64p, _f64p, _f64p, _i32p]
            lib.orc_sample_hash.restype = ctypes.c_uint64
            lib.orc_sample_hash.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
            lib.orc_brute_phi.restype = ctypes.c_int
            lib.orc_brute_phi.argtypes = G + [_i32p, ctypes.c_int32, ctypes.c_int32, _u64p, _u64p]
            lib.orc_brute_gain.restype = ctypes.c_int
            lib.orc_brute_gain.argtypes = G + [_i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _u64p]
            _lib = lib
    return _lib


def _g(graph):
    rp = np.ascontiguousarray(graph.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(graph.col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    return rp.shape[0] - 1, rp, ci


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _wp(graph, w):
    """Entry weights (float64[nnz], Section 5.4's weighted walks) as a pointer; None: unweighted."""
    if w is None:
        return None
    w = np.ascontiguousarray(w, dtype=np.float64)
    if w.shape != (int(np.asarray(graph.col_idx).shape[0]),):
        raise ValueError("weights must hold one value per CSR entry")
    return w.ctypes.data_as(_f64p)  # the pointer keeps the array alive


def _S(S):
    s = np.ascontiguousarray(np.asarray(S if S is not None else [], dtype=np.int32).ravel())
    if s.size == 0:
        return np.zeros(1, dtype=np.int32), 0
    return s, int(s.size)


def set_threads(t: int) -> None:
    """Threads for the oracle's row loops (OpenMP builds). Results are bitwise the same for any t."""
    _load().orc_set_threads(int(t))


def threads() -> int:
    """Threads the row loops use now (1 for a build without OpenMP)."""
    return int(_load().orc_threads())


def dmax(graph) -> int:
    n, rp, _ = _g(graph)
    return int(_load().orc_dmax(n, _ptr(rp, _i32p)))


def transpose(graph, w=None):
    """(row_ptr, col_idx, weights or None) of the transposed CSR (the reverse graph)."""
    n, rp, ci = _g(graph)
    nnz = int(np.asarray(graph.col_idx).shape[0])
    rpt = np.zeros(n + 1, dtype=np.int32)
    cit = np.zeros(max(nnz, 1), dtype=np.int32)
    wt = np.zeros(max(nnz, 1), dtype=np.float64) if w is not None else None
    _load().orc_transpose(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), _ptr(rpt, _i32p), _ptr(cit, _i32p),
                          None if wt is None else _ptr(wt, _f64p))
    return rpt, cit[:nnz], (None if wt is None else wt[:nnz])


def _tp(graph, w, directed):
    """Pointers to the transposed CSR for a directed graph (psi of Lemma initialize), else NULLs."""
    if not directed:
        return None, None, None
    rpt, cit, wt = transpose(graph, w)
    if cit.size == 0:
        cit = np.zeros(1, dtype=np.int32)
    return _ptr(rpt, _i32p), _ptr(cit, _i32p), (None if wt is None else _ptr(wt, _f64p))


def delta(graph, w=None, directed: bool = False) -> float:
    """The degree bound of Eq. comb-bound: d_max (min of the largest in- and out-degree for a
    directed graph), or the largest weighted degree with weights."""
    n, rp, _ = _g(graph)
    rpt, _, wt = _tp(graph, w, directed)
    return float(_load().orc_delta2(n, _ptr(rp, _i32p), _wp(graph, w), rpt, wt))


def default_alpha(graph, w=None, directed: bool = False) -> float:
    """alpha = 1/(1 + delta): below 1/delta, as the combinatorial bound requires (Sec. 3.1.2)."""
    return 1.0 / (1.0 + delta(graph, w, directed))


def normalized_weights(graph) -> np.ndarray:
    """Entry weights of D^{-1/2} A D^{-1/2} (Section 5.4), one per CSR entry."""
    n, rp, ci = _g(graph)
    out = np.zeros(max(int(np.asarray(graph.col_idx).shape[0]), 1), dtype=np.float64)
    _load().orc_normalized_weights(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _ptr(out, _f64p))
    return out[:int(np.asarray(graph.col_idx).shape[0])]


def walk_totals(graph, alpha: float, L: int, w=None):
    """(t, Wa): t[r, x] = alpha^r omega_r(x) (Eq. katz-def terms), Wa[r] = alpha^r W_r."""
    n, rp, ci = _g(graph)
    t = np.zeros((L + 1, max(n, 1)), dtype=np.float64)
    Wa = np.zeros(L + 1, dtype=np.float64)
    rc = _load().orc_walk_totals_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), alpha, L, _ptr(t, _f64p), _ptr(Wa, _f64p))
    if rc != 0:
        raise MemoryError("oracle walk_totals failed")
    return t[:, :n], Wa


def comb_bound(graph, alpha: float, Wa_l: float, w=None, directed: bool = False) -> float:
    """B_l of Eq. comb-bound from Wa_l = alpha^l W_l."""
    return float(_load().orc_comb_bound_d(delta(graph, w, directed), alpha, Wa_l))


def select_L(graph, alpha: float, eps: float, Lcap: int = 400, w=None, directed: bool = False):
    """(L, B_L): smallest l >= 1 with B_l < eps (Algorithm 1 stop test). L = -1 if none."""
    n, rp, ci = _g(graph)
    B = ctypes.c_double(float("nan"))
    rpt, _, wt = _tp(graph, w, directed)
    L = _load().orc_select_L_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), rpt, wt, alpha, eps, Lcap,
                               ctypes.byref(B))
    return int(L), float(B.value)


def spectral_bound(graph, alpha: float, Wa_l: float, sigma: float) -> float:
    """B_l of Lemma spectral-bound from Wa_l = alpha^l W_l and sigma >= sigma_max."""
    n = int(np.asarray(graph.row_ptr).shape[0] - 1)
    return float(_load().orc_spectral_bound_d(n, sigma, alpha, Wa_l))


def select_L_spectral(graph, alpha: float, eps: float, sigma: float, Lcap: int = 4000, w=None):
    """(L, B_L) of Algorithm 1's stop test with the spectral bound. L = -1 if none."""
    n, rp, ci = _g(graph)
    B = ctypes.c_double(float("nan"))
    L = _load().orc_select_L_spectral_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), sigma, alpha, eps, Lcap,
                                        ctypes.byref(B))
    return int(L), float(B.value)


def score(graph, S, alpha: float, L: int, terms: bool = False, long_double: bool = False, w=None):
    """GED_{<=L}(S) by the two-state recurrences (Sec. 3.1.1). terms=True also returns alpha^i phi_i."""
    n, rp, ci = _g(graph)
    s, sl = _S(S)
    lib = _load()
    if long_double:
        return float(lib.orc_score_ld_as_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), _ptr(s, _i32p), sl, alpha, L))
    tv = np.zeros(L + 1, dtype=np.float64)
    val = float(lib.orc_score_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), _ptr(s, _i32p), sl, alpha, L, _ptr(tv, _f64p)))
    return (val, tv) if terms else val


def score_by_complement(graph, S, alpha: float, L: int, w=None) -> float:
    """GED_{<=L}(S) as sum_i alpha^i (W_i - M_i) (Def. ged-walk; cancels for small S)."""
    n, rp, ci = _g(graph)
    s, sl = _S(S)
    return float(_load().orc_score_by_complement_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), _ptr(s, _i32p), sl,
                                                   alpha, L))


def gain(graph, S, x: int, alpha: float, L: int, long_double: bool = False, w=None) -> float:
    """GED_{<=L}(S, x), counted directly as the weighted walks through x avoiding S."""
    n, rp, ci = _g(graph)
    s, sl = _S(S)
    lib = _load()
    f = lib.orc_gain_ld_as_d if long_double else lib.orc_gain_d
    return float(f(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), _ptr(s, _i32p), sl, int(x), alpha, L))


def upper_bounds(graph, S, alpha: float, L: int, w=None, directed: bool = False) -> np.ndarray:
    """sum_{i<=L} alpha^i P_i(S, x) for every x (Lemma initialize)."""
    n, rp, ci = _g(graph)
    s, sl = _S(S)
    ub = np.zeros(max(n, 1), dtype=np.float64)
    rpt, cit, wt = _tp(graph, w, directed)
    _load().orc_upper_bounds_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), rpt, cit, wt, _ptr(s, _i32p), sl,
                               alpha, L, _ptr(ub, _f64p))
    return ub[:n]


def greedy(graph, k: int, alpha: float, L: int, mode: str = "all", init=None, w=None, directed: bool = False):
    """Greedy maximisation at fixed L: (group, gains, evaluations). mode 'all' or 'lazy'."""
    n, rp, ci = _g(graph)
    ini, il = _S(init)
    group = np.zeros(max(k, 1), dtype=np.int32)
    gains = np.zeros(max(k, 1), dtype=np.float64)
    ev = ctypes.c_int64(0)
    rpt, cit, wt = _tp(graph, w, directed)
    rc = _load().orc_greedy_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), rpt, cit, wt, k, alpha, L,
                              0 if mode == "all" else 1,
                              _ptr(ini, _i32p), il, _ptr(group, _i32p), _ptr(gains, _f64p), ctypes.byref(ev))
    if rc != 0:
        raise ValueError("oracle greedy: invalid arguments")
    return group[:k].copy(), gains[:k].copy(), int(ev.value)


def sample_hash(seed: int, step: int, v: int) -> int:
    """The counter-based draw of stochastic greedy: splitmix64's first output from seed ^ (step<<32) ^ v."""
    return int(_load().orc_sample_hash(seed, step, v))


def greedy_stochastic(graph, k: int, alpha: float, L: int, eta: float, seed: int, w=None):
    """Stochastic greedy (Appendix D) at fixed L: (group, gains, evaluations)."""
    n, rp, ci = _g(graph)
    group = np.zeros(max(k, 1), dtype=np.int32)
    gains = np.zeros(max(k, 1), dtype=np.float64)
    ev = ctypes.c_int64(0)
    rc = _load().orc_greedy_stochastic_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), k, alpha, L, eta, seed,
                                         _ptr(group, _i32p), _ptr(gains, _f64p), ctypes.byref(ev))
    if rc != 0:
        raise ValueError("oracle stochastic greedy: invalid arguments")
    return group[:k].copy(), gains[:k].copy(), int(ev.value)


def greedy_adaptive(graph, k: int, alpha: float, eps_sep: float, lcap: int = 4096, w=None, directed: bool = False):
    """Lazy greedy with l-doubling and eps_sep-separation (Algorithm 2).

    Returns a dict: group, gains (L_l(S, u) at each step's l), ell (each step's l), evals, and
    the separation tests as arrays att_step, att_ell, att_gu, att_gv (-1 without v), att_B.
    """
    n, rp, ci = _g(graph)
    group = np.zeros(max(k, 1), dtype=np.int32)
    gains = np.zeros(max(k, 1), dtype=np.float64)
    ell = np.zeros(max(k, 1), dtype=np.int32)
    cap = 4 * k + 64
    a_step = np.zeros(cap, dtype=np.int32)
    a_ell = np.zeros(cap, dtype=np.int32)
    a_gu = np.zeros(cap, dtype=np.float64)
    a_gv = np.zeros(cap, dtype=np.float64)
    a_B = np.zeros(cap, dtype=np.float64)
    ev = ctypes.c_int64(0)
    na = ctypes.c_int32(0)
    rpt, cit, wt = _tp(graph, w, directed)
    rc = _load().orc_greedy_adaptive_d(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _wp(graph, w), rpt, cit, wt, k, alpha,
                                       eps_sep, lcap,
                                       _ptr(group, _i32p), _ptr(gains, _f64p), _ptr(ell, _i32p), ctypes.byref(ev),
                                       cap, _ptr(a_step, _i32p), _ptr(a_ell, _i32p), _ptr(a_gu, _f64p),
                                       _ptr(a_gv, _f64p), _ptr(a_B, _f64p), ctypes.byref(na))
    if rc == -2:
        raise ValueError("oracle adaptive greedy: l exceeded lcap")
    if rc != 0:
        raise ValueError("oracle adaptive greedy: invalid arguments")
    m = min(int(na.value), cap)
    return {"group": group[:k].copy(), "gains": gains[:k].copy(), "ell": ell[:k].copy(), "evals": int(ev.value),
            "att_step": a_step[:m].copy(), "att_ell": a_ell[:m].copy(), "att_gu": a_gu[:m].copy(),
            "att_gv": a_gv[:m].copy(), "att_B": a_B[:m].copy()}


def brute_phi(graph, S, i: int):
    """(phi_i(S), W_i) by enumerating every i-walk (exact integers)."""
    n, rp, ci = _g(graph)
    s, sl = _S(S)
    phi, w = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _load().orc_brute_phi(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _ptr(s, _i32p), sl, i, ctypes.byref(phi),
                          ctypes.byref(w))
    return int(phi.value), int(w.value)


def brute_gain(graph, S, x: int, i: int) -> int:
    """Number of i-walks that visit x and avoid S, by enumeration."""
    n, rp, ci = _g(graph)
    s, sl = _S(S)
    out = ctypes.c_uint64(0)
    _load().orc_brute_gain(n, _ptr(rp, _i32p), _ptr(ci, _i32p), _ptr(s, _i32p), sl, int(x), i, ctypes.byref(out))
    return int(out.value)
