"""ctypes binding of libgedwalk.so (the C ABI declared in include/gedwalk.h).

Argument marshalling only: every step of GED-Walk scoring and maximisation runs in the
library's CUDA kernels. There is no CPU fallback; when the library is missing or cannot
be loaded, every call raises.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import sys
import threading
import weakref
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libgedwalk.so")

OK, ERR_INVALID, ERR_OOM, ERR_NOT_CONVERGENT, ERR_DEVICE, ERR_TIMEOUT, ERR_BUSY, ERR_NOT_FOUND = range(8)
FP64, FP32 = 0, 1
EPS_OVER_K, EPS_PLAIN = 0, 1
GAINS_ALL = 1
STOCHASTIC = 2
ADAPTIVE_L = 4
DEVICE_LOOP = 8
BOUND_COMBINATORIAL, BOUND_SPECTRAL = 0, 1
UPLOAD_TRUSTED = 1
UPLOAD_DIRECTED = 2
REQ_SCORE, REQ_MAXIMIZE = 0, 1

_STATUS_NAMES = {OK: "OK", ERR_INVALID: "INVALID", ERR_OOM: "OOM", ERR_NOT_CONVERGENT: "NOT_CONVERGENT",
                 ERR_DEVICE: "DEVICE", ERR_TIMEOUT: "TIMEOUT", ERR_BUSY: "BUSY", ERR_NOT_FOUND: "NOT_FOUND"}

# every exported entry point of include/gedwalk.h
EXPORTS = [
    "gedwalk_params_default", "gedwalk_set_allocator", "gedwalk_graph_upload", "gedwalk_graph_upload_weighted",
    "gedwalk_graph_info_weighted", "gedwalk_graph_free", "gedwalk_truncation_ex", "gedwalk_sigma_max",
    "gedwalk_graph_info", "gedwalk_truncation", "gedwalk_score", "gedwalk_score_batch", "gedwalk_batch_tuning",
    "gedwalk_batch_set_width",
    "gedwalk_gains",
    "gedwalk_maximize", "gedwalk_maximize_stats", "gedwalk_maximize_lengths", "gedwalk_serve_create", "gedwalk_serve_submit",
    "gedwalk_serve_poll", "gedwalk_serve_stats", "gedwalk_serve_counters_read", "gedwalk_serve_destroy",
    "gedwalk_score_step_noalloc",
    "gedwalk_profile", "gedwalk_profile_read", "gedwalk_last_error",
]


class GedWalkError(RuntimeError):
    """A failing call: .status is the gedwalk_status code, the message the library's last error."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ServeCounters(ctypes.Structure):
    """gedwalk_serve_counters: a server's admission and batching counters (int64 each)."""
    _fields_ = [(name, ctypes.c_int64) for name in (
        "completed", "batches", "batched_requests", "peak_bytes", "budget", "charged_bytes", "idle_held_bytes",
        "admitted_at_submit", "admitted_after_wait", "peak_maximize_running", "releases", "released_bytes",
        "pending")]


class ProfileStats(ctypes.Structure):
    """gedwalk_profile_stats: launch count and event-timed sweep launches."""
    _fields_ = [
        ("launches", ctypes.c_int64),
        ("sweep_launches", ctypes.c_int64),
        ("sweep_ms", ctypes.c_double),
        ("sweep_bytes", ctypes.c_double),
        ("top_mode", ctypes.c_int32),
        ("top_cols", ctypes.c_int32),
        ("top_fp64", ctypes.c_int32),
        ("top_pad", ctypes.c_int32),
        ("top_launches", ctypes.c_int64),
        ("top_ms", ctypes.c_double),
        ("top_bytes", ctypes.c_double),
    ]


class Params(ctypes.Structure):
    """gedwalk_params, field for field; build one with make_params()."""
    _fields_ = [
        ("alpha", ctypes.c_double),
        ("epsilon", ctypes.c_double),
        ("L", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("greedy_eps_rule", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("stream", ctypes.c_int64),
        ("eta", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("bound", ctypes.c_int32),
        ("lookahead", ctypes.c_int32),
        ("spec_cols", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()


def load(path: Optional[str] = None, torch_allocator: bool = True):
    """Loads libgedwalk.so (built by paper_1910_13874_gb300.build). Raises if it is missing.

    On first load it routes the library's device allocations through PyTorch's caching allocator
    (use_torch_allocator) unless torch_allocator is False.
    """
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build the CUDA library first "
                               "(python -m paper_1910_13874_gb300.build); there is no CPU fallback")
        lib = ctypes.CDLL(p)
        vp = ctypes.c_void_p
        sig = {
            "gedwalk_params_default": (None, [ctypes.POINTER(Params)]),
            "gedwalk_set_allocator": (ctypes.c_int, [_ALLOC_FN, _FREE_FN, vp]),
            "gedwalk_graph_upload": (ctypes.c_int, [_i32p, _i32p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                                    ctypes.POINTER(vp)]),
            "gedwalk_graph_upload_weighted": (ctypes.c_int, [_i32p, _i32p, ctypes.c_int32, ctypes.c_int64, _f64p,
                                                             ctypes.c_int32, ctypes.POINTER(vp)]),
            "gedwalk_graph_info_weighted": (ctypes.c_int, [vp, _i32p, _f64p]),
            "gedwalk_truncation_ex": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int32, _i32p,
                                                     _f64p]),
            "gedwalk_sigma_max": (ctypes.c_int, [vp, ctypes.c_int32, _f64p, _f64p]),
            "gedwalk_graph_free": (ctypes.c_int, [vp]),
            "gedwalk_graph_info": (ctypes.c_int, [vp, _i32p, _i64p, _i32p, _f64p]),
            "gedwalk_truncation": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, _i32p, _f64p]),
            "gedwalk_score": (ctypes.c_int, [vp, _i32p, ctypes.c_int32, ctypes.POINTER(Params), _f64p, _i32p,
                                             _f64p]),
            "gedwalk_score_batch": (ctypes.c_int, [vp, _i32p, _i32p, ctypes.c_int32, ctypes.POINTER(Params),
                                                   _f64p, _i32p]),
            "gedwalk_batch_tuning": (ctypes.c_int, [vp, _i32p, _f64p, ctypes.c_int32, _i32p, _i32p]),
            "gedwalk_batch_set_width": (ctypes.c_int, [vp, ctypes.c_int32]),
            "gedwalk_gains": (ctypes.c_int, [vp, _i32p, ctypes.c_int32, ctypes.POINTER(Params), _f64p, _i32p]),
            "gedwalk_maximize": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.POINTER(Params), _i32p, _f64p, _f64p,
                                                _i32p, _i32p, ctypes.c_int32]),
            "gedwalk_maximize_stats": (ctypes.c_int, [vp, _i64p, _i64p, _i64p, _i64p]),
            "gedwalk_maximize_lengths": (ctypes.c_int, [vp, _i32p, ctypes.c_int32, _i32p, _i64p]),
            "gedwalk_serve_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_int64,
                                                    ctypes.c_int32, ctypes.POINTER(vp)]),
            "gedwalk_serve_submit": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, _i32p, ctypes.c_int32,
                                                    ctypes.POINTER(Params), _u64p]),
            "gedwalk_serve_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_int32, _f64p, _i32p, _f64p, _f64p,
                                                  _i32p]),
            "gedwalk_serve_stats": (ctypes.c_int, [vp, _i64p, _i64p, _i64p, _i64p]),
            "gedwalk_serve_counters_read": (ctypes.c_int, [vp, ctypes.POINTER(ServeCounters)]),
            "gedwalk_serve_destroy": (ctypes.c_int, [vp]),
            "gedwalk_score_step_noalloc": (ctypes.c_int, [vp, vp, ctypes.c_int32, vp, vp, vp, ctypes.c_double, vp,
                                                          ctypes.c_int64]),
            "gedwalk_profile": (ctypes.c_int, [ctypes.c_int32]),
            "gedwalk_profile_read": (ctypes.c_int, [ctypes.POINTER(ProfileStats)]),
            "gedwalk_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    if torch_allocator:
        use_torch_allocator()
    return _lib


def _check(st: int):
    if st != OK:
        msg = load().gedwalk_last_error().decode(errors="replace")
        raise GedWalkError(st, msg)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).ravel())


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def make_params(alpha: float = 0.0, epsilon: float = 1e-4, L: int = 0, precision: str = "fp32",
                eps_rule: str = "over_k", gains_all: bool = False, stream: int = 0, stochastic: bool = False,
                eta: float = 0.1, seed: int = 0, adaptive: bool = False, bound: str = "combinatorial",
                lookahead: int = 0, spec_cols: int = 0, device_loop: bool = False) -> Params:
    """gedwalk_params from keywords: precision "fp32"/"fp64", eps_rule "over_k"/"plain", bound
    "combinatorial"/"spectral", the flags as booleans; 0 keeps the library's default (alpha
    1/(1+d_max), L from the bound, lookahead 7 in FP32 and 3 in FP64)."""
    p = Params()
    load().gedwalk_params_default(ctypes.byref(p))
    p.alpha = alpha
    p.epsilon = epsilon
    p.L = L
    p.precision = FP64 if precision in ("fp64", "f64", FP64) else FP32
    p.greedy_eps_rule = EPS_PLAIN if eps_rule == "plain" else EPS_OVER_K
    p.flags = ((GAINS_ALL if gains_all else 0) | (STOCHASTIC if stochastic else 0) | (ADAPTIVE_L if adaptive else 0)
               | (DEVICE_LOOP if device_loop else 0))
    p.bound = {"combinatorial": BOUND_COMBINATORIAL, "spectral": BOUND_SPECTRAL}[bound]
    p.stream = int(stream)
    p.eta = eta
    p.seed = seed
    p.lookahead = int(lookahead)
    p.spec_cols = int(spec_cols)
    return p


_torch_hooks = None
_hook_refs = []  # every hook pair ever installed: a block is freed through the hook that made it


def use_torch_allocator():
    """Routes the library's device allocations through PyTorch's caching allocator."""
    global _torch_hooks
    import torch

    if _torch_hooks is not None:
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream))
        except Exception:  # out of memory: the library reports GEDWALK_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _hook_refs.append(hooks)
    if not _exit_hook:  # registered after torch's own exit handlers, so it runs before them
        atexit.register(_close_servers)
        _exit_hook.append(True)
    _torch_hooks = hooks
    _check(load(torch_allocator=False).gedwalk_set_allocator(hooks[0], hooks[1], None))


def score_step_noalloc(d_row_ptr: int, d_col_idx: int, n: int, d_mask: int, d_x: int, d_y: int, alpha: float,
                       d_hit_sum: int, stream: int = 0):
    """One two-state step on caller-owned device buffers (raw device addresses); allocates nothing."""
    _check(load().gedwalk_score_step_noalloc(d_row_ptr, d_col_idx, n, d_mask, d_x, d_y, alpha, d_hit_sum, stream))


def profile(enable: bool = True):
    """Starts (or stops) timing sweep launches; resets the counters."""
    _check(load().gedwalk_profile(1 if enable else 0))


def profile_read() -> dict:
    """Waits for the timed sweep launches and returns gedwalk_profile_stats as a dict."""
    st = ProfileStats()
    _check(load().gedwalk_profile_read(ctypes.byref(st)))
    return {"launches": st.launches, "sweep_launches": st.sweep_launches, "sweep_ms": st.sweep_ms,
            "sweep_bytes": st.sweep_bytes, "top_mode": st.top_mode, "top_cols": st.top_cols,
            "top_fp64": st.top_fp64, "top_launches": st.top_launches, "top_ms": st.top_ms,
            "top_bytes": st.top_bytes}


class Graph:
    """A device-resident graph (undirected CSR uploaded with gedwalk_graph_upload)."""

    def __init__(self, row_ptr, col_idx, trusted: bool = False, weighted: bool = False, vertex_scale=None,
                 directed: bool = False):
        """weighted: walks weighted by w(v,u) = s_v s_u (gedwalk_graph_upload_weighted); vertex_scale
        gives s (float64[n]), None the normalised adjacency D^{-1/2} A D^{-1/2}. directed: the rows
        are successor lists of a directed graph."""
        lib = load()
        rp = _i32(row_ptr)
        ci = _i32(col_idx)
        n = rp.shape[0] - 1
        h = ctypes.c_void_p()
        ci_arg = ci if ci.size else np.zeros(1, np.int32)
        fl = (UPLOAD_TRUSTED if trusted else 0) | (UPLOAD_DIRECTED if directed else 0)
        if weighted or vertex_scale is not None:
            sc = None
            if vertex_scale is not None:
                sc = np.ascontiguousarray(vertex_scale, dtype=np.float64)
                if sc.shape != (n,):
                    raise ValueError("vertex_scale must hold n values")
            _check(lib.gedwalk_graph_upload_weighted(_ptr(rp, _i32p), _ptr(ci_arg, _i32p), n, ci.size,
                                                     None if sc is None else _ptr(sc, _f64p), fl, ctypes.byref(h)))
        else:
            _check(lib.gedwalk_graph_upload(_ptr(rp, _i32p), _ptr(ci_arg, _i32p), n, ci.size, fl, ctypes.byref(h)))
        self._h = h
        n_, nnz, dmax, alpha = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
        _check(lib.gedwalk_graph_info(h, ctypes.byref(n_), ctypes.byref(nnz), ctypes.byref(dmax),
                                      ctypes.byref(alpha)))
        self.n, self.nnz, self.dmax, self.alpha_default = n_.value, nnz.value, dmax.value, alpha.value
        wt, dl = ctypes.c_int32(), ctypes.c_double()
        _check(lib.gedwalk_graph_info_weighted(h, ctypes.byref(wt), ctypes.byref(dl)))
        self.weighted, self.delta = bool(wt.value), dl.value
        self.directed = bool(directed)

    @classmethod
    def from_host(cls, g, trusted: bool = False, weighted: bool = False, vertex_scale=None, directed: bool = False):
        """Uploads a host graph with row_ptr / col_idx arrays (such as graphgen's)."""
        return cls(g.row_ptr, g.col_idx, trusted=trusted, weighted=weighted, vertex_scale=vertex_scale,
                   directed=directed)

    @property
    def handle(self):
        """The gedwalk_graph_t (ctypes.c_void_p)."""
        return self._h

    def free(self):
        """Releases the graph's device memory (gedwalk_graph_free); later calls on it fail."""
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gedwalk_graph_free(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():  # the process exit releases the device memory; no hook may run now
            return
        try:
            self.free()
        except Exception:
            pass

    def truncation(self, alpha: float = 0.0, epsilon: float = 1e-4, bound: str = "combinatorial"):
        """(L, B_L) for (alpha, epsilon) with the combinatorial or the spectral tail bound."""
        L, b = ctypes.c_int32(), ctypes.c_double()
        if bound == "combinatorial":
            _check(load().gedwalk_truncation(self._h, alpha, epsilon, ctypes.byref(L), ctypes.byref(b)))
        else:
            kind = {"spectral": BOUND_SPECTRAL}[bound]
            _check(load().gedwalk_truncation_ex(self._h, alpha, epsilon, kind, ctypes.byref(L), ctypes.byref(b)))
        return L.value, b.value

    def sigma_max(self, iters: int = 300):
        """(upper, lower) bounds of the largest singular value of A (gedwalk_sigma_max)."""
        up, lo = ctypes.c_double(), ctypes.c_double()
        _check(load().gedwalk_sigma_max(self._h, iters, ctypes.byref(up), ctypes.byref(lo)))
        return up.value, lo.value

    def score(self, S: Sequence[int], params: Optional[Params] = None, **kw):
        """(score, L, tail_bound) of one group."""
        p = params or make_params(**kw)
        s = _i32(S)
        out, L, b = ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
        s_arg = s if s.size else np.zeros(1, np.int32)
        _check(load().gedwalk_score(self._h, _ptr(s_arg, _i32p), s.size, ctypes.byref(p), ctypes.byref(out),
                                    ctypes.byref(L), ctypes.byref(b)))
        return out.value, L.value, b.value

    def score_batch(self, offsets, members, params: Optional[Params] = None, **kw):
        """(scores[G], L) of groups members[offsets[j]:offsets[j+1]]."""
        p = params or make_params(**kw)
        off = _i32(offsets)
        mem = _i32(members)
        G = off.size - 1
        out = np.zeros(max(G, 1), dtype=np.float64)
        L = ctypes.c_int32()
        mem_arg = mem if mem.size else np.zeros(1, np.int32)
        _check(load().gedwalk_score_batch(self._h, _ptr(off, _i32p), _ptr(mem_arg, _i32p), G, ctypes.byref(p),
                                          _ptr(out, _f64p), ctypes.byref(L)))
        return out[:G], L.value

    def batch_tuning(self):
        """(widths, us per column, chosen width) of the batched-scoring autotuner on this graph."""
        cnt, chosen = ctypes.c_int32(), ctypes.c_int32()
        _check(load().gedwalk_batch_tuning(self._h, None, None, 0, ctypes.byref(cnt), ctypes.byref(chosen)))
        cols = np.zeros(max(cnt.value, 1), dtype=np.int32)
        us = np.zeros(max(cnt.value, 1), dtype=np.float64)
        _check(load().gedwalk_batch_tuning(self._h, _ptr(cols, _i32p), _ptr(us, _f64p), cnt.value, ctypes.byref(cnt),
                                           ctypes.byref(chosen)))
        return cols[:cnt.value].tolist(), us[:cnt.value].tolist(), chosen.value

    def batch_set_width(self, cols: int):
        """Pins the batched-scoring column-block width (8, 16, 32, 64), or 0 to tune it again."""
        _check(load().gedwalk_batch_set_width(self._h, int(cols)))

    def gains(self, S: Sequence[int], params: Optional[Params] = None, **kw):
        """(gains[n], L): exact truncated marginal gain of every vertex."""
        p = params or make_params(**kw)
        s = _i32(S)
        out = np.zeros(self.n, dtype=np.float64)
        L = ctypes.c_int32()
        s_arg = s if s.size else np.zeros(1, np.int32)
        _check(load().gedwalk_gains(self._h, _ptr(s_arg, _i32p), s.size, ctypes.byref(p), _ptr(out, _f64p),
                                    ctypes.byref(L)))
        return out, L.value

    def maximize(self, k: int, params: Optional[Params] = None, init=None, **kw):
        """(group[k], gains[k], score, L) of greedy maximisation."""
        p = params or make_params(**kw)
        grp = np.zeros(max(k, 1), dtype=np.int32)
        gains = np.zeros(max(k, 1), dtype=np.float64)
        score, L = ctypes.c_double(), ctypes.c_int32()
        ini = _i32(init if init is not None else [])
        ini_arg = ini if ini.size else np.zeros(1, np.int32)
        _check(load().gedwalk_maximize(self._h, k, ctypes.byref(p), _ptr(grp, _i32p), _ptr(gains, _f64p),
                                       ctypes.byref(score), ctypes.byref(L), _ptr(ini_arg, _i32p), ini.size))
        return grp[:k].copy(), gains[:k].copy(), score.value, L.value

    def maximize_stats(self):
        """Counters of the last maximize: evaluations, batches, sweeps, spec_misses."""
        vals = [ctypes.c_int64() for _ in range(4)]
        _check(load().gedwalk_maximize_stats(self._h, *[ctypes.byref(v) for v in vals]))
        return dict(zip(("evaluations", "batches", "sweeps", "spec_misses"), (v.value for v in vals)))

    def maximize_lengths(self):
        """(ell, separation_failures): the walk length of each step of the last maximize."""
        cnt = ctypes.c_int32()
        fails = ctypes.c_int64()
        _check(load().gedwalk_maximize_lengths(self._h, None, 0, ctypes.byref(cnt), None))
        ell = np.zeros(max(cnt.value, 1), dtype=np.int32)
        _check(load().gedwalk_maximize_lengths(self._h, ell.ctypes.data_as(_i32p), cnt.value, ctypes.byref(cnt),
                                               ctypes.byref(fails)))
        return ell[:cnt.value].copy(), int(fails.value)


_live_servers = weakref.WeakSet()
_exit_hook = []


def _close_servers():
    # A server's threads may still call the allocator hook (Python); stop them before the
    # interpreter shuts down.
    for srv in list(_live_servers):
        try:
            srv.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over device-resident graphs (gedwalk_serve_*)."""

    def __init__(self, graphs: Sequence[Graph], mem_budget: int = 0, max_batch: int = 0):
        arr = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
        h = ctypes.c_void_p()
        _check(load().gedwalk_serve_create(arr, len(graphs), mem_budget, max_batch, ctypes.byref(h)))
        self._h = h
        _live_servers.add(self)
        self._graphs = list(graphs)
        self._kmax = {}

    def submit_score(self, graph: int, S, params: Optional[Params] = None, **kw) -> int:
        """Queues the scoring of group S on graph index `graph`; returns its ticket."""
        p = params or make_params(**kw)
        s = _i32(S)
        t = ctypes.c_uint64()
        s_arg = s if s.size else np.zeros(1, np.int32)
        _check(load().gedwalk_serve_submit(self._h, graph, REQ_SCORE, _ptr(s_arg, _i32p), s.size, ctypes.byref(p),
                                           ctypes.byref(t)))
        return t.value

    def submit_maximize(self, graph: int, k: int, params: Optional[Params] = None, **kw) -> int:
        """Queues a greedy maximisation of size k on graph index `graph`; returns its ticket."""
        p = params or make_params(**kw)
        t = ctypes.c_uint64()
        dummy = np.zeros(1, np.int32)
        _check(load().gedwalk_serve_submit(self._h, graph, REQ_MAXIMIZE, _ptr(dummy, _i32p), k, ctypes.byref(p),
                                           ctypes.byref(t)))
        self._kmax[t.value] = k
        return t.value

    def poll(self, ticket: int, wait_us: int = -1):
        """None while pending; else dict(score, group, gains, latency_us)."""
        k = self._kmax.get(ticket, 0)
        grp = np.zeros(max(k, 1), dtype=np.int32)
        gains = np.zeros(max(k, 1), dtype=np.float64)
        score, lat, done = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        st = load().gedwalk_serve_poll(self._h, ticket, wait_us, ctypes.byref(score), _ptr(grp, _i32p),
                                       _ptr(gains, _f64p), ctypes.byref(lat), ctypes.byref(done))
        if st == OK and not done.value:
            return None
        self._kmax.pop(ticket, None)
        _check(st)
        return {"score": score.value, "group": grp[:k].copy(), "gains": gains[:k].copy(), "latency_us": lat.value}

    def stats(self):
        """The server's counters (gedwalk_serve_counters) as a dict."""
        c = ServeCounters()
        _check(load().gedwalk_serve_counters_read(self._h, ctypes.byref(c)))
        return {name: getattr(c, name) for name, _ in ServeCounters._fields_}

    def close(self):
        """Stops the server (gedwalk_serve_destroy): admitted requests finish, waiting ones end BUSY."""
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gedwalk_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass
