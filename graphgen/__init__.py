"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

The module builds undirected, unweighted CSR graphs (``row_ptr`` int32[n+1], ``col_idx``
int32[nnz], every row strictly increasing, no self-loops) and random vertex groups. It
holds none of the GED-Walk arithmetic. The generator families follow the paper's
synthetic-graph setup (Appendix C): Erdos-Renyi, Barabasi-Albert and R-MAT with the
Graph 500 parameters (edge factor 16, a=0.57, b=c=0.19, d=0.05).

The heavy generators live in ``graphgen.c`` and are compiled with gcc on first use (or by
``__graft_entry__.build()``) into ``graphgen/_build/libgraphgen.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


class _CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("nnz", ctypes.c_int64),
        ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
        ("col_idx", ctypes.POINTER(ctypes.c_int32)),
    ]


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (host code only, any architecture)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.gg_er.restype = P(_CSR)
            lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64]
            lib.gg_ba.restype = P(_CSR)
            lib.gg_ba.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64]
            lib.gg_rmat.restype = P(_CSR)
            lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int32]
            lib.gg_rmat_ex.restype = P(_CSR)
            lib.gg_rmat_ex.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32]
            lib.gg_from_arcs.restype = P(_CSR)
            lib.gg_from_arcs.argtypes = [ctypes.c_int32, ctypes.c_int64, P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.gg_from_edges.restype = P(_CSR)
            lib.gg_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [P(_CSR)]
            lib.gg_rng_fill.restype = None
            lib.gg_rng_fill.argtypes = [ctypes.c_uint64, P(ctypes.c_uint64), ctypes.c_int64]
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected CSR graph on host memory."""

    row_ptr: np.ndarray  # int32[n+1]
    col_idx: np.ndarray  # int32[nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    @property
    def d_max(self) -> int:
        return int(self.degrees.max()) if self.n > 0 else 0

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n), dtype=np.int64)
        for v in range(self.n):
            a[v, self.col_idx[self.row_ptr[v]:self.row_ptr[v + 1]]] = 1
        return a


def _take(ptr, name: str) -> Graph:
    if not ptr:
        raise MemoryError(f"graph generator {name} failed (invalid arguments or out of memory)")
    lib = _load()
    c = ptr.contents
    n, nnz = int(c.n), int(c.nnz)
    rp = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy()
    ci = np.ctypeslib.as_array(c.col_idx, shape=(max(nnz, 1),))[:nnz].copy()
    lib.gg_free(ptr)
    return Graph(rp, ci, name)


def erdos_renyi(n: int, avg_degree: float, seed: int) -> Graph:
    """G(n, p) with p = avg_degree / (n - 1)."""
    p = 0.0 if n < 2 else min(1.0, float(avg_degree) / (n - 1))
    return _take(_load().gg_er(n, p, seed), f"er(n={n},deg={avg_degree},seed={seed})")


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    return _take(_load().gg_ba(n, m, seed), f"ba(n={n},m={m},seed={seed})")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True, directed: bool = False) -> Graph:
    """R-MAT; directed keeps the tuples as arcs (successor-list CSR) instead of symmetrising."""
    return _take(_load().gg_rmat_ex(scale, edge_factor, a, b, c, seed, int(permute), int(directed)),
                 f"rmat(scale={scale},ef={edge_factor},seed={seed}{',directed' if directed else ''})")


def from_edges(n: int, edges) -> Graph:
    """Symmetric CSR from an undirected edge list (pairs); duplicates and self-loops dropped."""
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    P = ctypes.POINTER(ctypes.c_int32)
    return _take(_load().gg_from_edges(n, e.shape[0], src.ctypes.data_as(P), dst.ctypes.data_as(P)),
                 f"edges(n={n},m={e.shape[0]})")


def from_arcs(n: int, arcs) -> Graph:
    """Directed CSR of successor lists (row u: the v with u -> v); duplicates and self-loops dropped."""
    e = np.asarray(arcs, dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    P = ctypes.POINTER(ctypes.c_int32)
    return _take(_load().gg_from_arcs(n, e.shape[0], src.ctypes.data_as(P), dst.ctypes.data_as(P)),
                 f"arcs(n={n},m={e.shape[0]})")


def random_digraph(n: int, p: float, seed: int) -> Graph:
    """Directed G(n, p): every ordered pair (u, v), u != v, is an arc with probability p (numpy RNG)."""
    rng = np.random.default_rng(seed)
    a = rng.random((n, n)) < p
    np.fill_diagonal(a, False)
    u, v = np.nonzero(a)
    if u.size == 0:
        return Graph(np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
    return from_arcs(n, np.stack([u, v], axis=1))


def complete(n: int) -> Graph:
    return from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n)])


def star(leaves: int) -> Graph:
    """Star K_{1,leaves}; vertex 0 is the centre."""
    return from_edges(leaves + 1, [(0, v) for v in range(1, leaves + 1)])


def path(n: int) -> Graph:
    return from_edges(n, [(v, v + 1) for v in range(n - 1)])


def cycle(n: int) -> Graph:
    return from_edges(n, [(v, (v + 1) % n) for v in range(n)])


def rng_u64(seed: int, count: int) -> np.ndarray:
    """The xoshiro256** stream used by the C generators, for Python-side draws."""
    out = np.empty(count, dtype=np.uint64)
    _load().gg_rng_fill(seed, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), count)
    return out


def random_groups(n: int, count: int, size_lo: int, size_hi: int, seed: int):
    """`count` groups, sizes uniform in [size_lo, size_hi], members uniform without replacement.

    Returns (offsets int32[count+1], members int32[sum sizes]); members of a group are sorted.
    """
    rng = np.random.default_rng(seed)
    sizes = rng.integers(size_lo, size_hi + 1, size=count)
    sizes = np.minimum(sizes, n)
    offsets = np.zeros(count + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(sizes)
    members = np.empty(int(offsets[-1]), dtype=np.int32)
    for g in range(count):
        members[offsets[g]:offsets[g + 1]] = np.sort(rng.choice(n, size=int(sizes[g]), replace=False))
    return offsets, members


def random_graph_small(n: int, p: float, seed: int) -> Graph:
    """Tiny random graph for brute-force checks (dense pair loop, numpy RNG)."""
    rng = np.random.default_rng(seed)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]
    return from_edges(n, edges) if edges else Graph(np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
