"""Seeded synthetic graph inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the graph method itself: it emits edge
tuples (R-MAT or a 2-D grid with random edge deletions) and chooses source
vertices. Each side then builds its own matrix from the tuples.

Input recipe (the workloads of the paper's Section 8, re-created
synthetically because the real datasets are not available):

* R-MAT with a=0.57, b=0.19, c=0.19, d=0.05 (Section 8, dataset paragraph),
  2^scale vertices, edgefactor * 2^scale generated edges, a seeded random
  vertex permutation, self-loops dropped, both directions emitted
  (the paper's datasets are undirected without self-loops, Table 11
  caption). Duplicates are left for the matrix build to remove.
* Grid: rows x cols 4-neighbour lattice, each undirected edge deleted with
  probability p, weights uniform in [1, wmax]; a road-network stand-in.
* Weights of {u, v} are a hash of the unordered pair, so A stays symmetric.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgen.so")
_lock = threading.Lock()
_lib = None

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.gen_draw.restype = ctypes.c_uint64
            lib.gen_draw.argtypes = [ctypes.c_uint64] * 3
            lib.gen_edge_weight.restype = ctypes.c_uint32
            lib.gen_edge_weight.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            lib.gen_permutation.restype = None
            lib.gen_permutation.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p]
            lib.gen_rmat.restype = ctypes.c_uint64
            lib.gen_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint32, u32p, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_int, u32p, u32p, ctypes.c_void_p]
            lib.gen_grid.restype = ctypes.c_uint64
            lib.gen_grid.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_uint32, u32p, u32p, ctypes.c_void_p]
            lib.gen_sources.restype = ctypes.c_uint32
            lib.gen_sources.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_uint32, u32p]
            lib.gen_touched.restype = None
            lib.gen_touched.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, ctypes.c_void_p]
            _lib = lib
    return _lib


def _u32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


class Tuples:
    """Edge tuples of an undirected graph on n vertices (both directions)."""

    def __init__(self, n, src, dst, w, name):
        self.n = int(n)
        self.src = src
        self.dst = dst
        self.w = w
        self.name = name

    @property
    def ntuples(self) -> int:
        return int(self.src.shape[0])


def thresholds(abcd=RMAT_ABCD):
    a, b, c, _ = abcd
    t = [int(a * 2**32), int((a + b) * 2**32), int((a + b + c) * 2**32)]
    return np.array([min(x, 2**32 - 1) for x in t], dtype=np.uint32)


def rmat(scale: int, edgefactor: int = 16, seed: int = 1, wmax: int = 0,
         permute: bool = True, abcd=RMAT_ABCD) -> Tuples:
    """R-MAT tuples: 2^scale vertices; wmax>0 adds weights in [1, wmax]."""
    lib = _load()
    nedges = edgefactor << scale
    src = np.empty(2 * nedges, dtype=np.uint32)
    dst = np.empty(2 * nedges, dtype=np.uint32)
    w = np.empty(2 * nedges, dtype=np.uint32) if wmax > 0 else None
    thr = thresholds(abcd)
    k = lib.gen_rmat(scale, edgefactor, _u32p(thr), seed, wmax, 1 if permute else 0,
                     _u32p(src), _u32p(dst), w.ctypes.data if w is not None else None)
    src, dst = src[:k], dst[:k]
    if w is not None:
        w = w[:k]
    return Tuples(1 << scale, src, dst, w, f"rmat_s{scale}_e{edgefactor}_seed{seed}")


def grid(rows: int, cols: int, p_delete: float = 0.1, seed: int = 3, wmax: int = 0) -> Tuples:
    """rows x cols 4-neighbour lattice with each edge deleted w.p. p_delete."""
    lib = _load()
    cap = 2 * (rows * (cols - 1) + (rows - 1) * cols)
    src = np.empty(max(cap, 1), dtype=np.uint32)
    dst = np.empty(max(cap, 1), dtype=np.uint32)
    w = np.empty(max(cap, 1), dtype=np.uint32) if wmax > 0 else None
    thr = min(int(p_delete * 2**32), 2**32 - 1)
    k = lib.gen_grid(rows, cols, thr, seed, wmax, _u32p(src), _u32p(dst),
                     w.ctypes.data if w is not None else None)
    src, dst = src[:k], dst[:k]
    if w is not None:
        w = w[:k]
    return Tuples(rows * cols, src, dst, w, f"grid_{rows}x{cols}_p{p_delete}_seed{seed}")


def touched(t: Tuples) -> np.ndarray:
    """uint8 flag per vertex: 1 if it appears in any tuple (non-isolated)."""
    lib = _load()
    out = np.empty(t.n, dtype=np.uint8)
    lib.gen_touched(t.n, t.ntuples, _u32p(t.src), out.ctypes.data)
    return out


def sources(t: Tuples, k: int, seed: int = 1) -> np.ndarray:
    """k distinct non-isolated vertices drawn uniformly (seeded), draw order."""
    lib = _load()
    has = touched(t)
    out = np.empty(max(k, 1), dtype=np.uint32)
    got = lib.gen_sources(seed, t.n, has.ctypes.data, k, _u32p(out))
    return out[:got]


def first_nonisolated(t: Tuples) -> int:
    """Lowest-id vertex with at least one edge (grid source)."""
    has = touched(t)
    nz = np.flatnonzero(has)
    return int(nz[0]) if nz.size else 0


def permutation(n: int, seed: int) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.uint32)
    lib.gen_permutation(seed, n, _u32p(out))
    return out


def draw(seed: int, stream: int, counter: int) -> int:
    return int(_load().gen_draw(seed, stream, counter))


def from_edges(n: int, edges, weights=None, name: str = "small") -> Tuples:
    """Tuples of a small undirected graph given as a list of {u, v} pairs
    (each pair emitted in both directions; used for hand-made test graphs)."""
    e = np.asarray(list(edges), dtype=np.uint32).reshape(-1, 2)
    src = np.concatenate([e[:, 0], e[:, 1]]).astype(np.uint32)
    dst = np.concatenate([e[:, 1], e[:, 0]]).astype(np.uint32)
    w = None
    if weights is not None:
        ww = np.asarray(weights, dtype=np.uint32)
        w = np.concatenate([ww, ww]).astype(np.uint32)
    return Tuples(n, src, dst, w, name)


def random_small(n: int, p: float, seed: int, wmax: int = 0) -> Tuples:
    """Erdos-Renyi G(n, p) on a few vertices (for brute-force pins)."""
    edges, ws = [], []
    for u in range(n):
        for v in range(u + 1, n):
            x = draw(seed, 0x534d414c, u * n + v)
            if (x & 0xFFFFFFFF) < int(p * 2**32):
                edges.append((u, v))
                ws.append(1 + (x >> 32) % wmax if wmax else 1)
    return from_edges(n, edges, ws if wmax else None, name=f"gnp_{n}_{p}_{seed}")
