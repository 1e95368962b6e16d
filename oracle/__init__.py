"""ORACLE -- test infrastructure only.

A plain, slow, obviously-correct CPU implementation of what the CUDA path
computes, written from the GraphBLAST paper (Yang, Buluc, Owens, ACM TOMS
2021, arXiv 1908.01407). Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product package never
does. It shares no code with the CUDA library: the only thing both sides
consume is the seeded tuple generator in ``gen/``.

The numeric kernels live in ``oracle.c`` (plain single-threaded C, compiled
with gcc into ``liboracle.so``); ``graphblas.py`` holds the semantics of the
generic operations (masked mxv/vxm/mxm, eWiseAdd/Mult, reduce) as
pure-Python loops for small inputs.

Every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, invariants, brute force and independent library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DUP_FIRST, DUP_SECOND, DUP_PLUS, DUP_MIN, DUP_MAX = range(5)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, single-threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp = ctypes.c_void_p
            u32, u64 = ctypes.c_uint32, ctypes.c_uint64
            lib.orc_csr_build.restype = ctypes.c_int64
            lib.orc_csr_build.argtypes = [u32, u32, u64, vp, vp, vp, ctypes.c_int, vp, vp, vp]
            lib.orc_bfs.restype = None
            lib.orc_bfs.argtypes = [u32, vp, vp, u32, vp]
            lib.orc_bfs_parent_violations.restype = u64
            lib.orc_bfs_parent_violations.argtypes = [u32, vp, vp, u32, vp, vp]
            lib.orc_sssp.restype = ctypes.c_int
            lib.orc_sssp.argtypes = [u32, vp, vp, vp, u32, vp]
            lib.orc_pagerank.restype = None
            lib.orc_pagerank.argtypes = [u32, vp, vp, vp, ctypes.c_double, u32, vp, vp]
            lib.orc_pagerank_delta.restype = u32
            lib.orc_pagerank_delta.argtypes = [u32, vp, vp, vp, ctypes.c_double, ctypes.c_float, u32, vp, vp]
            lib.orc_cc.restype = None
            lib.orc_cc.argtypes = [u32, vp, vp, vp]
            lib.orc_tc.restype = u64
            lib.orc_tc.argtypes = [u32, vp, vp]
            lib.orc_degree_order.restype = None
            lib.orc_degree_order.argtypes = [u32, vp, vp]
            lib.orc_masked_LL.restype = u64
            lib.orc_masked_LL.argtypes = [u32, vp, vp, vp]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class CSR:
    """Oracle-side CSR: rowptr uint64[n+1], colidx uint32[m], optional uint32 vals."""

    def __init__(self, n, rowptr, colidx, vals=None, ncols=None):
        self.n = int(n)
        self.ncols = int(ncols if ncols is not None else n)
        self.rowptr = rowptr
        self.colidx = colidx
        self.vals = vals

    @property
    def m(self) -> int:
        return int(self.rowptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int64)

    def row(self, i):
        return self.colidx[self.rowptr[i]:self.rowptr[i + 1]]


def csr_build(nrows, rows, cols, vals=None, dup=DUP_FIRST, ncols=None) -> CSR:
    """Sorted, de-duplicated CSR from tuples (Table 4 'build')."""
    lib = _load()
    ncols = nrows if ncols is None else ncols
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
    nt = rows.shape[0]
    rowptr = np.empty(nrows + 1, dtype=np.uint64)
    colidx = np.empty(max(nt, 1), dtype=np.uint32)
    ov = np.empty(max(nt, 1), dtype=np.uint32) if vals is not None else None
    m = lib.orc_csr_build(nrows, ncols, nt, _p(rows), _p(cols), _p(vals), dup,
                          _p(rowptr), _p(colidx), _p(ov))
    if m < 0:
        raise ValueError("oracle csr_build: index out of range")
    colidx = colidx[:m].copy()
    if ov is not None:
        ov = ov[:m].copy()
    return CSR(nrows, rowptr, colidx, ov, ncols)


def csr_from_tuples(t, dup=DUP_FIRST) -> CSR:
    return csr_build(t.n, t.src, t.dst, t.w, dup)


def bfs(g: CSR, src: int) -> np.ndarray:
    """int32 depth per vertex (source 0, unreachable -1)."""
    lv = np.empty(g.n, dtype=np.int32)
    _load().orc_bfs(g.n, _p(g.rowptr), _p(g.colidx), src, _p(lv))
    return lv


def bfs_parent_violations(g: CSR, src: int, levels, parents) -> int:
    levels = np.ascontiguousarray(levels, dtype=np.int32)
    parents = np.ascontiguousarray(parents, dtype=np.int32)
    return int(_load().orc_bfs_parent_violations(g.n, _p(g.rowptr), _p(g.colidx), src,
                                                  _p(levels), _p(parents)))


def sssp(g: CSR, src: int) -> np.ndarray:
    """uint32 shortest distances (unreachable UINT32_MAX); weights = g.vals."""
    if g.vals is None:
        raise ValueError("sssp needs edge weights")
    d = np.empty(g.n, dtype=np.uint32)
    rc = _load().orc_sssp(g.n, _p(g.rowptr), _p(g.colidx), _p(g.vals), src, _p(d))
    if rc != 0:
        raise OverflowError("a finite distance does not fit in uint32")
    return d


def _in_edges(g: CSR, directed: bool):
    """(in-neighbour CSR, out-degree row pointer or None) of graph g, whose
    rows are out-edges; a symmetric graph is its own transpose."""
    if not directed:
        return g, None
    rows = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.rowptr).astype(np.int64))
    return csr_build(g.n, g.colidx, rows), g.rowptr


def pagerank(g: CSR, alpha: float = 0.85, iters: int = 50, directed: bool = False):
    """FP64 PageRank vector and per-iteration L1 residuals. g's rows are
    out-edges; directed=False reads g as symmetric (rows are in-edges too)."""
    gi, od = _in_edges(g, directed)
    p = np.empty(g.n, dtype=np.float64)
    r = np.empty(max(iters, 1), dtype=np.float64)
    _load().orc_pagerank(g.n, _p(gi.rowptr), _p(gi.colidx), _p(od) if od is not None else None, alpha, iters,
                         _p(p), _p(r))
    return p, r[:iters]


def pagerank_delta(g: CSR, alpha: float = 0.85, eps: float = 1e-6, max_iters: int = 100, directed: bool = False):
    """FP64 adaptive PageRank (PageRankDelta): (p, iterations, active per
    iteration). Converged vertices are masked out of later iterations."""
    gi, od = _in_edges(g, directed)
    p = np.empty(g.n, dtype=np.float64)
    act = np.zeros(max(max_iters, 1), dtype=np.uint32)
    it = _load().orc_pagerank_delta(g.n, _p(gi.rowptr), _p(gi.colidx), _p(od) if od is not None else None, alpha,
                                    eps, max_iters, _p(p), _p(act))
    return p, int(it), act[:it]


def pagerank_residual(g: CSR, x, alpha: float = 0.85) -> float:
    """L1 size of one more PageRank step from x, ||T(x) - x||_1, in FP64,
    with T the recurrence of reading 5 (Section 7.3): T(x)(v) = (1-a)/n +
    a * (sum over edges u -> v of x(u)/outdeg(u) + D(x)/n), D(x) the sum of x
    over vertices without out-edges. g's rows are out-edges (for a
    symmetric g they are the in-edges too, and the formula is the same).
    T is an a-contraction in L1 (its linear part is column-stochastic), so
    ||x - p*||_1 <= r(x) / (1 - a) for the fixed point p*: how far any
    approximate PageRank vector is from p* is bounded by something computed
    from the vector alone."""
    x = np.asarray(x, dtype=np.float64)
    n = g.n
    outdeg = np.diff(g.rowptr).astype(np.int64)
    share = np.where(outdeg > 0, x / np.maximum(outdeg, 1), 0.0)
    u = np.repeat(np.arange(n, dtype=np.int64), outdeg)
    pulled = np.bincount(g.colidx.astype(np.int64), weights=share[u], minlength=n)
    dangling = x[outdeg == 0].sum()
    tx = (1.0 - alpha) / n + alpha * (pulled + dangling / n)
    return float(np.abs(tx - x).sum())


def cc(g: CSR) -> np.ndarray:
    """uint32 component label = smallest vertex id of the component."""
    lab = np.empty(g.n, dtype=np.uint32)
    _load().orc_cc(g.n, _p(g.rowptr), _p(g.colidx), _p(lab))
    return lab


def tc(g: CSR) -> int:
    """Number of triangles of the symmetric graph g."""
    return int(_load().orc_tc(g.n, _p(g.rowptr), _p(g.colidx)))


def degree_order(g: CSR) -> np.ndarray:
    """new_id[old]: decreasing degree, ties by lower old id."""
    out = np.empty(g.n, dtype=np.uint32)
    _load().orc_degree_order(g.n, _p(g.rowptr), _p(out))
    return out


def relabel(g: CSR, new_id) -> CSR:
    """The same graph with vertex v renamed new_id[v] (rows re-sorted)."""
    new_id = np.asarray(new_id, dtype=np.uint32)
    rows = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.rowptr).astype(np.int64))
    return csr_build(g.n, new_id[rows], new_id[g.colidx], g.vals, DUP_FIRST)


def tril(g: CSR) -> CSR:
    """Strictly lower triangle L of g (entries (i, j) with j < i)."""
    rows = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.rowptr).astype(np.int64))
    keep = g.colidx < rows
    return csr_build(g.n, rows[keep], g.colidx[keep],
                     g.vals[keep] if g.vals is not None else None)


def masked_LL(g: CSR):
    """(C values of C<L> = L*L over plus.pair in L's row-major order, total)."""
    nnzL = int(np.count_nonzero(
        g.colidx < np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.rowptr).astype(np.int64))))
    out = np.empty(max(nnzL, 1), dtype=np.uint32)
    total = _load().orc_masked_LL(g.n, _p(g.rowptr), _p(g.colidx), _p(out))
    return out[:nnzL], int(total)


def multi_bfs(g: CSR, sources) -> np.ndarray:
    """k x n depths: one independent BFS per source (Section 3.3, mxm as a
    multi-nodeset traversal)."""
    return np.stack([bfs(g, int(s)) for s in sources]) if len(sources) else np.zeros((0, g.n), np.int32)

