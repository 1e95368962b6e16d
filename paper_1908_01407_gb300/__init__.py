"""Python binding of libgbx.so, the GB300 (sm_103a) masked-semiring graph
library (GraphBLAST, Yang, Buluc, Owens, arXiv 1908.01407).

This module only marshals arguments: every step of every operation runs in
the CUDA library. PyTorch supplies device memory (tensors passed by
data_ptr) and streams. If libgbx.so is missing the import of the library
fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .metrics import teps  # noqa: F401  (host-side metric helpers)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbx.so")

# ----------------------------------------------------------------- enums
SUCCESS, NO_VALUE, NULL_POINTER, INVALID_VALUE, INVALID_INDEX, DOMAIN_MISMATCH, DIMENSION_MISMATCH, \
    OUT_OF_MEMORY, NOT_IMPLEMENTED, TIMEOUT, PANIC, INSUFFICIENT_SPACE = range(12)
INFO_NAMES = ["GB_SUCCESS", "GB_NO_VALUE", "GB_NULL_POINTER", "GB_INVALID_VALUE", "GB_INVALID_INDEX",
              "GB_DOMAIN_MISMATCH", "GB_DIMENSION_MISMATCH", "GB_OUT_OF_MEMORY", "GB_NOT_IMPLEMENTED",
              "GB_TIMEOUT", "GB_PANIC", "GB_INSUFFICIENT_SPACE"]
HOST, DEVICE = 0, 1
BOOL, INT32, UINT32, UINT64, FP32, FP64 = range(6)
NOP, PLUS, TIMES, MIN, MAX, LOR, LAND, FIRST, SECOND, PAIR, MINUS = range(11)
MONOID_PLUS, MONOID_TIMES, MONOID_MIN, MONOID_MAX, MONOID_LOR, MONOID_LAND = range(6)
PLUS_TIMES, LOR_LAND, MIN_PLUS, MAX_PLUS, MIN_TIMES, MIN_SECOND, PLUS_PAIR = range(7)
F_MASK, F_OUTP, F_INP0, F_INP1, F_DIRECTION, F_SWITCH_BETA, F_SCHEDULE, F_SSSP_DELTA = range(8)
SSSP_DELTA_NONE = 2**31 - 1   # no buckets: the plain changed-set iteration
DEFAULT, SCMP, STRUCTURE = 0, 1, 2
REPLACE = 1
TRAN = 1
AUTO, PUSH, PULL = 0, 1, 2
SCHED_AUTO, SCHED_GRID, SCHED_CLUSTER, SCHED_ASYNC = 0, 1, 2, 3
BUILD_DEFAULT, SYMMETRIC, CSR_ONLY = 0, 1, 2
REQ_BFS, REQ_SSSP, REQ_PAGERANK = 0, 1, 2

NP_DTYPE = {BOOL: np.uint8, INT32: np.int32, UINT32: np.uint32, UINT64: np.uint64,
            FP32: np.float32, FP64: np.float64}


class GBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        name = INFO_NAMES[code] if 0 <= code < len(INFO_NAMES) else str(code)
        super().__init__(f"{name}: {msg}")


class BfsStats(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_uint32), ("push_levels", ctypes.c_uint32), ("pull_levels", ctypes.c_uint32),
                ("status", ctypes.c_uint32), ("vertices_reached", ctypes.c_uint64),
                ("edges_examined", ctypes.c_uint64), ("frontier_edges", ctypes.c_uint64),
                ("alg_bytes", ctypes.c_uint64), ("trace_len", ctypes.c_uint32),
                ("trace_dir", ctypes.c_uint32 * 32), ("trace_vertices", ctypes.c_uint32 * 32),
                ("trace_edges", ctypes.c_uint64 * 32), ("trace_us", ctypes.c_float * 32),
                ("init_us", ctypes.c_float), ("final_us", ctypes.c_float), ("schedule", ctypes.c_uint32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("trace")}
        n = self.trace_len
        d["trace"] = [{"dir": "pull" if self.trace_dir[i] == 2 else "push", "vertices": self.trace_vertices[i],
                       "edges": self.trace_edges[i], "us": round(self.trace_us[i], 2)} for i in range(n)]
        return d


class ServerCfg(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_uint32), ("batch_window_us", ctypes.c_uint32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("pagerank_iters", ctypes.c_uint32),
                ("pagerank_damping", ctypes.c_float)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("graph_id", ctypes.c_uint32), ("src", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n", ctypes.c_uint32), ("latency_us", ctypes.c_double),
                ("batch_size", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("batched_bfs", ctypes.c_uint64), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("qps", ctypes.c_double), ("hbm_in_use", ctypes.c_uint64),
                ("hbm_peak", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_I = ctypes.c_int
_PP = ctypes.POINTER(ctypes.c_void_p)

# (name, argtypes); every function returns gb_info (int)
_SIGS = {
    "gb_init": [_I, _PP], "gb_context_set_stream": [_P, _P], "gb_context_synchronize": [_P],
    "gb_context_pool_stats": [_P, _P, _P], "gb_context_inject_alloc_failures": [_P, _U32],
    "gb_context_selftest_wait": [_P, _U32, _P],
    "gb_finalize": [_P], "gb_context_profile": [_P, _I],
    "gb_context_profile_get": [_P, ctypes.c_char_p, _P, _P], "gb_last_error": [ctypes.c_char_p, ctypes.c_size_t],
    "gb_matrix_new": [_PP, _P, _I, _U64, _U64],
    "gb_matrix_build": [_P, _P, _P, _P, _U64, _I, _I, _U32],
    "gb_matrix_nrows": [_P, _P], "gb_matrix_ncols": [_P, _P], "gb_matrix_nvals": [_P, _P],
    "gb_matrix_extract_tuples": [_P, _P, _P, _P, _P, _I],
    "gb_matrix_export_csr": [_P, _P, _P, _P, _I], "gb_matrix_export_csc": [_P, _P, _P, _P, _I],
    "gb_matrix_tril": [_P, _P], "gb_matrix_degree_order": [_P, _P, _P, _I], "gb_matrix_free": [_PP],
    "gb_vector_new": [_PP, _P, _I, _U64], "gb_vector_build": [_P, _P, _P, _U64, _I, _I],
    "gb_vector_build_dense": [_P, _P, _I], "gb_vector_fill": [_P, _P],
    "gb_vector_set_element": [_P, _U32, _P], "gb_vector_extract_element": [_P, _U32, _P],
    "gb_vector_extract_tuples": [_P, _P, _P, _P, _I], "gb_vector_extract_dense": [_P, _P, _P, _P, _I],
    "gb_vector_size": [_P, _P], "gb_vector_nvals": [_P, _P], "gb_vector_dup": [_PP, _P],
    "gb_vector_clear": [_P], "gb_vector_free": [_PP],
    "gb_desc_new": [_PP], "gb_desc_set": [_P, _I, _I], "gb_desc_get": [_P, _I, _P], "gb_desc_toggle": [_P, _I],
    "gb_desc_free": [_PP],
    "gb_mxv": [_P, _P, _I, _I, _P, _P, _P], "gb_vxm": [_P, _P, _I, _I, _P, _P, _P],
    "gb_mxm": [_P, _P, _I, _I, _P, _P, _P],
    "gb_ewise_add": [_P, _P, _I, _I, _P, _P, _P], "gb_ewise_mult": [_P, _P, _I, _I, _P, _P, _P],
    "gb_reduce_vector": [_P, _I, _I, _P], "gb_reduce_matrix": [_P, _I, _I, _P],
    "gb_reduce_rows": [_P, _P, _I, _I, _P, _P],
    "gb_bfs": [_P, _P, _U32, _P, _P, _I, _P, _P],
    "gb_bfs_noalloc": [_P, _P, _P, _P, _U32, _U64, _U32, _P, _P, _P, _P],
    "gb_bfs_autotune": [_P, _P, _P, _U32, _P, _P], "gb_bfs_set_shape": [_P, _U32, _U32],
    "gb_bfs_get_shape": [_P, _P, _P], "gb_bfs_multi": [_P, _P, _P, _U32, _P, _I, _P, _P],
    "gb_bfs_batch": [_P, _P, _P, _U32, _P, _P, _I, _P],
    "gb_sssp": [_P, _P, _U32, _P, _I, _P, _P, _P], "gb_pagerank": [_P, _P, ctypes.c_float, _U32, _P, _P, _I],
    "gb_cc": [_P, _P, _P, _I, _P, _P], "gb_tc": [_P, _P, _P, _P],
    "gb_cc_fastsv": [_P, _P, _P, _I, _P], "gb_cc_async": [_P, _P, _P, _I, _U32, _P],
    "gb_pagerank_delta": [_P, _P, ctypes.c_float, ctypes.c_float, _U32, _P, _I, _P, _P, _P],
    "gb_pagerank_autotune": [_P, _P, _P, _P, _P, _P], "gb_pagerank_set_tile": [_P, _U32],
    "gb_pagerank_set_order": [_P, _I, _U32],
    "gb_server_create": [_PP, _P, _P], "gb_server_add_graph": [_P, _P, _P], "gb_server_submit": [_P, _P, _P],
    "gb_server_wait": [_P, _U64, _U32, _P], "gb_server_fetch": [_P, _U64, _P, _I],
    "gb_server_stats_get": [_P, _P], "gb_server_destroy": [_PP],
}


def lib():
    """The loaded libgbx.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.gb_version.restype = ctypes.c_char_p
        L.gb_version.argtypes = []
        _lib = L
    return _lib


def build_library():
    """Compile libgbx.so in-tree (nvcc, sm_103a)."""
    import importlib
    return importlib.import_module(__name__ + ".build").build()


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib().gb_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(rc: int):
    if rc != SUCCESS:
        raise GBError(rc, last_error())
    return rc


def version() -> str:
    return lib().gb_version().decode()


# ---------------------------------------------------------- marshalling
def _torch():
    import torch
    return torch


def _ptr_mem(x):
    """(pointer, gb_mem, keepalive) for a torch tensor or numpy array."""
    if x is None:
        return None, HOST, None
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x)
        return x.ctypes.data, HOST, x
    torch = _torch()
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (DEVICE if x.is_cuda else HOST), x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _out_mem(x):
    p, mem, keep = _ptr_mem(x)
    if isinstance(keep, np.ndarray) and keep is not x:
        raise ValueError("output numpy array must be contiguous")
    return p, mem


class Context:
    """gb_context: one GPU, one stream, a device memory pool."""

    def __init__(self, device: int = 0, stream=None):
        h = ctypes.c_void_p()
        check(lib().gb_init(device, ctypes.byref(h)))
        self.h = h
        self.device = device
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (legacy default)."""
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        check(lib().gb_context_set_stream(self.h, ctypes.c_void_p(stream or 0)))

    def use_torch_stream(self):
        torch = _torch()
        self.set_stream(torch.cuda.current_stream(self.device))

    def synchronize(self):
        check(lib().gb_context_synchronize(self.h))

    def pool_stats(self):
        held, peak = ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().gb_context_pool_stats(self.h, ctypes.byref(held), ctypes.byref(peak)))
        return held.value, peak.value

    def profile(self, enable: bool):
        """Start (clearing old records) or stop per-kernel event timing."""
        check(lib().gb_context_profile(self.h, 1 if enable else 0))

    def profile_get(self, kernel: str):
        """(total milliseconds, launches) recorded for `kernel`."""
        ms, k = ctypes.c_double(), ctypes.c_uint64()
        check(lib().gb_context_profile_get(self.h, kernel.encode(), ctypes.byref(ms), ctypes.byref(k)))
        return ms.value, k.value

    def inject_alloc_failures(self, count: int):
        check(lib().gb_context_inject_alloc_failures(self.h, count))

    def selftest_wait(self, limit_us: int) -> int:
        """Run the bounded-wait self-test; returns the status word the
        waiting block recorded (TIMEOUT when the wait ran out as it must)."""
        st = ctypes.c_int32(-1)
        check(lib().gb_context_selftest_wait(self.h, limit_us, ctypes.byref(st)))
        return st.value

    def close(self):
        if self.h:
            check(lib().gb_finalize(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Matrix:
    """gb_matrix: CSR + CSC on the device."""

    def __init__(self, ctx: Context, type_: int, nrows: int, ncols: int):
        h = ctypes.c_void_p()
        check(lib().gb_matrix_new(ctypes.byref(h), ctx.h, type_, nrows, ncols))
        self.h, self.ctx, self.type = h, ctx, type_

    @classmethod
    def from_tuples(cls, ctx, nrows, rows, cols, vals=None, type_=None, dup=FIRST, flags=BUILD_DEFAULT,
                    ncols=None):
        if type_ is None:
            type_ = UINT32
        A = cls(ctx, type_, nrows, nrows if ncols is None else ncols)
        A.build(rows, cols, vals, dup, flags)
        return A

    def build(self, rows, cols, vals=None, dup=FIRST, flags=BUILD_DEFAULT):
        pr, mr, kr = _ptr_mem(rows)
        pc, mc, kc = _ptr_mem(cols)
        pv, mv, kv = _ptr_mem(vals)
        n = int(kr.shape[0])
        if mr != mc or (vals is not None and mv != mr):
            raise ValueError("rows, cols and vals must all be on the host or all on the device")
        check(lib().gb_matrix_build(self.h, pr, pc, pv, n, dup, mr, flags))

    def _q(self, f):
        v = ctypes.c_uint64()
        check(f(self.h, ctypes.byref(v)))
        return v.value

    @property
    def nrows(self):
        return self._q(lib().gb_matrix_nrows)

    @property
    def ncols(self):
        return self._q(lib().gb_matrix_ncols)

    @property
    def nvals(self):
        return self._q(lib().gb_matrix_nvals)

    def export_csr(self, with_vals=False):
        """(rowptr, colidx[, vals]) as host numpy arrays."""
        n, m = self.nrows, self.nvals
        rp = np.empty(n + 1, np.uint32)
        ci = np.empty(max(m, 1), np.uint32)
        v = np.empty(max(m, 1), NP_DTYPE[self.type]) if with_vals else None
        check(lib().gb_matrix_export_csr(self.h, rp.ctypes.data, ci.ctypes.data,
                                         v.ctypes.data if v is not None else None, HOST))
        return (rp, ci[:m]) + ((v[:m],) if with_vals else ())

    def export_csc(self, with_vals=False):
        n, m = self.ncols, self.nvals
        cp = np.empty(n + 1, np.uint32)
        ri = np.empty(max(m, 1), np.uint32)
        v = np.empty(max(m, 1), NP_DTYPE[self.type]) if with_vals else None
        check(lib().gb_matrix_export_csc(self.h, cp.ctypes.data, ri.ctypes.data,
                                         v.ctypes.data if v is not None else None, HOST))
        return (cp, ri[:m]) + ((v[:m],) if with_vals else ())

    def extract_tuples(self, with_vals=False):
        m = self.nvals
        r = np.empty(max(m, 1), np.uint32)
        c = np.empty(max(m, 1), np.uint32)
        v = np.empty(max(m, 1), NP_DTYPE[self.type]) if with_vals else None
        cnt = ctypes.c_uint64(max(m, 1))
        check(lib().gb_matrix_extract_tuples(self.h, r.ctypes.data, c.ctypes.data,
                                             v.ctypes.data if v is not None else None, ctypes.byref(cnt), HOST))
        k = cnt.value
        return (r[:k], c[:k]) + ((v[:k],) if with_vals else ())

    def tril(self):
        L = Matrix(self.ctx, self.type, self.nrows, self.ncols)
        check(lib().gb_matrix_tril(L.h, self.h))
        return L

    def degree_order(self):
        """(B, new_id): the matrix relabelled by decreasing degree."""
        B = Matrix(self.ctx, self.type, self.nrows, self.ncols)
        nid = np.empty(max(self.nrows, 1), np.uint32)
        check(lib().gb_matrix_degree_order(B.h, self.h, nid.ctypes.data, HOST))
        return B, nid[:self.nrows]

    def free(self):
        if self.h:
            check(lib().gb_matrix_free(ctypes.byref(self.h)))
            self.h = None


class Vector:
    """gb_vector: dense values + presence bitmap (+ sparse list)."""

    def __init__(self, ctx: Context, type_: int, n: int):
        h = ctypes.c_void_p()
        check(lib().gb_vector_new(ctypes.byref(h), ctx.h, type_, n))
        self.h, self.ctx, self.type, self.n = h, ctx, type_, n

    def _scalar(self, x):
        a = np.array([x], dtype=NP_DTYPE[self.type])
        return a, a.ctypes.data

    def build(self, idx, vals=None, dup=FIRST):
        pi, mi, ki = _ptr_mem(idx)
        pv, mv, kv = _ptr_mem(vals)
        if vals is not None and mv != mi:
            raise ValueError("idx and vals must both be host or both device")
        check(lib().gb_vector_build(self.h, pi, pv, int(ki.shape[0]), dup, mi))
        return self

    def build_dense(self, vals):
        pv, mv, kv = _ptr_mem(vals)
        check(lib().gb_vector_build_dense(self.h, pv, mv))
        return self

    def fill(self, x):
        keep, p = self._scalar(x)
        check(lib().gb_vector_fill(self.h, p))
        return self

    def set_element(self, i, x):
        keep, p = self._scalar(x)
        check(lib().gb_vector_set_element(self.h, i, p))

    def extract_element(self, i):
        out = np.zeros(1, NP_DTYPE[self.type])
        rc = lib().gb_vector_extract_element(self.h, i, out.ctypes.data)
        if rc == NO_VALUE:
            return None
        check(rc)
        return out[0].item()

    @property
    def nvals(self):
        v = ctypes.c_uint64()
        check(lib().gb_vector_nvals(self.h, ctypes.byref(v)))
        return v.value

    @property
    def size(self):
        v = ctypes.c_uint64()
        check(lib().gb_vector_size(self.h, ctypes.byref(v)))
        return v.value

    def extract_tuples(self):
        k = max(self.nvals, 1)
        idx = np.empty(k, np.uint32)
        vals = np.empty(k, NP_DTYPE[self.type])
        cnt = ctypes.c_uint64(k)
        check(lib().gb_vector_extract_tuples(self.h, idx.ctypes.data, vals.ctypes.data, ctypes.byref(cnt), HOST))
        return idx[:cnt.value], vals[:cnt.value]

    def to_dict(self):
        i, v = self.extract_tuples()
        return {int(a): b.item() for a, b in zip(i, v)}

    def extract_dense(self, absent=0):
        vals = np.empty(max(self.n, 1), NP_DTYPE[self.type])
        pres = np.empty(max(self.n, 1), np.uint8)
        keep, p = self._scalar(absent)
        check(lib().gb_vector_extract_dense(self.h, vals.ctypes.data, pres.ctypes.data, p, HOST))
        return vals[:self.n], pres[:self.n]

    def dup(self):
        h = ctypes.c_void_p()
        check(lib().gb_vector_dup(ctypes.byref(h), self.h))
        v = Vector.__new__(Vector)
        v.h, v.ctx, v.type, v.n = h, self.ctx, self.type, self.n
        return v

    def clear(self):
        check(lib().gb_vector_clear(self.h))
        return self

    def free(self):
        if self.h:
            check(lib().gb_vector_free(ctypes.byref(self.h)))
            self.h = None


class Descriptor:
    def __init__(self, **fields):
        h = ctypes.c_void_p()
        check(lib().gb_desc_new(ctypes.byref(h)))
        self.h = h
        names = {"mask": F_MASK, "outp": F_OUTP, "inp0": F_INP0, "inp1": F_INP1,
                 "direction": F_DIRECTION, "beta": F_SWITCH_BETA, "schedule": F_SCHEDULE,
                 "sssp_delta": F_SSSP_DELTA}
        for k, v in fields.items():
            self.set(names[k], v)

    def set(self, field, value):
        check(lib().gb_desc_set(self.h, field, value))
        return self

    def get(self, field):
        v = ctypes.c_int()
        check(lib().gb_desc_get(self.h, field, ctypes.byref(v)))
        return v.value

    def toggle(self, field):
        check(lib().gb_desc_toggle(self.h, field))
        return self

    def free(self):
        if self.h:
            check(lib().gb_desc_free(ctypes.byref(self.h)))
            self.h = None


def _h(x):
    return x.h if x is not None else None


# ------------------------------------------------------------ operations
def mxv(w, mask, accum, semiring, A, u, desc=None):
    check(lib().gb_mxv(w.h, _h(mask), accum, semiring, A.h, u.h, _h(desc)))
    return w


def vxm(w, mask, accum, semiring, u, A, desc=None):
    check(lib().gb_vxm(w.h, _h(mask), accum, semiring, u.h, A.h, _h(desc)))
    return w


def mxm(C, M, accum, semiring, A, B, desc=None):
    check(lib().gb_mxm(C.h, _h(M), accum, semiring, A.h, B.h, _h(desc)))
    return C


def ewise_add(w, mask, accum, op, u, v, desc=None):
    check(lib().gb_ewise_add(w.h, _h(mask), accum, op, u.h, v.h, _h(desc)))
    return w


def ewise_mult(w, mask, accum, op, u, v, desc=None):
    check(lib().gb_ewise_mult(w.h, _h(mask), accum, op, u.h, v.h, _h(desc)))
    return w


def reduce_vector(u, monoid, accum=NOP, init=None):
    out = np.zeros(1, NP_DTYPE[u.type])
    if init is not None:
        out[0] = init
    check(lib().gb_reduce_vector(out.ctypes.data, accum, monoid, u.h))
    return out[0].item()


def reduce_matrix(A, monoid, accum=NOP, init=None):
    out = np.zeros(1, NP_DTYPE[A.type])
    if init is not None:
        out[0] = init
    check(lib().gb_reduce_matrix(out.ctypes.data, accum, monoid, A.h))
    return out[0].item()


def reduce_rows(w, mask, accum, monoid, A, desc=None):
    check(lib().gb_reduce_rows(w.h, _h(mask), accum, monoid, A.h, _h(desc)))
    return w


# ------------------------------------------------------------ algorithms
def bfs(ctx, A, src, levels=None, parents=None, desc=None, stats=True):
    """Direction-optimised BFS. levels/parents: caller buffers (torch CUDA
    tensors or numpy arrays) of nrows int32, or None to get new CUDA tensors.
    Returns (levels, parents, stats-dict or None)."""
    n = A.nrows
    if levels is None:
        torch = _torch()
        levels = torch.empty(n, dtype=torch.int32, device=f"cuda:{ctx.device}")
        if parents is None and parents is not False:
            parents = torch.empty(n, dtype=torch.int32, device=f"cuda:{ctx.device}")
    if parents is False:
        parents = None
    pl, ml = _out_mem(levels)
    pp, mp = _out_mem(parents) if parents is not None else (None, ml)
    if parents is not None and mp != ml:
        raise ValueError("levels and parents must both be host or both device")
    st = BfsStats()
    check(lib().gb_bfs(ctx.h, A.h, src, pl, pp, ml, _h(desc), ctypes.byref(st) if stats else None))
    return levels, parents, (st.as_dict() if stats else None)


def bfs_set_shape(A, pull_width=0, blocks_per_sm=0):
    """BFS tile shape of A: pull candidates per lane (0 = default, 1, 2, 4)
    and blocks per SM (0 = as many as fit, 1..4)."""
    check(lib().gb_bfs_set_shape(A.h, pull_width, blocks_per_sm))


def bfs_get_shape(A):
    """(pull width in effect, blocks per SM or 0 = as many as fit) of A."""
    w = ctypes.c_uint32()
    b = ctypes.c_uint32()
    check(lib().gb_bfs_get_shape(A.h, ctypes.byref(w), ctypes.byref(b)))
    return w.value, b.value


def bfs_autotune(ctx, A, srcs):
    """Pick the push/pull switch beta for A from timed BFS runs; returns
    (beta, mean ms per BFS at that beta). The choice is kept on A."""
    srcs = np.ascontiguousarray(srcs, dtype=np.uint32)
    b = ctypes.c_uint32()
    ms = ctypes.c_double()
    check(lib().gb_bfs_autotune(ctx.h, A.h, srcs.ctypes.data, int(srcs.shape[0]), ctypes.byref(b),
                                ctypes.byref(ms)))
    return b.value, ms.value


def _header_define(name: str) -> int:
    """Value of a numeric #define of include/gbx.h (the one place a limit of
    the C ABI is stated)."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gbx.h")
    m = re.search(r"#define\s+" + name + r"\s+(\d+)u?", open(hdr).read())
    if not m:
        raise RuntimeError(f"{name} is not defined in {hdr}")
    return int(m.group(1))


NOALLOC_MAX_VERTICES = _header_define("GB_NOALLOC_MAX_VERTICES")


def bfs_noalloc(rowptr, colidx, colptr, rowidx, n, nnz, src, levels, parents=None, status=None, stream=None):
    """gb_bfs_noalloc: BFS with the library's built-in scratch (no device
    allocation on the call path). All arrays are CUDA tensors; colidx and
    rowidx must be 16-byte aligned and readable 16 bytes past their end.
    status: an int32 CUDA tensor of one element (or None) that receives the
    kernel's exit status (0, or GB_TIMEOUT when a bounded wait ran out).
    stream: a torch.cuda.Stream (default: the current stream)."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    ptrs = [x.data_ptr() if x is not None else None
            for x in (rowptr, colidx, colptr, rowidx, levels, parents, status)]
    check(lib().gb_bfs_noalloc(ptrs[0], ptrs[1], ptrs[2], ptrs[3], n, nnz, src, ptrs[4], ptrs[5], ptrs[6],
                               ctypes.c_void_p(stream.cuda_stream)))
    return levels, parents


def bfs_batch(ctx, A, srcs, levels=None, parents=None, desc=None):
    """gb_bfs_batch: one direction-optimised BFS per source; row q of the
    k x nrows int32 levels/parents (torch CUDA tensors or host arrays, e.g.
    pinned CPU tensors) is source q's result. Host outputs are copied while
    the next run traverses. parents=False skips parents."""
    srcs = np.ascontiguousarray(srcs, dtype=np.uint32)
    k, n = int(srcs.shape[0]), A.nrows
    if levels is None:
        torch = _torch()
        levels = torch.empty((k, n), dtype=torch.int32, device=f"cuda:{ctx.device}")
        if parents is None:
            parents = torch.empty((k, n), dtype=torch.int32, device=f"cuda:{ctx.device}")
    if parents is False:
        parents = None
    pl, ml = _out_mem(levels)
    pp, mp = _out_mem(parents) if parents is not None else (None, ml)
    if parents is not None and mp != ml:
        raise ValueError("levels and parents must both be host or both device")
    check(lib().gb_bfs_batch(ctx.h, A.h, srcs.ctypes.data, k, pl, pp, ml, _h(desc)))
    return levels, parents


def bfs_multi(ctx, A, srcs, levels=None, desc=None, stats=True):
    srcs = np.ascontiguousarray(srcs, dtype=np.uint32)
    k, n = int(srcs.shape[0]), A.nrows
    if levels is None:
        torch = _torch()
        levels = torch.empty((k, n), dtype=torch.int32, device=f"cuda:{ctx.device}")
    pl, ml = _out_mem(levels)
    st = BfsStats()
    check(lib().gb_bfs_multi(ctx.h, A.h, srcs.ctypes.data, k, pl, ml, _h(desc),
                             ctypes.byref(st) if stats else None))
    return levels, (st.as_dict() if stats else None)


def sssp(ctx, A, src, dist=None, desc=None, stats=False):
    """SSSP; returns (dist, iterations), or (dist, iterations, stats-dict)
    with stats=True."""
    n = A.nrows
    if dist is None:
        torch = _torch()
        dist = torch.empty(n, dtype=torch.int32, device=f"cuda:{ctx.device}")
    pd, md = _out_mem(dist)
    it = ctypes.c_uint32()
    st = BfsStats()
    check(lib().gb_sssp(ctx.h, A.h, src, pd, md, _h(desc), ctypes.byref(it), ctypes.byref(st) if stats else None))
    return (dist, it.value, st.as_dict()) if stats else (dist, it.value)


def pagerank(ctx, A, damping=0.85, iters=50, rank=None, residuals=True):
    n = A.nrows
    if rank is None:
        torch = _torch()
        rank = torch.empty(n, dtype=torch.float32, device=f"cuda:{ctx.device}")
    pr, mr = _out_mem(rank)
    res = np.empty(max(iters, 1), np.float64) if residuals else None
    check(lib().gb_pagerank(ctx.h, A.h, damping, iters, pr, res.ctypes.data if res is not None else None, mr))
    return rank, (res[:iters] if res is not None else None)


def pagerank_autotune(ctx, A):
    """Pick the PageRank SpMV layout for A from timed runs; returns (tile
    nonzeros, degree order 0/1, staged ranks, ms per iteration). The choice
    is kept on A."""
    t = ctypes.c_uint32()
    o = ctypes.c_int32()
    k = ctypes.c_uint32()
    ms = ctypes.c_double()
    check(lib().gb_pagerank_autotune(ctx.h, A.h, ctypes.byref(t), ctypes.byref(o), ctypes.byref(k), ctypes.byref(ms)))
    return t.value, o.value, k.value, ms.value


def pagerank_set_tile(A, tile_nnz):
    check(lib().gb_pagerank_set_tile(A.h, tile_nnz))


def pagerank_set_order(A, degree_order, staged_ranks=0):
    """0: PageRank runs on A as stored; 1: on its degree-ordered copy with
    staged_ranks ranks in shared memory (0 = the default)."""
    check(lib().gb_pagerank_set_order(A.h, degree_order, staged_ranks))


def pagerank_delta(ctx, A, damping=0.85, eps=1e-4, max_iters=100, rank=None):
    """Adaptive PageRank (PageRankDelta). Returns (rank, iterations,
    residuals[iterations], active[iterations])."""
    n = A.nrows
    if rank is None:
        torch = _torch()
        rank = torch.empty(n, dtype=torch.float32, device=f"cuda:{ctx.device}")
    pr, mr = _out_mem(rank)
    it = ctypes.c_uint32()
    res = np.zeros(max(max_iters, 1), np.float64)
    act = np.zeros(max(max_iters, 1), np.uint32)
    check(lib().gb_pagerank_delta(ctx.h, A.h, damping, eps, max_iters, pr, mr, ctypes.byref(it),
                                  res.ctypes.data, act.ctypes.data))
    k = it.value
    return rank, k, res[:k], act[:k]


def cc_fastsv(ctx, A, labels=None):
    """Connected components by FastSV; returns (labels, iterations)."""
    n = A.nrows
    if labels is None:
        torch = _torch()
        labels = torch.empty(n, dtype=torch.int32, device=f"cuda:{ctx.device}")
    pl, ml = _out_mem(labels)
    it = ctypes.c_uint32()
    check(lib().gb_cc_fastsv(ctx.h, A.h, pl, ml, ctypes.byref(it)))
    return labels, it.value


def cc(ctx, A, labels=None):
    n = A.nrows
    if labels is None:
        torch = _torch()
        labels = torch.empty(n, dtype=torch.int32, device=f"cuda:{ctx.device}")
    pl, ml = _out_mem(labels)
    it = ctypes.c_uint32()
    check(lib().gb_cc(ctx.h, A.h, pl, ml, ctypes.byref(it), None))
    return labels, it.value


def cc_async(ctx, A, labels=None, stats=False, bucket=0):
    """Connected components by min-label propagation without level
    barriers, labels taken in buckets of `bucket` values (0 = automatic,
    nrows or more = one bucket); returns labels, or (labels, stats-dict)
    with stats=True."""
    n = A.nrows
    if labels is None:
        torch = _torch()
        labels = torch.empty(n, dtype=torch.int32, device=f"cuda:{ctx.device}")
    pl, ml = _out_mem(labels)
    st = BfsStats()
    check(lib().gb_cc_async(ctx.h, A.h, pl, ml, bucket, ctypes.byref(st) if stats else None))
    return (labels, st.as_dict()) if stats else labels


def tc(ctx, L, C=None):
    cnt = ctypes.c_uint64()
    check(lib().gb_tc(ctx.h, L.h, ctypes.byref(cnt), _h(C)))
    return cnt.value


class Server:
    """gb_server: batched, continuously admitting request loop."""

    def __init__(self, ctx, max_inflight=8, batch_window_us=200, hbm_budget_bytes=0, pagerank_iters=50,
                 pagerank_damping=0.85):
        cfg = ServerCfg(max_inflight, batch_window_us, hbm_budget_bytes, pagerank_iters, pagerank_damping)
        h = ctypes.c_void_p()
        check(lib().gb_server_create(ctypes.byref(h), ctx.h, ctypes.byref(cfg)))
        self.h, self.ctx = h, ctx
        self.graphs = []

    def add_graph(self, A):
        gid = ctypes.c_uint32()
        check(lib().gb_server_add_graph(self.h, A.h, ctypes.byref(gid)))
        self.graphs.append(A)
        return gid.value

    def submit(self, kind, graph_id, src=0):
        req = Request(kind, graph_id, src)
        t = ctypes.c_uint64()
        check(lib().gb_server_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def wait(self, ticket, timeout_ms=60000):
        r = Result()
        check(lib().gb_server_wait(self.h, ticket, timeout_ms, ctypes.byref(r)))
        return r

    def fetch(self, ticket, n, kind):
        dt = {REQ_BFS: np.int32, REQ_SSSP: np.uint32, REQ_PAGERANK: np.float32}[kind]
        out = np.empty(max(n, 1), dt)
        check(lib().gb_server_fetch(self.h, ticket, out.ctypes.data, HOST))
        return out[:n]

    def fetch_into(self, ticket, out):
        """Copy a finished result into a caller buffer (torch tensor or numpy array)."""
        p, mem = _out_mem(out)
        check(lib().gb_server_fetch(self.h, ticket, p, mem))
        return out

    def stats(self):
        s = ServerStats()
        check(lib().gb_server_stats_get(self.h, ctypes.byref(s)))
        return s.as_dict()

    def destroy(self):
        if self.h:
            check(lib().gb_server_destroy(ctypes.byref(self.h)))
            self.h = None
