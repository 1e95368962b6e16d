"""ORACLE -- test infrastructure only.

Semantics of the generic GraphBLAS operations as plain Python loops over
dictionaries, for small inputs. Written from Section 3 of the GraphBLAST
paper: semirings and monoids (Section 3.1.3-3.1.4, Table 5), masking and its
structural complement (Section 3.2.1), the descriptor (Table 6), and the
operations of Table 7 (mxv, vxm, mxm, eWiseAdd, eWiseMult, reduce).

Readings where the paper is silent:
* accum: the paper ignores it (Section 3.6); here w = accum(w, t) on the
  positions the mask lets through, as the GraphBLAS C API defines it.
* REPLACE: the paper leaves it out (Section 3.6); here positions outside the
  mask are cleared when it is set.
* No mask allows every position; the complement of no mask allows none.
* A matrix built without values is structural: every stored entry is 1.
* MIN_PLUS / MAX_PLUS on integer types add with saturation, so the
  additive identity (type max / type min) absorbs like +-infinity.
* Integer PLUS/TIMES wrap modulo 2^bits (two's complement for int32).
* Floating-point types are computed here in double precision.
"""
from __future__ import annotations

import math

TYPES = ("bool", "int32", "uint32", "uint64", "fp32", "fp64")

_BITS = {"int32": 32, "uint32": 32, "uint64": 64}


def tmax(t):
    return {"bool": True, "int32": 2**31 - 1, "uint32": 2**32 - 1, "uint64": 2**64 - 1,
            "fp32": math.inf, "fp64": math.inf}[t]


def tmin(t):
    return {"bool": False, "int32": -2**31, "uint32": 0, "uint64": 0,
            "fp32": -math.inf, "fp64": -math.inf}[t]


def cast(t, x):
    if t == "bool":
        return bool(x)
    if t in ("fp32", "fp64"):
        return float(x)
    x = int(x)
    b = _BITS[t]
    x &= (1 << b) - 1
    if t == "int32" and x >= 2**31:
        x -= 2**32
    return x


def _sat_add(t, a, b):
    if t in ("fp32", "fp64"):
        return a + b
    if t == "bool":
        return bool(a) or bool(b)
    return max(tmin(t), min(tmax(t), int(a) + int(b)))


BINOPS = {
    "PLUS": lambda t, a, b: cast(t, a + b) if t != "bool" else (bool(a) or bool(b)),
    "TIMES": lambda t, a, b: cast(t, a * b) if t != "bool" else (bool(a) and bool(b)),
    "MIN": lambda t, a, b: min(a, b),
    "MAX": lambda t, a, b: max(a, b),
    "LOR": lambda t, a, b: cast(t, bool(a) or bool(b)),
    "LAND": lambda t, a, b: cast(t, bool(a) and bool(b)),
    "FIRST": lambda t, a, b: a,
    "SECOND": lambda t, a, b: b,
    "PAIR": lambda t, a, b: cast(t, 1),
    "MINUS": lambda t, a, b: cast(t, a - b) if t != "bool" else (bool(a) != bool(b)),
}

# monoid: (binop name, identity as a function of type)
MONOIDS = {
    "PLUS": ("PLUS", lambda t: cast(t, 0)),
    "TIMES": ("TIMES", lambda t: cast(t, 1)),
    "MIN": ("MIN", tmax),
    "MAX": ("MAX", tmin),
    "LOR": ("LOR", lambda t: cast(t, 0)),
    "LAND": ("LAND", lambda t: cast(t, 1)),
}

# semiring: (add monoid, multiply op); Table 5 plus the two used by the
# connected-components and triangle-counting listings (min.second, plus.pair)
SEMIRINGS = {
    "PLUS_TIMES": ("PLUS", "TIMES"),
    "LOR_LAND": ("LOR", "LAND"),
    "MIN_PLUS": ("MIN", "SATPLUS"),
    "MAX_PLUS": ("MAX", "SATPLUS"),
    "MIN_TIMES": ("MIN", "TIMES"),
    "MIN_SECOND": ("MIN", "SECOND"),
    "PLUS_PAIR": ("PLUS", "PAIR"),
}


def mult(sr, t, a, b):
    op = SEMIRINGS[sr][1]
    if op == "SATPLUS":
        return _sat_add(t, a, b)
    return BINOPS[op](t, a, b)


def add(sr, t, a, b):
    return BINOPS[MONOIDS[SEMIRINGS[sr][0]][0]](t, a, b)


def identity(sr, t):
    return MONOIDS[SEMIRINGS[sr][0]][1](t)


class Vec:
    """Sparse vector: size n, {index: value}, element type."""

    def __init__(self, n, t, entries=None):
        self.n, self.t = n, t
        self.e = dict(entries or {})

    def copy(self):
        return Vec(self.n, self.t, self.e)


class Mat:
    """Sparse matrix: nrows x ncols, {(i, j): value}; structural if t is None
    at build time (every stored value is then 1)."""

    def __init__(self, nrows, ncols, t, entries=None):
        self.nrows, self.ncols, self.t = nrows, ncols, t
        self.e = dict(entries or {})

    def T(self):
        return Mat(self.ncols, self.nrows, self.t, {(j, i): v for (i, j), v in self.e.items()})

    def rows(self):
        r = {}
        for (i, j), v in self.e.items():
            r.setdefault(i, {})[j] = v
        return r


def mask_allows(mask_e, i, structural, scmp):
    """Section 3.2.1: a stored nonzero lets the output through; the
    structural complement inverts that. With `structural` only presence
    counts. A missing mask allows everything, and its complement nothing
    (GraphBLAS C API reading of GrB_COMP with no mask)."""
    if mask_e is None:
        return not scmp
    if structural:
        m = i in mask_e
    else:
        m = i in mask_e and bool(mask_e[i])
    return (not m) if scmp else m


def _finish(w_e, t_e, allowed, accum, t, replace, keys):
    """Merge the product t into w on allowed positions (accum optional)."""
    out = {}
    for i in keys:
        if allowed(i):
            if accum is not None:
                if i in w_e and i in t_e:
                    out[i] = BINOPS[accum](t, w_e[i], t_e[i])
                elif i in w_e:
                    out[i] = w_e[i]
                elif i in t_e:
                    out[i] = t_e[i]
            elif i in t_e:
                out[i] = t_e[i]
        elif not replace and i in w_e:
            out[i] = w_e[i]
    return out


def mxv(w: Vec, mask: Vec | None, accum, sr, A: Mat, u: Vec, *, tran=False,
        structural=False, scmp=False, replace=False) -> Vec:
    """w<mask> = accum(w, A (+).(x) u) (Table 7 mxv; TRAN uses A^T)."""
    if tran:
        A = A.T()
    t = w.t
    prod = {}
    for (i, j), a in A.e.items():
        if j in u.e:
            term = mult(sr, t, cast(t, a), cast(t, u.e[j]))
            prod[i] = add(sr, t, prod[i], term) if i in prod else term
    keys = range(w.n)
    me = mask.e if mask is not None else None
    return Vec(w.n, t, _finish(w.e, prod, lambda i: mask_allows(me, i, structural, scmp),
                               accum, t, replace, keys))


def vxm(w: Vec, mask: Vec | None, accum, sr, u: Vec, A: Mat, *, tran=False,
        structural=False, scmp=False, replace=False) -> Vec:
    """w<mask> = accum(w, u (+).(x) A): w(j) = (+)_i u(i) (x) A(i,j)."""
    if tran:
        A = A.T()
    t = w.t
    prod = {}
    for (i, j), a in A.e.items():
        if i in u.e:
            term = mult(sr, t, cast(t, u.e[i]), cast(t, a))
            prod[j] = add(sr, t, prod[j], term) if j in prod else term
    me = mask.e if mask is not None else None
    return Vec(w.n, t, _finish(w.e, prod, lambda i: mask_allows(me, i, structural, scmp),
                               accum, t, replace, range(w.n)))


def mxm(C: Mat, M: Mat | None, accum, sr, A: Mat, B: Mat, *, tran0=False, tran1=False,
        structural=False, scmp=False, replace=False) -> Mat:
    """C<M> = accum(C, A (+).(x) B) (Table 7 mxm; Section 6.3.4 masked SpGEMM)."""
    if tran0:
        A = A.T()
    if tran1:
        B = B.T()
    t = C.t
    arows, brows = A.rows(), B.rows()
    prod = {}
    for i, ar in arows.items():
        for k, a in ar.items():
            for j, b in brows.get(k, {}).items():
                term = mult(sr, t, cast(t, a), cast(t, b))
                prod[(i, j)] = add(sr, t, prod[(i, j)], term) if (i, j) in prod else term
    keys = [(i, j) for i in range(C.nrows) for j in range(C.ncols)]
    me = M.e if M is not None else None
    return Mat(C.nrows, C.ncols, t,
               _finish(C.e, prod, lambda ij: mask_allows(me, ij, structural, scmp),
                       accum, t, replace, keys))


def ewise_add(w: Vec, mask, accum, op, u: Vec, v: Vec, *, structural=False, scmp=False,
              replace=False) -> Vec:
    """Union: op where both present, the present value otherwise (Table 7)."""
    t = w.t
    prod = {}
    for i in set(u.e) | set(v.e):
        if i in u.e and i in v.e:
            prod[i] = BINOPS[op](t, cast(t, u.e[i]), cast(t, v.e[i]))
        else:
            prod[i] = cast(t, u.e[i] if i in u.e else v.e[i])
    me = mask.e if mask is not None else None
    return Vec(w.n, t, _finish(w.e, prod, lambda i: mask_allows(me, i, structural, scmp),
                               accum, t, replace, range(w.n)))


def ewise_mult(w: Vec, mask, accum, op, u: Vec, v: Vec, *, structural=False, scmp=False,
               replace=False) -> Vec:
    """Intersection: op where both present (Table 7)."""
    t = w.t
    prod = {i: BINOPS[op](t, cast(t, u.e[i]), cast(t, v.e[i])) for i in set(u.e) & set(v.e)}
    me = mask.e if mask is not None else None
    return Vec(w.n, t, _finish(w.e, prod, lambda i: mask_allows(me, i, structural, scmp),
                               accum, t, replace, range(w.n)))


def reduce_vector(t, monoid, u: Vec):
    """Monoid reduction of the stored values to a scalar (Table 7 reduce)."""
    op, ident = MONOIDS[monoid]
    acc = ident(t)
    for i in sorted(u.e):
        acc = BINOPS[op](t, acc, cast(t, u.e[i]))
    return acc


def reduce_matrix(t, monoid, A: Mat):
    op, ident = MONOIDS[monoid]
    acc = ident(t)
    for k in sorted(A.e):
        acc = BINOPS[op](t, acc, cast(t, A.e[k]))
    return acc


def reduce_rows(w: Vec, mask, accum, monoid, A: Mat, *, tran=False, structural=False,
                scmp=False, replace=False) -> Vec:
    """w(i) = (+)_j A(i, j) over stored entries, starting from the monoid's
    identity; rows without entries give no value (Table 7 reduce to vector)."""
    if tran:
        A = A.T()
    t = w.t
    op, ident = MONOIDS[monoid]
    prod = {}
    for (i, j) in sorted(A.e):
        a = cast(t, A.e[(i, j)])
        prod[i] = BINOPS[op](t, prod[i] if i in prod else ident(t), a)
    me = mask.e if mask is not None else None
    return Vec(w.n, t, _finish(w.e, prod, lambda i: mask_allows(me, i, structural, scmp),
                               accum, t, replace, range(w.n)))
