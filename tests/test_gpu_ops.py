"""GPU parity of the generic operations (mxv, vxm, mxm, eWiseAdd, eWiseMult,
reduce) against the oracle's plain semantics (oracle/graphblas.py), over
seeded random cases covering every supported (semiring, type) pair, both
directions, every mask form, accumulators, REPLACE and transposes."""
import itertools
import math

import numpy as np
import pytest

import paper_1908_01407_gb300 as gb
from oracle import graphblas as gbo

pytestmark = pytest.mark.gpu

SUPPORTED = {
    "PLUS_TIMES": ["int32", "uint32", "fp32", "fp64"],
    "MIN_PLUS": ["int32", "uint32", "fp32", "fp64"],
    "MIN_TIMES": ["int32", "uint32", "fp32", "fp64"],
    "MAX_PLUS": ["int32", "fp32", "fp64"],
    "LOR_LAND": ["bool"],
    "MIN_SECOND": ["int32", "uint32", "fp32", "fp64"],
    "PLUS_PAIR": ["int32", "uint32", "uint64", "fp32"],
}
GBT = {"bool": gb.BOOL, "int32": gb.INT32, "uint32": gb.UINT32, "uint64": gb.UINT64, "fp32": gb.FP32,
       "fp64": gb.FP64}
SR = {"PLUS_TIMES": gb.PLUS_TIMES, "LOR_LAND": gb.LOR_LAND, "MIN_PLUS": gb.MIN_PLUS, "MAX_PLUS": gb.MAX_PLUS,
      "MIN_TIMES": gb.MIN_TIMES, "MIN_SECOND": gb.MIN_SECOND, "PLUS_PAIR": gb.PLUS_PAIR}
BOP = {"PLUS": gb.PLUS, "TIMES": gb.TIMES, "MIN": gb.MIN, "MAX": gb.MAX, "LOR": gb.LOR, "LAND": gb.LAND,
       "FIRST": gb.FIRST, "SECOND": gb.SECOND, "PAIR": gb.PAIR, "MINUS": gb.MINUS}
MON = {"PLUS": gb.MONOID_PLUS, "TIMES": gb.MONOID_TIMES, "MIN": gb.MONOID_MIN, "MAX": gb.MONOID_MAX,
       "LOR": gb.MONOID_LOR, "LAND": gb.MONOID_LAND}


def rand_val(rng, t):
    if t == "bool":
        return bool(rng.integers(0, 2))
    if t in ("uint32", "uint64"):
        return int(rng.integers(0, 20))
    if t == "int32":
        return int(rng.integers(-9, 10))
    if t == "fp32":
        return float(np.float32(rng.uniform(-9, 9)))   # a value FP32 holds exactly
    return float(rng.uniform(-9, 9))


# Floating-point outputs are compared with a bound derived from the
# arithmetic, not a fixed tolerance. The oracle computes in double from
# inputs the type holds exactly; the GPU computes in the type, in another
# order. An output made of k terms a (x) b (a product or a sum, then the
# add monoid over the terms) and an optional accumulated old value w has
# every intermediate bounded by S = |w| + sum(|a||b| + |a| + |b|), and each
# of its at most k + 2 rounded operations errs by at most u * S (u = 2^-24
# for fp32, 2^-53 for fp64; a min/max only selects), so the GPU result is
# within (k + 3) * u * S of the exact one, and the oracle's double result
# within (k + 3) * 2^-53 * S of it.
UNIT = {"fp32": 2.0 ** -24, "fp64": 2.0 ** -53}


def float_bound(t, terms, w_old=0.0):
    if t not in UNIT:
        return 0.0
    S = abs(float(w_old)) + sum(abs(float(a)) * abs(float(b)) + abs(float(a)) + abs(float(b)) for a, b in terms)
    return (len(terms) + 3) * (UNIT[t] + 2.0 ** -53) * S


def rand_dict(rng, n, k, t):
    idx = rng.choice(n, min(k, n), replace=False) if n else []
    return {int(i): gbo.cast(t, rand_val(rng, t)) for i in idx}


def rand_mat(rng, nr, nc, k, t):
    e = {}
    for _ in range(k):
        if nr and nc:
            e[(int(rng.integers(nr)), int(rng.integers(nc)))] = gbo.cast(t, rand_val(rng, t))
    return e


def gpu_vec(ctx, d, t, n):
    v = gb.Vector(ctx, GBT[t], n)
    if d:
        idx = np.array(sorted(d), dtype=np.uint32)
        vals = np.array([d[i] for i in sorted(d)], dtype=gb.NP_DTYPE[GBT[t]])
        v.build(idx, vals)
    return v


def gpu_mat(ctx, e, t, nr, nc, structural=False, flags=gb.BUILD_DEFAULT):
    A = gb.Matrix(ctx, GBT[t], nr, nc)
    keys = sorted(e)
    r = np.array([k[0] for k in keys], dtype=np.uint32)
    c = np.array([k[1] for k in keys], dtype=np.uint32)
    v = None if structural else np.array([e[k] for k in keys], dtype=gb.NP_DTYPE[GBT[t]])
    A.build(r, c, v, flags=flags)
    return A


def close(a, b, t, tol=0.0):
    if t == "fp32" and abs(b) > float(np.finfo(np.float32).max):
        b = math.copysign(math.inf, b)              # the exact value overflows FP32
    if t in ("fp32", "fp64"):
        if math.isinf(a) or math.isinf(b):
            return a == b
        return abs(a - b) <= tol
    if t == "bool":
        return bool(a) == bool(b)
    return int(a) == int(b)


def assert_vec(v, want: gbo.Vec, tol=lambda i: 0.0):
    got = v.to_dict()
    assert set(got) == set(want.e), (sorted(set(got) ^ set(want.e))[:10])
    for i, x in want.e.items():
        assert close(got[i], x, want.t, tol(i)), (i, got[i], x, tol(i))


CASES = []
for sr, types in SUPPORTED.items():
    for t in types:
        CASES.append((sr, t))


@pytest.mark.parametrize("sr,t", CASES)
def test_mxv_vxm_all_semirings_masks_directions(ctx, sr, t):
    rng = np.random.default_rng(abs(hash((sr, t))) % 2**32)
    mask_kinds = ["none", "value", "structure", "scmp", "scmp_structure", "none_scmp"]
    count = 0
    for op, direction, mk, accum, replace, tran, (nr, nc) in itertools.product(
            ["mxv", "vxm"], [gb.AUTO, gb.PUSH, gb.PULL], mask_kinds, [None, "acc"], [False, True], [False, True],
            [(37, 70), (129, 33)]):
        if rng.random() > 0.12:      # a seeded sample of the full product
            continue
        count += 1
        structural_A = rng.random() < 0.3
        E = rand_mat(rng, nr, nc, int(nr * nc * 0.08), t)
        if structural_A:
            E = {k: gbo.cast(t, 1) for k in E}
        A = gpu_mat(ctx, E, t, nr, nc, structural=structural_A)
        Am = gbo.Mat(nr, nc, t, E)
        # dimensions of u / w for this form
        out_rows = (op == "mxv") != tran
        nout, nin = (nr, nc) if out_rows else (nc, nr)
        ud = rand_dict(rng, nin, max(1, nin // 3), t)
        wd = rand_dict(rng, nout, nout // 4, t)
        mt = ["bool", "int32", "fp64"][int(rng.integers(3))]
        md = rand_dict(rng, nout, nout // 2, mt) if mk not in ("none", "none_scmp") else None
        acc_op = None
        if accum:
            acc_op = {"bool": "LOR", "int32": "PLUS", "uint32": "MAX", "uint64": "PLUS", "fp32": "MIN",
                      "fp64": "PLUS"}[t]
        u = gpu_vec(ctx, ud, t, nin)
        w = gpu_vec(ctx, wd, t, nout)
        mask = gpu_vec(ctx, md, mt, nout) if md is not None else None
        mval = 0
        if "scmp" in mk:
            mval |= gb.SCMP
        if "structure" in mk:
            mval |= gb.STRUCTURE
        d = gb.Descriptor(mask=mval, outp=gb.REPLACE if replace else gb.DEFAULT, direction=direction)
        if tran:
            d.set(gb.F_INP0 if op == "mxv" else gb.F_INP1, gb.TRAN)
        accb = BOP[acc_op] if acc_op else gb.NOP
        if op == "mxv":
            gb.mxv(w, mask, accb, SR[sr], A, u, d)
            want = gbo.mxv(gbo.Vec(nout, t, wd), gbo.Vec(nout, mt, md) if md is not None else None, acc_op, sr, Am,
                           gbo.Vec(nin, t, ud), tran=tran, structural="structure" in mk, scmp="scmp" in mk,
                           replace=replace)
        else:
            gb.vxm(w, mask, accb, SR[sr], u, A, d)
            want = gbo.vxm(gbo.Vec(nout, t, wd), gbo.Vec(nout, mt, md) if md is not None else None, acc_op, sr,
                           gbo.Vec(nin, t, ud), Am, tran=tran, structural="structure" in mk, scmp="scmp" in mk,
                           replace=replace)
        def tol(i, E=E, ud=ud, wd=wd, out_rows=out_rows, accum=accum):
            terms = [(a, ud[j]) for (r, c), a in E.items()
                     for j in [c if out_rows else r] if (r if out_rows else c) == i and j in ud]
            return float_bound(t, terms, wd.get(i, 0.0) if accum else 0.0)
        assert_vec(w, want, tol)
        for x in (A, u, w, mask, d):
            if x is not None:
                x.free()
    assert count > 5


def test_mxv_domain_and_dimension_errors(ctx):
    A = gpu_mat(ctx, {(0, 1): 1.0}, "fp64", 4, 5)
    u = gpu_vec(ctx, {0: 1.0}, "fp64", 5)
    w = gpu_vec(ctx, {}, "fp64", 4)
    with pytest.raises(gb.GBError) as e:
        gb.mxv(w, None, gb.NOP, gb.LOR_LAND, A, u)
    assert e.value.code == gb.DOMAIN_MISMATCH
    bad = gpu_vec(ctx, {}, "fp64", 3)
    with pytest.raises(gb.GBError) as e:
        gb.mxv(bad, None, gb.NOP, gb.PLUS_TIMES, A, u)
    assert e.value.code == gb.DIMENSION_MISMATCH
    u32 = gpu_vec(ctx, {0: 1}, "uint32", 5)
    with pytest.raises(gb.GBError) as e:
        gb.mxv(w, None, gb.NOP, gb.PLUS_TIMES, A, u32)
    assert e.value.code == gb.DOMAIN_MISMATCH


def test_csr_only_matrix_falls_back_to_the_available_direction(ctx):
    rng = np.random.default_rng(4)
    E = rand_mat(rng, 90, 90, 700, "fp64")
    A = gpu_mat(ctx, E, "fp64", 90, 90, flags=gb.CSR_ONLY)
    ud = rand_dict(rng, 90, 5, "fp64")
    for direction in (gb.AUTO, gb.PUSH, gb.PULL):
        w = gpu_vec(ctx, {}, "fp64", 90)
        gb.mxv(w, None, gb.NOP, gb.PLUS_TIMES, A, gpu_vec(ctx, ud, "fp64", 90), gb.Descriptor(direction=direction))
        assert_vec(w, gbo.mxv(gbo.Vec(90, "fp64"), None, None, "PLUS_TIMES", gbo.Mat(90, 90, "fp64", E),
                              gbo.Vec(90, "fp64", ud)))


def test_running_example_on_gpu():
    """The paper's running example (Section 3.4) through vxm with the
    complemented visited mask."""
    from tests.conftest import read_golden
    import torch
    f = read_golden("running_example.txt")
    n = int(f["n"])
    edges = [tuple(map(int, e.split("-"))) for e in f["edges"].split()]
    with gb.Context(0) as c:
        A = gpu_mat(c, {e: True for e in edges}, "bool", n, n, structural=True)
        u = gpu_vec(c, {int(i): True for i in f["frontier"].split()}, "bool", n)
        v = gpu_vec(c, {int(i): True for i in f["visited"].split()}, "bool", n)
        for direction in (gb.PUSH, gb.PULL):
            w = gpu_vec(c, {}, "bool", n)
            gb.vxm(w, v, gb.NOP, gb.LOR_LAND, u, A, gb.Descriptor(mask=gb.SCMP, direction=direction))
            assert sorted(w.to_dict()) == [int(x) for x in f["next_frontier"].split()]
        torch.cuda.synchronize()


@pytest.mark.parametrize("t", ["bool", "int32", "uint32", "uint64", "fp32", "fp64"])
def test_ewise_and_reduce(ctx, t):
    rng = np.random.default_rng(len(t))
    n = 301
    ops = ["PLUS", "TIMES", "MIN", "MAX", "LOR", "LAND", "FIRST", "SECOND", "PAIR", "MINUS"]
    for op in ops:
        ud, vd, wd = rand_dict(rng, n, 120, t), rand_dict(rng, n, 90, t), rand_dict(rng, n, 50, t)
        md = rand_dict(rng, n, 150, "int32")
        for add in (True, False):
            for mk in (None, gb.DEFAULT, gb.SCMP, gb.STRUCTURE):
                w = gpu_vec(ctx, wd, t, n)
                mask = gpu_vec(ctx, md, "int32", n) if mk is not None else None
                d = gb.Descriptor(mask=mk or 0)
                f = gb.ewise_add if add else gb.ewise_mult
                f(w, mask, gb.NOP, BOP[op], gpu_vec(ctx, ud, t, n), gpu_vec(ctx, vd, t, n), d)
                g = gbo.ewise_add if add else gbo.ewise_mult
                want = g(gbo.Vec(n, t, wd), gbo.Vec(n, "int32", md) if mk is not None else None, None, op,
                         gbo.Vec(n, t, ud), gbo.Vec(n, t, vd), structural=mk == gb.STRUCTURE, scmp=mk == gb.SCMP)
                assert_vec(w, want, lambda i: float_bound(t, [(ud.get(i, 0.0), vd.get(i, 0.0))]))
    for mon in MON:
        ud = rand_dict(rng, n, 40, t)
        got = gb.reduce_vector(gpu_vec(ctx, ud, t, n), MON[mon])
        # a reduction of k values: k - 1 rounded operations on partial results bounded by sum |x|
        # (a product of k values is bounded by prod max(1, |x|) instead)
        red = lambda vals: float_bound(t, [(1.0, 0.0)] * len(vals)) * (
            float(np.prod([max(1.0, abs(x)) for x in vals])) if mon == "TIMES" else
            sum(abs(x) for x in vals) / max(len(vals), 1) + 1.0) if t in UNIT else 0.0
        assert close(got, gbo.reduce_vector(t, mon, gbo.Vec(n, t, ud)), t, red(list(ud.values())))
        got = gb.reduce_vector(gpu_vec(ctx, {}, t, n), MON[mon])
        assert close(got, gbo.reduce_vector(t, mon, gbo.Vec(n, t, {})), t)
        E = rand_mat(rng, 50, 70, 400, t)
        A = gpu_mat(ctx, E, t, 50, 70)
        assert close(gb.reduce_matrix(A, MON[mon]), gbo.reduce_matrix(t, mon, gbo.Mat(50, 70, t, E)), t,
                     red(list(E.values())))
        for tran in (False, True):
            nout = 70 if tran else 50
            w = gpu_vec(ctx, {}, t, nout)
            gb.reduce_rows(w, None, gb.NOP, MON[mon], A, gb.Descriptor(inp0=gb.TRAN if tran else 0))
            rows = {}
            for (r, c), x in E.items():
                rows.setdefault(c if tran else r, []).append(x)
            assert_vec(w, gbo.reduce_rows(gbo.Vec(nout, t), None, None, mon, gbo.Mat(50, 70, t, E), tran=tran),
                       lambda i: red(rows.get(i, [])))


def test_reduce_accumulates_into_prior_value(ctx):
    v = gpu_vec(ctx, {1: 5, 7: 6}, "int32", 10)
    assert gb.reduce_vector(v, gb.MONOID_PLUS, accum=gb.PLUS, init=100) == 111


@pytest.mark.parametrize("sr,t", CASES)
def test_mxm_masked(ctx, sr, t):
    rng = np.random.default_rng(7 + len(sr) + len(t))
    for tran0, tran1, mk, acc, replace in itertools.product(
            [False, True], [False, True], ["structure", "value", "none", "scmp", "scmp_structure", "none_scmp"],
            [None, "acc"], [False, True]):
        if rng.random() > 0.3:
            continue
        nr, nk, nc = 41, 37, 53
        Ae = rand_mat(rng, nk if tran0 else nr, nr if tran0 else nk, 300, t)
        Be = rand_mat(rng, nc if tran1 else nk, nk if tran1 else nc, 300, t)
        Me = rand_mat(rng, nr, nc, 600, "int32")
        Ce = rand_mat(rng, nr, nc, 200, t)
        A = gpu_mat(ctx, Ae, t, nk if tran0 else nr, nr if tran0 else nk)
        B = gpu_mat(ctx, Be, t, nc if tran1 else nk, nk if tran1 else nc)
        has_m = not mk.startswith("none")
        M = gpu_mat(ctx, Me, "int32", nr, nc) if has_m else None
        C = gpu_mat(ctx, Ce, t, nr, nc)
        acc_op = {"bool": "LOR", "int32": "PLUS", "uint32": "MAX", "uint64": "PLUS", "fp32": "MIN",
                  "fp64": "PLUS"}[t] if acc else None
        mval = (gb.STRUCTURE if "structure" in mk else 0) | (gb.SCMP if "scmp" in mk else 0)
        d = gb.Descriptor(mask=mval, outp=gb.REPLACE if replace else 0,
                          inp0=gb.TRAN if tran0 else 0, inp1=gb.TRAN if tran1 else 0)
        gb.mxm(C, M, BOP[acc_op] if acc_op else gb.NOP, SR[sr], A, B, d)
        want = gbo.mxm(gbo.Mat(nr, nc, t, Ce), gbo.Mat(nr, nc, "int32", Me) if has_m else None, acc_op, sr,
                       gbo.Mat(A.nrows, A.ncols, t, Ae), gbo.Mat(B.nrows, B.ncols, t, Be), tran0=tran0, tran1=tran1,
                       structural="structure" in mk, scmp="scmp" in mk, replace=replace)
        r, c, v = C.extract_tuples(with_vals=True)
        got = {(int(i), int(j)): x.item() for i, j, x in zip(r, c, v)}
        assert set(got) == set(want.e)
        At = {(j, i): v for (i, j), v in Ae.items()} if tran0 else Ae
        Bt = {(j, i): v for (i, j), v in Be.items()} if tran1 else Be
        Brow = {}
        for (kk, j), b in Bt.items():
            Brow.setdefault(kk, {})[j] = b
        for k, x in want.e.items():
            i, j = k
            terms = [(a, Brow[kk][j]) for (ii, kk), a in At.items() if ii == i and kk in Brow and j in Brow[kk]]
            tol = float_bound(t, terms, Ce.get(k, 0.0) if acc_op else 0.0)
            assert close(got[k], x, t, tol), (k, got[k], x, tol)
        for x in (A, B, M, C, d):
            if x is not None:
                x.free()


def test_vector_object_roundtrip(ctx):
    v = gb.Vector(ctx, gb.FP64, 100)
    assert v.nvals == 0 and v.size == 100
    v.build(np.array([5, 3, 5, 99], np.uint32), np.array([1.0, 2.0, 4.0, 8.0]), dup=gb.PLUS)
    assert v.to_dict() == {3: 2.0, 5: 5.0, 99: 8.0}
    assert v.extract_element(5) == 5.0 and v.extract_element(6) is None
    v.set_element(6, -1.5)
    assert v.nvals == 4
    dense, pres = v.extract_dense(absent=7.0)
    assert dense[0] == 7.0 and dense[6] == -1.5 and pres.sum() == 4
    w = v.dup()
    v.clear()
    assert v.nvals == 0 and w.nvals == 4
    w.fill(2.5)
    assert w.nvals == 100 and w.extract_element(42) == 2.5
    with pytest.raises(gb.GBError) as e:
        v.build(np.array([100], np.uint32), np.array([1.0]))
    assert e.value.code == gb.INVALID_INDEX
    v.build_dense(np.arange(100, dtype=np.float64))
    assert v.nvals == 100 and v.extract_element(37) == 37.0
    for x in (v, w):
        x.free()
