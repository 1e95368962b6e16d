"""GPU parity of the algorithms built on the library: SSSP (bit-exact
distances), connected components (bit-exact canonical labels), PageRank
(L1 <= 1e-5 against the FP64 oracle) and triangle counting (exact count and
exact per-entry C of C<L> = L*L), through the C ABI."""
import itertools

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1908_01407_gb300 as gb

pytestmark = pytest.mark.gpu

PR_L1_TOL = 1e-5


def build(ctx, t, weights=True, flags=gb.SYMMETRIC):
    g = oracle.csr_from_tuples(t)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w if (weights and t.w is not None) else None,
                              type_=gb.UINT32, flags=flags)
    return g, A


def sssp_gpu(ctx, A, src, direction=gb.AUTO):
    d = gb.Descriptor(direction=direction)
    dist = np.empty(A.nrows, np.uint32)
    _, it = gb.sssp(ctx, A, src, dist, d)
    d.free()
    return dist, it


# ------------------------------------------------------------------- SSSP
def test_sssp_small_graphs_all_directions(ctx):
    cases = [gen.from_edges(12, [(i, i + 1) for i in range(11)], [37] * 11),
             gen.random_small(12, 0.35, 104, wmax=20),
             gen.random_small(9, 0.2, 7, wmax=5),
             gen.grid(33, 17, 0.15, seed=5, wmax=1000),
             gen.from_edges(1, [], [])]
    for t in cases:
        if t.w is None:
            t = gen.Tuples(t.n, t.src, t.dst, np.ones_like(t.src), t.name)
        g, A = build(ctx, t)
        for src in sorted({0, t.n // 2, t.n - 1}):
            want = oracle.sssp(g, src)
            for direction in (gb.AUTO, gb.PUSH, gb.PULL):
                got, _ = sssp_gpu(ctx, A, src, direction)
                assert np.array_equal(got, want), (t.name, src, direction)
        A.free()


@pytest.mark.parametrize("scale,seed", [(12, 21), (14, 2)])
def test_sssp_rmat(ctx, scale, seed):
    t = gen.rmat(scale, 16, seed=seed, wmax=255)
    g, A = build(ctx, t)
    for s in gen.sources(t, 4, seed=1):
        want = oracle.sssp(g, int(s))
        got, it = sssp_gpu(ctx, A, int(s))
        assert np.array_equal(got, want)
        assert it >= 1
    # device output buffer
    dist = torch.empty(t.n, dtype=torch.int32, device="cuda")
    gb.sssp(ctx, A, int(gen.sources(t, 1, seed=1)[0]), dist)
    assert np.array_equal(dist.cpu().numpy().view(np.uint32), oracle.sssp(g, int(gen.sources(t, 1, seed=1)[0])))
    A.free()


def test_sssp_errors(ctx):
    t = gen.rmat(8, 4, seed=1)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)    # structural: no weights
    with pytest.raises(gb.GBError) as e:
        gb.sssp(ctx, A, 0, np.empty(t.n, np.uint32))
    assert e.value.code == gb.DOMAIN_MISMATCH
    t = gen.rmat(8, 4, seed=1, wmax=9)
    g, A = build(ctx, t)
    with pytest.raises(gb.GBError) as e:
        gb.sssp(ctx, A, t.n, np.empty(t.n, np.uint32))
    assert e.value.code == gb.INVALID_INDEX


# --------------------------------------------------------------------- CC
@pytest.mark.parametrize("case", ["rmat14", "rmat_sparse", "grid", "small"])
def test_cc(ctx, case):
    t = {"rmat14": lambda: gen.rmat(14, 16, seed=1),
         "rmat_sparse": lambda: gen.rmat(13, 1, seed=9),
         "grid": lambda: gen.grid(96, 80, 0.45, seed=3),
         "small": lambda: gen.random_small(12, 0.15, 205)}[case]()
    g, A = build(ctx, t, weights=False)
    want = oracle.cc(g)
    lab = np.empty(t.n, np.uint32)
    _, it = gb.cc(ctx, A, lab)
    assert np.array_equal(lab, want)
    assert it >= 1
    A.free()


@pytest.mark.parametrize("case", ["rmat14", "rmat_sparse", "grid", "small", "single", "path"])
def test_cc_fastsv(ctx, case):
    t = {"rmat14": lambda: gen.rmat(14, 16, seed=1),
         "rmat_sparse": lambda: gen.rmat(13, 1, seed=9),
         "grid": lambda: gen.grid(96, 80, 0.45, seed=3),
         "small": lambda: gen.random_small(12, 0.15, 205),
         "single": lambda: gen.from_edges(1, []),
         "path": lambda: gen.from_edges(300, [(i + 1, i) for i in range(299)])}[case]()
    g, A = build(ctx, t, weights=False)
    want = oracle.cc(g)
    lab = np.empty(t.n, np.uint32)
    _, it = gb.cc_fastsv(ctx, A, lab)
    assert np.array_equal(lab, want)
    assert it >= 1
    # device output buffer gives the same labels
    dl = torch.empty(t.n, dtype=torch.int32, device="cuda")
    gb.cc_fastsv(ctx, A, dl)
    assert np.array_equal(dl.cpu().numpy().view(np.uint32), want)
    A.free()


def test_cc_fastsv_weak_components_and_errors(ctx):
    """A directed matrix: components of the underlying undirected graph."""
    rng = np.random.default_rng(8)
    n = 2000
    r = rng.integers(0, n, 1500).astype(np.uint32)
    c = rng.integers(0, n, 1500).astype(np.uint32)
    A = gb.Matrix.from_tuples(ctx, n, r, c)
    g = oracle.csr_build(n, np.concatenate([r, c]), np.concatenate([c, r]))
    lab = np.empty(n, np.uint32)
    gb.cc_fastsv(ctx, A, lab)
    assert np.array_equal(lab, oracle.cc(g))
    A.free()
    B = gb.Matrix.from_tuples(ctx, n, r, c, flags=gb.CSR_ONLY)
    with pytest.raises(gb.GBError) as e:
        gb.cc_fastsv(ctx, B, lab)
    assert e.value.code == gb.INVALID_VALUE
    B.free()


# ---------------------------------------------------------------- PageRank
@pytest.mark.parametrize("order", [0, 1, 57344])
@pytest.mark.parametrize("tile", [256, 512, 1024])
@pytest.mark.parametrize("case", ["rmat14", "rmat17", "rmat12_e4", "grid", "star", "cycle"])
def test_pagerank_l1_vs_fp64_oracle(ctx, case, tile, order):
    """order 1 runs on the degree-ordered copy with the default 32,768
    staged ranks, 57344 with the largest staged set: below that many
    vertices every rank is staged; R-MAT scale 17 (131,072) also gathers
    the rest from global memory."""
    t = {"rmat14": lambda: gen.rmat(14, 16, seed=1),
         "rmat17": lambda: gen.rmat(17, 16, seed=4),
         "rmat12_e4": lambda: gen.rmat(12, 4, seed=3),
         "grid": lambda: gen.grid(70, 50, 0.1, seed=3),
         "star": lambda: gen.from_edges(300, [(0, i) for i in range(1, 300)]),
         "cycle": lambda: gen.from_edges(1000, [(i, (i + 1) % 1000) for i in range(1000)])}[case]()
    g, A = build(ctx, t, weights=False)
    gb.pagerank_set_tile(A, tile)
    gb.pagerank_set_order(A, 1 if order else 0, order if order > 1 else 0)
    want, wres = oracle.pagerank(g, 0.85, 50)
    rank = np.empty(t.n, np.float32)
    _, res = gb.pagerank(ctx, A, 0.85, 50, rank)
    l1 = np.abs(rank.astype(np.float64) - want).sum()
    assert l1 <= PR_L1_TOL, l1
    assert abs(rank.astype(np.float64).sum() - 1.0) < 1e-5
    # residuals follow the oracle's (FP32 rounding allows small differences)
    assert np.all(np.abs(res - wres) <= 1e-6 + 1e-3 * wres), (res[:5], wres[:5])
    if case == "cycle":
        assert np.max(np.abs(rank - 1.0 / t.n)) < 1e-9
    A.free()


@pytest.mark.parametrize("order", [0, 1])
def test_pagerank_is_bit_reproducible(ctx, order):
    t = gen.rmat(17, 8, seed=5)
    g, A = build(ctx, t, weights=False)
    gb.pagerank_set_order(A, order)
    r1 = np.empty(t.n, np.float32)
    r2 = np.empty(t.n, np.float32)
    gb.pagerank(ctx, A, 0.85, 20, r1)
    gb.pagerank(ctx, A, 0.85, 20, r2)
    assert np.array_equal(r1.view(np.uint32), r2.view(np.uint32))
    A.free()


# --------------------------------------------------------------------- TC
def tc_pipeline(ctx, t):
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    B, new_id = A.degree_order()
    L = B.tril()
    return A, B, L, new_id


@pytest.mark.parametrize("case", ["k12", "wheel", "tree", "rmat12", "rmat14", "grid", "empty", "k3"])
def test_tc_count_and_entries(ctx, case):
    t = {"k12": lambda: gen.from_edges(12, list(itertools.combinations(range(12), 2))),
         "empty": lambda: gen.from_edges(6, []),                       # no entries in L at all
         "k3": lambda: gen.from_edges(3, [(0, 1), (1, 2), (0, 2)]),     # one triangle, counted at one entry
         "wheel": lambda: gen.from_edges(10, [(0, i) for i in range(1, 10)] + [(i, i % 9 + 1) for i in range(1, 10)]),
         "tree": lambda: gen.from_edges(31, [(i, (i - 1) // 2) for i in range(1, 31)]),
         "rmat12": lambda: gen.rmat(12, 16, seed=4),
         "rmat14": lambda: gen.rmat(14, 16, seed=4),
         "grid": lambda: gen.grid(40, 40, 0.0, seed=1)}[case]()
    g = oracle.csr_from_tuples(t)
    A, B, L, new_id = tc_pipeline(ctx, t)
    want_new = oracle.degree_order(g)
    assert np.array_equal(new_id, want_new)
    h = oracle.relabel(g, want_new)
    want_vals, want_total = oracle.masked_LL(h)
    assert want_total == oracle.tc(g)
    C = gb.Matrix(ctx, gb.UINT32, t.n, t.n)
    assert gb.tc(ctx, L) == want_total
    assert gb.tc(ctx, L, C) == want_total
    r, c, v = C.extract_tuples(with_vals=True)
    Lr, Lc = L.extract_tuples()
    assert np.array_equal(r, Lr) and np.array_equal(c, Lc)
    assert np.array_equal(v, want_vals)
    for x in (A, B, L, C):
        x.free()


def test_tc_total_with_rows_longer_than_the_shared_buffer(ctx):
    """K_600: equal degrees, so after the relabel row i of L holds i entries;
    rows past 512 are searched in global memory. C(600, 3) triangles, the
    same total with and without the per-entry C."""
    n = 600
    t = gen.from_edges(n, list(itertools.combinations(range(n), 2)))
    A, B, L, _ = tc_pipeline(ctx, t)
    want = n * (n - 1) * (n - 2) // 6
    assert gb.tc(ctx, L) == want
    C = gb.Matrix(ctx, gb.UINT32, n, n)
    assert gb.tc(ctx, L, C) == want
    for x in (A, B, L, C):
        x.free()


def test_tc_agrees_with_generic_masked_mxm(ctx):
    t = gen.rmat(11, 16, seed=6)
    A, B, L, _ = tc_pipeline(ctx, t)
    C = gb.Matrix(ctx, gb.UINT32, t.n, t.n)
    gb.mxm(C, L, gb.NOP, gb.PLUS_PAIR, L, L, gb.Descriptor(mask=gb.STRUCTURE))
    total = gb.reduce_matrix(C, gb.MONOID_PLUS)
    assert total == gb.tc(ctx, L) == oracle.tc(oracle.csr_from_tuples(t))
    for x in (A, B, L, C):
        x.free()


# ----------------------------------------------------- full config sizes
@pytest.mark.slow
def test_sssp_pagerank_rmat_s22_full_size(ctx):
    """R-MAT scale 22, edge factor 16, seed 2, weights uniform in [1, 255]:
    SSSP from the first of the benchmark's sources and 50 PageRank
    iterations, against the oracle."""
    t = gen.rmat(22, 16, seed=2, wmax=255)
    g, A = build(ctx, t)
    s = int(gen.sources(t, 8, seed=1)[0])
    got, _ = sssp_gpu(ctx, A, s)
    assert np.array_equal(got, oracle.sssp(g, s))
    rank = np.empty(t.n, np.float32)
    want, _ = oracle.pagerank(g, 0.85, 50)
    for order in (0, 1):     # as stored, and the degree-ordered copy with staged ranks
        gb.pagerank_set_order(A, order)
        gb.pagerank(ctx, A, 0.85, 50, rank)
        assert np.abs(rank.astype(np.float64) - want).sum() <= PR_L1_TOL, order
    A.free()


@pytest.mark.slow
def test_grid_4096_bfs_sssp_cc_full_size(ctx):
    """4096 x 4096 grid, 10% of edges deleted (seed 3), weights in [1, 1000]:
    BFS, SSSP and connected components against the oracle."""
    t = gen.grid(4096, 4096, 0.1, seed=3, wmax=1000)
    g, A = build(ctx, t)
    src = gen.first_nonisolated(t)
    lv, par, st = gb.bfs(ctx, A, src)
    lv = lv.cpu().numpy()
    want = oracle.bfs(g, src)
    assert np.array_equal(lv, want)
    assert oracle.bfs_parent_violations(g, src, lv, par.cpu().numpy()) == 0
    got, _ = sssp_gpu(ctx, A, src)
    assert np.array_equal(got, oracle.sssp(g, src))
    lab = np.empty(t.n, np.uint32)
    gb.cc(ctx, A, lab)
    want = oracle.cc(g)
    assert np.array_equal(lab, want)
    gb.cc_fastsv(ctx, A, lab)
    assert np.array_equal(lab, want)
    A.free()


@pytest.mark.slow
def test_tc_rmat_s20_full_size(ctx):
    """R-MAT scale 20, edge factor 16, seed 4, degree-ordered, L = tril."""
    from tests.conftest import read_golden
    f = read_golden("tc_rmat_s20.txt")     # the oracle's count (tests/golden/make_golden.py)
    t = gen.rmat(20, 16, seed=4)
    A, B, L, _ = tc_pipeline(ctx, t)
    assert A.nvals == int(f["m_stored"])
    assert gb.tc(ctx, L) == int(f["triangles"])
    for x in (A, B, L):
        x.free()


# ------------------------------------------------------- multi-source BFS
@pytest.mark.parametrize("case,k", [("rmat14", 64), ("rmat14", 1), ("rmat13", 37), ("grid", 64), ("small", 5),
                                    ("path", 9),
                                    ("rmat13", 150), ("rmat14", 256), ("rmat14", 100), ("grid", 128),
                                    ("grid", 200), ("path", 130), ("small", 65), ("rmat13", 300)])
def test_bfs_multi_matches_independent_bfs(ctx, case, k):
    """k BFS as one Boolean SpMM over bit-packed frontiers: 64 sources per
    word of source bits, one launch for up to 256 (one, two or four words
    per vertex), consecutive launches beyond; every row equals the oracle's
    queue BFS from that source, in push, pull and automatic direction."""
    t = {"rmat14": lambda: gen.rmat(14, 16, seed=1),
         "rmat13": lambda: gen.rmat(13, 8, seed=8),
         "grid": lambda: gen.grid(60, 50, 0.1, seed=3),
         "small": lambda: gen.from_edges(9, [(0, 1), (1, 2), (3, 4)]),
         # levels up to 699: the per-vertex level bytes hold levels below 254, later ones go to the output directly
         "path": lambda: gen.from_edges(700, [(i, i + 1) for i in range(699)])}[case]()
    g = oracle.csr_from_tuples(t)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    rng = np.random.default_rng(k)
    srcs = rng.integers(0, t.n, k).astype(np.uint32)      # any vertices, isolated and repeated ones included
    want = oracle.multi_bfs(g, srcs)
    for direction in (gb.AUTO, gb.PUSH, gb.PULL):
        lv = np.empty((k, t.n), np.int32)
        _, st = gb.bfs_multi(ctx, A, srcs, lv, gb.Descriptor(direction=direction))
        assert np.array_equal(lv, want), direction
        assert st["status"] == 0
        if k <= 256:   # one launch: one direction per expanded level
            assert st["push_levels"] + st["pull_levels"] <= st["depth"]
    A.free()


def test_bfs_multi_errors(ctx):
    t = gen.rmat(8, 4, seed=1)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    with pytest.raises(gb.GBError) as e:
        gb.bfs_multi(ctx, A, np.zeros(0, np.uint32), np.empty((1, t.n), np.int32))
    assert e.value.code == gb.INVALID_VALUE
    with pytest.raises(gb.GBError) as e:
        gb.bfs_multi(ctx, A, np.array([t.n], np.uint32), np.empty((1, t.n), np.int32))
    assert e.value.code == gb.INVALID_INDEX
    A.free()


@pytest.mark.parametrize("case", ["grid", "rmat14", "path", "two"])
def test_sssp_single_cluster_schedule(ctx, case):
    """SSSP relaxed inside one thread-block cluster: distances equal Dijkstra's."""
    t = {"grid": lambda: gen.grid(120, 90, 0.15, seed=5, wmax=1000),
         "rmat14": lambda: gen.rmat(14, 16, seed=3, wmax=255),
         "path": lambda: gen.from_edges(400, [(i, i + 1) for i in range(399)],
                                        weights=[(7 * i) % 13 + 1 for i in range(399)]),
         "two": lambda: gen.from_edges(6, [(0, 1), (1, 2), (3, 4), (4, 5)], weights=[3, 5, 2, 9])}[case]()
    g, A = build(ctx, t)
    d = gb.Descriptor(schedule=gb.SCHED_CLUSTER)
    srcs = [int(s) for s in gen.sources(t, 3, seed=2)] if t.n > 10 else [0, 5]
    for src in srcs:
        dist = np.empty(t.n, np.uint32)
        _, it = gb.sssp(ctx, A, src, dist, desc=d)
        assert np.array_equal(dist, oracle.sssp(g, src))
        assert it >= 1
    d.free()
    A.free()


# ------------------------------------------------------- adaptive PageRank
PRD_EPS = (1e-5, 1e-4, 1e-3, 1e-2)   # the floor GB_PAGERANK_DELTA_MIN_EPS and up


def prd_parity(g, got, want, alpha=0.85):
    """The bar of adaptive PageRank (DESIGN reading 14). T, one step of the
    PageRank recurrence, is an alpha-contraction in L1, so any vector x is
    within r(x) / (1 - alpha) of the fixed point p*, r(x) = ||T(x) - x||_1
    (computed by the oracle in FP64). Hence, exactly,
        ||got - want||_1 <= (r(got) + r(want)) / (1 - alpha).
    And the GPU's run must be converged as far as the oracle's run with the
    same eps: the two apply one freeze rule to values that differ by FP32
    rounding, so only vertices within that rounding of the threshold can
    decide differently: r(got) <= 2 r(want) + 1e-6."""
    r_got = oracle.pagerank_residual(g, got, alpha)
    r_want = oracle.pagerank_residual(g, want, alpha)
    l1 = np.abs(got.astype(np.float64) - want).sum()
    # r is computed in FP64 as a sum of n differences of values near each other: its
    # absolute error is at most about n * 2^-52 * max(p), allowed for by the last term
    fp64 = 4 * g.n * 2.0 ** -52 * max(float(np.abs(want).max()), 1e-30) / (1 - alpha)
    assert l1 <= (r_got + r_want) / (1 - alpha) * (1 + 1e-9) + fp64, (l1, r_got, r_want)
    assert r_got <= 2 * r_want + 1e-6, (r_got, r_want)
    return l1, r_got, r_want


@pytest.mark.parametrize("case", ["rmat14", "grid", "star", "cycle", "dangling"])
def test_pagerank_delta_vs_fp64_oracle(ctx, case):
    """Adaptive PageRank against the FP64 oracle with the same eps, for every
    eps the API accepts from its floor up (GB_PAGERANK_DELTA_MIN_EPS = 1e-5;
    below it the call is refused): the contraction bound of prd_parity, the
    active counts never grow and start at n, iteration counts within 2, and
    runs bit-identical."""
    t = {"rmat14": lambda: gen.rmat(14, 16, seed=21),
         "grid": lambda: gen.grid(100, 90, 0.1, seed=2),
         "star": lambda: gen.from_edges(6000, [(0, i) for i in range(1, 6000)]),   # a row past 4096: block row
         "cycle": lambda: gen.from_edges(97, [(i, (i + 1) % 97) for i in range(97)]),
         "dangling": lambda: gen.from_edges(50, [(0, 1), (1, 2), (2, 0), (3, 4), (2, 5)])}[case]()
    g, A = build(ctx, t, weights=False)
    for eps in PRD_EPS:
        want, it_o, act_o = oracle.pagerank_delta(g, 0.85, eps, 200)
        got = np.empty(t.n, np.float32)
        _, it, res, act = gb.pagerank_delta(ctx, A, 0.85, eps, 200, got)
        assert abs(it - it_o) <= 2
        prd_parity(g, got, want)
        again = np.empty(t.n, np.float32)
        gb.pagerank_delta(ctx, A, 0.85, eps, 200, again)
        assert np.array_equal(got.view(np.uint32), again.view(np.uint32))
        assert act[0] == t.n and np.all(np.diff(act.astype(np.int64)) <= 0)
        if case == "cycle":
            assert it == 1
    A.free()


def test_pagerank_delta_refuses_eps_below_its_floor(ctx):
    t = gen.rmat(10, 8, seed=22)
    g, A = build(ctx, t, weights=False)
    got = np.empty(t.n, np.float32)
    for eps in (0.0, 1e-6, 9.9e-6, float("nan")):
        with pytest.raises(gb.GBError) as e:
            gb.pagerank_delta(ctx, A, 0.85, eps, 50, got)
        assert e.value.code == gb.INVALID_VALUE
    gb.pagerank_delta(ctx, A, 0.85, 1e-5, 50, got)     # the floor itself is accepted
    A.free()


def test_pagerank_delta_without_freezing_is_pagerank(ctx):
    """eps = -1 never freezes: 50 iterations equal plain PageRank's."""
    t = gen.rmat(13, 16, seed=22)
    g, A = build(ctx, t, weights=False)
    got = np.empty(t.n, np.float32)
    _, it, res, act = gb.pagerank_delta(ctx, A, 0.85, -1.0, 50, got)
    assert it == 50 and np.all(act == t.n)
    want, r = oracle.pagerank(g, 0.85, 50)
    assert np.abs(got.astype(np.float64) - want).sum() <= 1e-5
    assert np.allclose(res, r, rtol=1e-3, atol=1e-7)
    A.free()


def test_pagerank_and_delta_directed_matrix(ctx):
    """A non-symmetric matrix: rows are the in-edges (CSC), degrees the
    out-degrees; plain and adaptive PageRank against the directed oracle."""
    rng = np.random.default_rng(3)
    n = 3000
    r = rng.integers(0, n, 30000).astype(np.uint32)
    c = rng.integers(0, n, 30000).astype(np.uint32)
    A = gb.Matrix.from_tuples(ctx, n, r, c)
    g = oracle.csr_build(n, r, c)
    got = np.empty(n, np.float32)
    want, _ = oracle.pagerank(g, 0.85, 30, directed=True)
    for order in (0, 1):     # the degree order is by out-degree: the CSC's column references
        gb.pagerank_set_order(A, order)
        gb.pagerank(ctx, A, 0.85, 30, got, residuals=False)
        assert np.abs(got.astype(np.float64) - want).sum() <= 1e-5, order
    for eps in PRD_EPS:
        want, it_o, _ = oracle.pagerank_delta(g, 0.85, eps, 200, directed=True)
        _, it, _, _ = gb.pagerank_delta(ctx, A, 0.85, eps, 200, got)
        assert abs(it - it_o) <= 2
        prd_parity(g, got, want)
    A.free()


def test_tc_every_set_kind_on_disjoint_cliques(ctx):
    """65 disjoint K_514 (33,410 vertices, all of degree 513, so the degree
    relabel keeps every id and each L(i,j), j < i, lies inside one clique):
    C(i,j) = i - j - 1, the clique's vertices between them, and the total is
    65 * C(514, 3). Rows of vertices above 32,768 use the hash set (at most
    512 entries) or the binary search in global memory (513 entries), the
    others the bitmap, so all three kinds run, with and without C."""
    m, c = 514, 65
    iu, ju = np.triu_indices(m, 1)
    base = (np.arange(c, dtype=np.int64) * m)[:, None]
    a = (base + iu[None, :]).ravel().astype(np.uint32)
    b = (base + ju[None, :]).ravel().astype(np.uint32)
    n = m * c
    A = gb.Matrix.from_tuples(ctx, n, np.concatenate([a, b]), np.concatenate([b, a]), flags=gb.SYMMETRIC)
    B, new_id = A.degree_order()
    assert np.array_equal(np.asarray(new_id), np.arange(n))
    L = B.tril()
    want = c * m * (m - 1) * (m - 2) // 6
    assert gb.tc(ctx, L) == want
    C = gb.Matrix(ctx, gb.UINT32, n, n)
    assert gb.tc(ctx, L, C) == want
    r, col, v = C.extract_tuples(with_vals=True)
    assert len(v) == L.nvals
    assert np.array_equal(v.astype(np.int64), r.astype(np.int64) - col.astype(np.int64) - 1)
    for x in (A, B, L, C):
        x.free()


def test_sssp_stats_count_the_algorithmic_bytes_of_each_iteration(ctx):
    """gb_sssp's stats: the iterations and the per-iteration trace, and the
    algorithmic bytes recomputed on the host from that trace (4 n value
    writes; per push 8 per frontier vertex + 8 per frontier out-edge; per
    pull 4 (n + 1) + n / 8 + 4 m + 4 per frontier out-edge; 4 per improved
    value) equal the kernel's count, while the distances match Dijkstra."""
    t = gen.rmat(14, 16, seed=31, wmax=255)
    g, A = build(ctx, t)
    n, m = A.nrows, A.nvals
    src = int(gen.sources(t, 1, seed=1)[0])
    for direction in (gb.AUTO, gb.PUSH, gb.PULL):
        d = gb.Descriptor(direction=direction, sssp_delta=gb.SSSP_DELTA_NONE)   # the plain iteration
        dist = np.empty(n, np.uint32)
        _, it, st = gb.sssp(ctx, A, src, dist, d, stats=True)
        assert np.array_equal(dist, oracle.sssp(g, src))
        assert st["depth"] == it == st["push_levels"] + st["pull_levels"] == len(st["trace"])
        tr = st["trace"]
        want = 4.0 * n
        for k, lv in enumerate(tr):
            nxt = tr[k + 1]["vertices"] if k + 1 < len(tr) else 0
            if lv["dir"] == "pull":
                want += 4.0 * (n + 1) + n / 8.0 + 4.0 * m + 4.0 * lv["edges"]
            else:
                want += 8.0 * lv["vertices"] + 8.0 * lv["edges"]
            want += 4.0 * nxt
        assert abs(st["alg_bytes"] - want) <= 2, (st["alg_bytes"], want)
        if direction == gb.PULL:
            assert st["push_levels"] == 0
        d.free()
    A.free()


@pytest.mark.parametrize("case", ["rmat14", "grid", "directed", "path", "star"])
def test_sssp_near_far_buckets_match_dijkstra(ctx, case):
    """SSSP whose frontier is restricted to improved vertices below a bound
    that grows by delta (the far ones wait): Dijkstra's distances for every
    bucket width, from 1 (a bucket per distance) to one that holds every
    distance, and the automatic one; bit-exact."""
    if case == "directed":
        rng = np.random.default_rng(9)
        n = 3000
        r = rng.integers(0, n, 25000).astype(np.uint32)
        c = rng.integers(0, n, 25000).astype(np.uint32)
        w = rng.integers(1, 300, 25000).astype(np.uint32)
        A = gb.Matrix.from_tuples(ctx, n, r, c, w, type_=gb.UINT32)
        g = oracle.csr_build(n, r, c, w)
        srcs = [3, 2999]
    else:
        t = {"rmat14": lambda: gen.rmat(14, 16, seed=33, wmax=255),
             "grid": lambda: gen.grid(150, 130, 0.1, seed=5, wmax=1000),
             "path": lambda: gen.from_edges(700, [(i, i + 1) for i in range(699)], [1 + i % 7 for i in range(699)]),
             "star": lambda: gen.from_edges(5000, [(0, i) for i in range(1, 5000)],
                                            [1 + (i * 37) % 900 for i in range(1, 5000)])}[case]()
        g, A = build(ctx, t)
        n = t.n
        srcs = [int(x) for x in gen.sources(t, 2, seed=3)]
    for delta in (1, 5, 64, 2**31 - 2, 0):
        d = gb.Descriptor(sssp_delta=delta)
        for src in srcs:
            dist = np.empty(n, np.uint32)
            gb.sssp(ctx, A, src, dist, d)
            assert np.array_equal(dist, oracle.sssp(g, src)), (delta, src)
        d.free()
    A.free()


def test_pagerank_autotune_keeps_a_candidate_and_the_result(ctx):
    t = gen.rmat(14, 16, seed=41)
    g, A = build(ctx, t, weights=False)
    tile, order, staged, ms = gb.pagerank_autotune(ctx, A)
    assert tile in (256, 512, 1024) and order in (0, 1) and ms > 0
    if order == 1:
        assert tile in (256, 512) and staged in (16384, 32768)
    else:
        assert staged == 0
    rank = np.empty(t.n, np.float32)
    gb.pagerank(ctx, A, 0.85, 50, rank)
    want, _ = oracle.pagerank(g, 0.85, 50)
    assert np.abs(rank.astype(np.float64) - want).sum() <= PR_L1_TOL
    with pytest.raises(gb.GBError) as e:
        gb.pagerank_set_tile(A, 300)
    assert e.value.code == gb.INVALID_VALUE
    for bad in ((2, 0), (1, 1000), (1, 58368)):
        with pytest.raises(gb.GBError) as e:
            gb.pagerank_set_order(A, *bad)
        assert e.value.code == gb.INVALID_VALUE
    A.free()
