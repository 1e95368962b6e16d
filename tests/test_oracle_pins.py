"""Pins of the oracle against things other than itself: closed forms,
invariants, brute force on tiny graphs, and independent library routines
(scipy.sparse.csgraph, dense numpy linear algebra). Each test names the
passage of the paper whose definition it checks. CPU only."""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import gen
import oracle
from oracle import graphblas as gbo
from tests.conftest import read_golden


def g_from_edges(n, edges, weights=None):
    return oracle.csr_from_tuples(gen.from_edges(n, edges, weights))


def dense_adj(g):
    A = np.zeros((g.n, g.n), dtype=np.int64)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr).astype(np.int64))
    A[rows, g.colidx] = 1
    return A


def scipy_csr(g, weighted=False):
    data = g.vals.astype(np.float64) if weighted else np.ones(g.m)
    return sp.csr_matrix((data, g.colidx.astype(np.int64), g.rowptr.astype(np.int64)),
                         shape=(g.n, g.n))


def floyd_warshall(n, edges, weights=None):
    INF = float("inf")
    d = [[0 if i == j else INF for j in range(n)] for i in range(n)]
    for k, (u, v) in enumerate(edges):
        w = 1 if weights is None else weights[k]
        d[u][v] = min(d[u][v], w)
        d[v][u] = min(d[v][u], w)
    for k in range(n):
        for i in range(n):
            for j in range(n):
                if d[i][k] + d[k][j] < d[i][j]:
                    d[i][j] = d[i][k] + d[k][j]
    return d


def small_edges(n, p, seed, wmax=0):
    t = gen.random_small(n, p, seed, wmax)
    half = t.ntuples // 2
    edges = list(zip(t.src[:half].tolist(), t.dst[:half].tolist()))
    w = t.w[:half].tolist() if t.w is not None else None
    return edges, w


# ---------------------------------------------------------------- build ---
def test_csr_build_matches_scipy_sum_duplicates():
    rng = np.random.default_rng(7)
    n, nt = 300, 5000
    r = rng.integers(0, n, nt).astype(np.uint32)
    c = rng.integers(0, n, nt).astype(np.uint32)
    v = rng.integers(0, 1000, nt).astype(np.uint32)
    g = oracle.csr_build(n, r, c, v, oracle.DUP_PLUS)
    ref = sp.coo_matrix((v.astype(np.int64), (r, c)), shape=(n, n)).tocsr()
    ref.sum_duplicates()
    ref.sort_indices()
    assert np.array_equal(g.rowptr.astype(np.int64), ref.indptr)
    assert np.array_equal(g.colidx.astype(np.int64), ref.indices)
    assert np.array_equal(g.vals.astype(np.int64), ref.data)


@pytest.mark.parametrize("dup", ["first", "second", "min", "max"])
def test_csr_build_dup_ops_brute_force(dup):
    rng = np.random.default_rng(11)
    n, nt = 20, 400
    r = rng.integers(0, n, nt).astype(np.uint32)
    c = rng.integers(0, n, nt).astype(np.uint32)
    v = rng.integers(0, 50, nt).astype(np.uint32)
    code = {"first": oracle.DUP_FIRST, "second": oracle.DUP_SECOND,
            "min": oracle.DUP_MIN, "max": oracle.DUP_MAX}[dup]
    g = oracle.csr_build(n, r, c, v, code)
    want = {}
    for t in range(nt):
        k = (int(r[t]), int(c[t]))
        x = int(v[t])
        if k not in want:
            want[k] = x
        elif dup == "second":
            want[k] = x
        elif dup == "min":
            want[k] = min(want[k], x)
        elif dup == "max":
            want[k] = max(want[k], x)
    got = {}
    for i in range(n):
        for p in range(int(g.rowptr[i]), int(g.rowptr[i + 1])):
            got[(i, int(g.colidx[p]))] = int(g.vals[p])
        row = g.row(i)
        assert np.all(np.diff(row.astype(np.int64)) > 0)  # sorted, unique
    assert got == want


def test_csr_build_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.csr_build(4, np.array([0, 5], np.uint32), np.array([1, 1], np.uint32))


# ------------------------------------------------------------------ BFS ---
def test_bfs_path_star_complete_disconnected():
    n = 9
    path = g_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    assert oracle.bfs(path, 0).tolist() == list(range(n))
    assert oracle.bfs(path, 4).tolist() == [abs(i - 4) for i in range(n)]
    star = g_from_edges(n, [(0, i) for i in range(1, n)])
    assert oracle.bfs(star, 0).tolist() == [0] + [1] * (n - 1)
    assert oracle.bfs(star, 3).tolist() == [1, 2, 2, 0, 2, 2, 2, 2, 2]
    kn = g_from_edges(n, list(itertools.combinations(range(n), 2)))
    assert oracle.bfs(kn, 5).tolist() == [1] * 5 + [0] + [1] * 3
    two = g_from_edges(6, [(0, 1), (1, 2), (3, 4), (4, 5)])
    assert oracle.bfs(two, 0).tolist() == [0, 1, 2, -1, -1, -1]


def test_bfs_full_grid_is_manhattan_distance():
    k = 17
    g = oracle.csr_from_tuples(gen.grid(k, k, p_delete=0.0, seed=1))
    lv = oracle.bfs(g, 0)
    r, c = np.divmod(np.arange(k * k), k)
    assert np.array_equal(lv, r + c)
    lv = oracle.bfs(g, k * k - 1)
    assert np.array_equal(lv, (k - 1 - r) + (k - 1 - c))


@pytest.mark.parametrize("seed", range(12))
def test_bfs_brute_force_floyd_warshall(seed):
    n = 6 + seed % 7
    edges, _ = small_edges(n, 0.3, seed)
    g = g_from_edges(n, edges)
    d = floyd_warshall(n, edges)
    for s in range(n):
        want = [-1 if math.isinf(x) else int(x) for x in d[s]]
        assert oracle.bfs(g, s).tolist() == want


def test_bfs_matches_scipy_on_rmat():
    g = oracle.csr_from_tuples(gen.rmat(10, 8, seed=5))
    d = csg.shortest_path(scipy_csr(g), unweighted=True, indices=[3, 100, 777])
    for row, s in zip(d, [3, 100, 777]):
        want = np.where(np.isinf(row), -1, row).astype(np.int32)
        assert np.array_equal(oracle.bfs(g, s), want)


def test_bfs_parent_checker_accepts_scipy_tree_and_rejects_planted_mistakes():
    g = oracle.csr_from_tuples(gen.rmat(9, 8, seed=9))
    s = int(np.argmax(g.degrees()))
    lv = oracle.bfs(g, s)
    order, pred = csg.breadth_first_order(scipy_csr(g), s, directed=True,
                                          return_predecessors=True)
    par = np.where(pred < 0, -1, pred).astype(np.int32)
    par[s] = s
    assert oracle.bfs_parent_violations(g, s, lv, par) == 0
    reached = np.flatnonzero((lv > 1))
    v = int(reached[0])
    bad = par.copy()
    bad[v] = s                      # not adjacent (depth 2+) or wrong depth
    assert oracle.bfs_parent_violations(g, s, lv, bad) == 1
    bad = par.copy()
    bad[s] = -1
    assert oracle.bfs_parent_violations(g, s, lv, bad) == 1
    unreached = np.flatnonzero(lv < 0)
    if unreached.size:
        bad = par.copy()
        bad[unreached[0]] = s
        assert oracle.bfs_parent_violations(g, s, lv, bad) == 1


# ----------------------------------------------------------------- SSSP ---
def test_sssp_unit_weights_equal_bfs_and_path_weights():
    t = gen.rmat(9, 8, seed=3)
    ones = gen.Tuples(t.n, t.src, t.dst, np.ones_like(t.src), "ones")
    g = oracle.csr_from_tuples(ones)
    s = int(np.argmax(g.degrees()))
    lv = oracle.bfs(g, s)
    d = oracle.sssp(g, s)
    assert np.array_equal(np.where(lv < 0, 2**32 - 1, lv.astype(np.int64)).astype(np.uint32), d)
    n, w = 12, 37
    path = g_from_edges(n, [(i, i + 1) for i in range(n - 1)], [w] * (n - 1))
    assert oracle.sssp(path, 0).tolist() == [i * w for i in range(n)]


@pytest.mark.parametrize("seed", range(10))
def test_sssp_brute_force_floyd_warshall(seed):
    n = 6 + seed % 7
    edges, ws = small_edges(n, 0.35, 100 + seed, wmax=20)
    g = g_from_edges(n, edges, ws)
    d = floyd_warshall(n, edges, ws)
    for s in range(n):
        want = [2**32 - 1 if math.isinf(x) else int(x) for x in d[s]]
        assert oracle.sssp(g, s).tolist() == want


def test_sssp_matches_scipy_dijkstra_and_certificate():
    g = oracle.csr_from_tuples(gen.rmat(10, 8, seed=6, wmax=255))
    srcs = [0, 17, 999]
    ref = csg.dijkstra(scipy_csr(g, weighted=True), indices=srcs)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr).astype(np.int64))
    for row, s in zip(ref, srcs):
        d = oracle.sssp(g, s)
        want = np.where(np.isinf(row), 2**32 - 1, row).astype(np.uint32)
        assert np.array_equal(d, want)
        # triangle inequality on every edge
        du, dv = d[rows].astype(np.int64), d[g.colidx].astype(np.int64)
        fin = du < 2**32 - 1
        assert np.all(dv[fin] <= du[fin] + g.vals[fin])


def test_sssp_full_grid_unit_weights_manhattan():
    k = 15
    t = gen.grid(k, k, p_delete=0.0, seed=2)
    g = oracle.csr_from_tuples(gen.Tuples(t.n, t.src, t.dst, np.ones_like(t.src), "u"))
    r, c = np.divmod(np.arange(k * k), k)
    assert np.array_equal(oracle.sssp(g, 0).astype(np.int64), r + c)


# ------------------------------------------------------------- PageRank ---
def google_matrix(g, alpha):
    """Dense column-stochastic matrix of the same random-surfer model built
    with numpy (independent construction): a walker on j follows one of its
    deg(j) edges w.p. alpha, a vertex without edges jumps uniformly, and
    with prob. 1 - alpha the walker teleports uniformly."""
    n = g.n
    A = dense_adj(g).astype(np.float64)
    deg = A.sum(axis=1)
    P = np.zeros((n, n))
    for j in range(n):
        P[:, j] = A[j, :] / deg[j] if deg[j] > 0 else 1.0 / n
    return alpha * P + (1 - alpha) / n * np.ones((n, n))


@pytest.mark.parametrize("name", ["gnp", "dangling", "star"])
def test_pagerank_matches_dense_power_iteration_and_fixed_point(name):
    alpha = 0.85
    if name == "gnp":
        edges, _ = small_edges(11, 0.3, 42)
        g = g_from_edges(11, edges)
    elif name == "dangling":
        g = g_from_edges(10, [(0, 1), (1, 2), (2, 0), (3, 4), (2, 5)])   # 6..9 isolated
    else:
        g = g_from_edges(8, [(0, i) for i in range(1, 8)])
    G = google_matrix(g, alpha)
    x = np.full(g.n, 1.0 / g.n)
    for k in (1, 2, 7, 50):
        p, r = oracle.pagerank(g, alpha, k)
        y = x.copy()
        for _ in range(k):
            y = G @ y
        assert np.abs(p - y).sum() < 1e-12
        assert abs(p.sum() - 1.0) < 1e-12
    # exact fixed point by a dense linear solve: (I - G) p = 0, sum p = 1
    M = np.eye(g.n) - G
    M[-1, :] = 1.0
    rhs = np.zeros(g.n)
    rhs[-1] = 1.0
    pstar = np.linalg.solve(M, rhs)
    p300, _ = oracle.pagerank(g, alpha, 300)
    assert np.abs(p300 - pstar).sum() < 1e-12
    p50, r50 = oracle.pagerank(g, alpha, 50)
    assert np.abs(p50 - pstar).sum() <= 2 * alpha**50
    # L1 contraction: residual_k <= 2 alpha^k
    assert np.all(r50 <= 2 * alpha ** np.arange(50) + 1e-15)


@pytest.mark.parametrize("kind", ["cycle", "complete", "torus"])
def test_pagerank_uniform_on_regular_graphs(kind):
    if kind == "cycle":
        n = 13
        g = g_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    elif kind == "complete":
        n = 9
        g = g_from_edges(n, list(itertools.combinations(range(n), 2)))
    else:
        k = 6
        n = k * k
        e = set()
        for r in range(k):
            for c in range(k):
                a = r * k + c
                e.add(tuple(sorted((a, r * k + (c + 1) % k))))
                e.add(tuple(sorted((a, ((r + 1) % k) * k + c))))
        g = g_from_edges(n, sorted(e))
    for it in (1, 5, 50):
        p, r = oracle.pagerank(g, 0.85, it)
        assert np.max(np.abs(p - 1.0 / n)) < 1e-15
        assert np.all(r < 1e-14)


# ---------------------------------------------------- adaptive PageRank ---
@pytest.mark.parametrize("name", ["gnp", "dangling", "star"])
def test_pagerank_delta_without_freezing_is_the_power_iteration(name):
    """eps = -1 never freezes a vertex: k iterations of the adaptive form
    are k steps of the dense Google-matrix power iteration."""
    alpha = 0.85
    if name == "gnp":
        edges, _ = small_edges(11, 0.3, 43)
        g = g_from_edges(11, edges)
    elif name == "dangling":
        g = g_from_edges(10, [(0, 1), (1, 2), (2, 0), (3, 4), (2, 5)])
    else:
        g = g_from_edges(8, [(0, i) for i in range(1, 8)])
    G = google_matrix(g, alpha)
    for k in (1, 3, 20):
        p, it, act = oracle.pagerank_delta(g, alpha, -1.0, k)
        y = np.full(g.n, 1.0 / g.n)
        for _ in range(k):
            y = G @ y
        assert it == k and np.all(act == g.n)
        assert np.abs(p - y).sum() < 1e-12


def test_pagerank_delta_regular_graph_converges_at_once():
    n = 13
    g = g_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    p, it, act = oracle.pagerank_delta(g, 0.85, 1e-6, 50)
    assert it == 1 and list(act) == [n]
    assert np.max(np.abs(p - 1.0 / n)) < 1e-15


def test_pagerank_delta_frozen_vertices_stay_frozen():
    """A vertex that stops changing never changes again, active counts never
    grow, and a tiny eps ends next to the exact fixed point."""
    edges, _ = small_edges(12, 0.25, 7)
    g = g_from_edges(12, edges + [(0, 11)])
    alpha, eps = 0.85, 1e-4
    runs = [oracle.pagerank_delta(g, alpha, eps, k)[0] for k in range(1, 40)]
    _, it, act = oracle.pagerank_delta(g, alpha, eps, 200)
    assert np.all(np.diff(act.astype(np.int64)) <= 0)
    same_prev = set()
    for k in range(len(runs) - 1):
        same = {i for i in range(g.n) if runs[k][i] == runs[k + 1][i]}
        assert same_prev <= same
        same_prev = same
    G = google_matrix(g, alpha)
    M = np.eye(g.n) - G
    M[-1, :] = 1.0
    rhs = np.zeros(g.n)
    rhs[-1] = 1.0
    pstar = np.linalg.solve(M, rhs)
    p, it, _ = oracle.pagerank_delta(g, alpha, 1e-9, 500)
    assert it < 500 and np.abs(p - pstar).sum() < 1e-6


def test_pagerank_directed_matches_dense_power_iteration():
    """A directed graph (rows = out-edges, some vertices without out-edges):
    the pull over in-neighbours divided by out-degrees is the dense
    random-surfer model, for plain and (never freezing) adaptive PageRank."""
    rng = np.random.default_rng(17)
    n = 12
    r = rng.integers(0, n, 30).astype(np.uint32)
    c = rng.integers(0, n, 30).astype(np.uint32)
    keep = (r != c) & (r < 9)              # vertices 9..11 have no out-edges
    g = oracle.csr_build(n, r[keep], c[keep])
    G = google_matrix(g, 0.85)
    for k in (1, 4, 30):
        y = np.full(n, 1.0 / n)
        for _ in range(k):
            y = G @ y
        p, _ = oracle.pagerank(g, 0.85, k, directed=True)
        assert np.abs(p - y).sum() < 1e-12
        q, it, _ = oracle.pagerank_delta(g, 0.85, -1.0, k, directed=True)
        assert it == k and np.abs(q - y).sum() < 1e-12


def test_pagerank_residual_is_the_dense_step_and_bounds_the_error():
    """r(x) = ||T(x) - x||_1 against the dense Google matrix built
    independently (symmetric and directed graphs, random x), against the C
    oracle's logged change of each power-iteration step, and the contraction
    bound ||x - p*||_1 <= r(x) / (1 - a) with p* from a dense solve."""
    rng = np.random.default_rng(23)
    edges, _ = small_edges(11, 0.3, 44)
    sym = g_from_edges(11, edges + [(0, 10)])
    r = rng.integers(0, 12, 30).astype(np.uint32)
    c = rng.integers(0, 12, 30).astype(np.uint32)
    keep = (r != c) & (r < 9)
    dirg = oracle.csr_build(12, r[keep], c[keep])
    for g in (sym, dirg):
        G = google_matrix(g, 0.85)
        for _ in range(3):
            x = rng.random(g.n)
            x /= x.sum()
            assert abs(oracle.pagerank_residual(g, x, 0.85) - np.abs(G @ x - x).sum()) < 1e-14
        M = np.eye(g.n) - G
        M[-1, :] = 1.0
        rhs = np.zeros(g.n)
        rhs[-1] = 1.0
        pstar = np.linalg.solve(M, rhs)
        directed = g is dirg
        _, log = oracle.pagerank(g, 0.85, 12, directed=directed)
        for k in (1, 4, 11):
            pk, _ = oracle.pagerank(g, 0.85, k, directed=directed)
            rk = oracle.pagerank_residual(g, pk, 0.85)
            assert abs(rk - log[k]) < 1e-14                   # the step the C oracle took next
            assert np.abs(pk - pstar).sum() <= rk / 0.15 + 1e-14
        assert oracle.pagerank_residual(g, pstar, 0.85) < 1e-14


# ------------------------------------------------------------------- CC ---
def test_cc_known_components_and_full_grid():
    edges = [(0, 3), (3, 7), (1, 2), (5, 6), (6, 8), (8, 5)]
    g = g_from_edges(10, edges)
    assert oracle.cc(g).tolist() == [0, 1, 1, 0, 4, 5, 5, 0, 5, 9]
    grid = oracle.csr_from_tuples(gen.grid(20, 20, p_delete=0.0, seed=1))
    assert np.all(oracle.cc(grid) == 0)


@pytest.mark.parametrize("seed", range(10))
def test_cc_brute_force_transitive_closure(seed):
    n = 6 + seed % 7
    edges, _ = small_edges(n, 0.15, 200 + seed)
    g = g_from_edges(n, edges)
    R = np.eye(n, dtype=bool)
    for u, v in edges:
        R[u, v] = R[v, u] = True
    for _ in range(n):
        R = R | ((R.astype(int) @ R.astype(int)) > 0)
    want = [int(np.flatnonzero(R[i])[0]) for i in range(n)]
    assert oracle.cc(g).tolist() == want


def test_cc_matches_scipy_on_rmat():
    g = oracle.csr_from_tuples(gen.rmat(11, 2, seed=8))
    k, lab = csg.connected_components(scipy_csr(g), directed=False)
    first = np.full(k, g.n)
    np.minimum.at(first, lab, np.arange(g.n))
    assert np.array_equal(oracle.cc(g), first[lab].astype(np.uint32))


# ------------------------------------------------------------------- TC ---
def test_tc_closed_forms():
    for n in (3, 4, 5, 8, 12):
        kn = g_from_edges(n, list(itertools.combinations(range(n), 2)))
        assert oracle.tc(kn) == math.comb(n, 3)
    tree = g_from_edges(15, [(i, (i - 1) // 2) for i in range(1, 15)])
    assert oracle.tc(tree) == 0
    bip = g_from_edges(9, [(a, b) for a in range(4) for b in range(4, 9)])
    assert oracle.tc(bip) == 0
    assert oracle.tc(oracle.csr_from_tuples(gen.grid(12, 12, 0.0, seed=1))) == 0
    for r in (4, 5, 9):
        wheel = [(0, i) for i in range(1, r + 1)] + [(i, i % r + 1) for i in range(1, r + 1)]
        assert oracle.tc(g_from_edges(r + 1, wheel)) == r


@pytest.mark.parametrize("seed", range(8))
def test_tc_brute_force_triple_loop(seed):
    n = 7 + seed % 6
    edges, _ = small_edges(n, 0.5, 300 + seed)
    E = set(edges) | {(v, u) for u, v in edges}
    want = sum(1 for a, b, c in itertools.combinations(range(n), 3)
               if (a, b) in E and (b, c) in E and (a, c) in E)
    assert oracle.tc(g_from_edges(n, edges)) == want


def test_tc_trace_of_cube_and_masked_LL_against_dense_products():
    g = oracle.csr_from_tuples(gen.rmat(8, 8, seed=4))
    A = dense_adj(g)
    total = oracle.tc(g)
    assert total == int(np.trace(A @ A @ A)) // 6
    new = oracle.degree_order(g)
    h = oracle.relabel(g, new)
    assert oracle.tc(h) == total
    L = np.tril(dense_adj(h), -1)
    C = (L @ L) * L
    vals, s = oracle.masked_LL(h)
    assert s == total == int(C.sum())
    rows, cols = np.nonzero(L)          # row-major order, as in CSR
    assert np.array_equal(vals.astype(np.int64), C[rows, cols])


def test_degree_order_invariants():
    g = oracle.csr_from_tuples(gen.rmat(9, 4, seed=12))
    new = oracle.degree_order(g)
    assert np.array_equal(np.sort(new), np.arange(g.n))
    deg = g.degrees()
    order = np.empty(g.n, dtype=np.int64)
    order[new] = np.arange(g.n)           # order[r] = old id with rank r
    d = deg[order]
    assert np.all(np.diff(d) <= 0)
    same = np.diff(d) == 0
    assert np.all(np.diff(order)[same] > 0)   # ties: lower old id first
    h = oracle.relabel(g, new)
    assert sorted(h.degrees().tolist()) == sorted(deg.tolist())


# ------------------------------------------------------ generic semantics ---
def _rand_mat(n, k, t, seed, vals=(1, 9)):
    rng = np.random.default_rng(seed)
    e = {}
    for _ in range(k):
        i, j = int(rng.integers(n)), int(rng.integers(n))
        e[(i, j)] = gbo.cast(t, int(rng.integers(*vals)))
    return gbo.Mat(n, n, t, e)


def _rand_vec(n, k, t, seed, vals=(1, 9)):
    rng = np.random.default_rng(seed)
    return gbo.Vec(n, t, {int(i): gbo.cast(t, int(rng.integers(*vals)))
                          for i in rng.choice(n, k, replace=False)})


def test_mxv_plus_times_equals_dense_matmul():
    n = 40
    A = _rand_mat(n, 300, "int32", 1)
    u = _rand_vec(n, 15, "int32", 2)
    w = gbo.mxv(gbo.Vec(n, "int32"), None, None, "PLUS_TIMES", A, u)
    D = np.zeros((n, n), np.int64)
    for (i, j), a in A.e.items():
        D[i, j] = a
    x = np.zeros(n, np.int64)
    for i, v in u.e.items():
        x[i] = v
    y = D @ x
    touched = (D != 0) @ (x != 0)
    for i in range(n):
        if touched[i]:
            assert w.e[i] == y[i]
        else:
            assert i not in w.e
    wt = gbo.vxm(gbo.Vec(n, "int32"), None, None, "PLUS_TIMES", u, A.T())
    assert wt.e == w.e                                  # vxm(u, A^T) = mxv(A, u)
    wt2 = gbo.mxv(gbo.Vec(n, "int32"), None, None, "PLUS_TIMES", A.T(), u, tran=True)
    assert wt2.e == w.e


def test_mxv_min_plus_brute_and_saturation():
    n = 30
    A = _rand_mat(n, 200, "uint32", 3, (1, 100))
    u = _rand_vec(n, 10, "uint32", 4, (0, 1000))
    u.e[next(iter(u.e))] = 2**32 - 1                   # "infinity" must absorb
    w = gbo.mxv(gbo.Vec(n, "uint32"), None, None, "MIN_PLUS", A, u)
    for i in range(n):
        cands = [min(a + u.e[j], 2**32 - 1) for (r, j), a in A.e.items() if r == i and j in u.e]
        if cands:
            assert w.e[i] == min(cands)
        else:
            assert i not in w.e


def test_mask_semantics_special_cases():
    n = 25
    A = _rand_mat(n, 120, "fp64", 5)
    u = _rand_vec(n, 12, "fp64", 6)
    w0 = gbo.Vec(n, "fp64", {i: -1.0 for i in range(0, n, 3)})
    full = gbo.mxv(w0, None, None, "PLUS_TIMES", A, u)
    ones = gbo.Vec(n, "bool", {i: True for i in range(n)})
    assert gbo.mxv(w0, ones, None, "PLUS_TIMES", A, u).e == full.e
    empty = gbo.Vec(n, "bool")
    assert gbo.mxv(w0, empty, None, "PLUS_TIMES", A, u, scmp=True).e == full.e
    assert gbo.mxv(w0, None, None, "PLUS_TIMES", A, u, scmp=True).e == w0.e
    assert gbo.mxv(w0, None, None, "PLUS_TIMES", A, u, scmp=True, replace=True).e == {}
    assert gbo.mxv(w0, empty, None, "PLUS_TIMES", A, u).e == w0.e
    m = gbo.Vec(n, "int32", {i: (i % 2) for i in range(0, n, 2)})   # stored zeros
    val = gbo.mxv(w0, m, None, "PLUS_TIMES", A, u)
    st = gbo.mxv(w0, m, None, "PLUS_TIMES", A, u, structural=True)
    for i in range(n):
        allowed_val = i in m.e and m.e[i] != 0
        allowed_st = i in m.e
        for got, allowed in ((val, allowed_val), (st, allowed_st)):
            if allowed:
                assert got.e.get(i) == full.e.get(i)
            else:
                assert got.e.get(i) == w0.e.get(i)
    rep = gbo.mxv(w0, m, None, "PLUS_TIMES", A, u, replace=True)
    assert set(rep.e) <= {i for i in m.e if m.e[i] != 0}
    acc = gbo.mxv(w0, None, "PLUS", "PLUS_TIMES", A, u)
    t = gbo.mxv(gbo.Vec(n, "fp64"), None, None, "PLUS_TIMES", A, u)
    for i in range(n):
        a, b = w0.e.get(i), t.e.get(i)
        if a is None and b is None:
            assert i not in acc.e
        else:
            assert acc.e[i] == (a or 0.0) + (b or 0.0)


def test_masked_equals_unmasked_then_ewise_mult():
    n = 35
    A = _rand_mat(n, 250, "uint32", 8)
    u = _rand_vec(n, 9, "uint32", 9)
    m = gbo.Vec(n, "bool", {i: True for i in range(0, n, 2)})
    w = gbo.Vec(n, "uint32")
    masked = gbo.mxv(w, m, None, "PLUS_TIMES", A, u)
    un = gbo.mxv(w, None, None, "PLUS_TIMES", A, u)
    both = gbo.ewise_mult(gbo.Vec(n, "uint32"), None, None, "FIRST", un,
                          gbo.Vec(n, "uint32", {i: 1 for i in m.e}))
    assert masked.e == both.e


def test_ewise_reduce_small_cases():
    u = gbo.Vec(6, "int32", {0: 3, 2: 5, 4: -1})
    v = gbo.Vec(6, "int32", {2: 7, 3: 2})
    assert gbo.ewise_add(gbo.Vec(6, "int32"), None, None, "PLUS", u, v).e == {0: 3, 2: 12, 3: 2, 4: -1}
    assert gbo.ewise_mult(gbo.Vec(6, "int32"), None, None, "TIMES", u, v).e == {2: 35}
    assert gbo.reduce_vector("int32", "PLUS", u) == 7
    assert gbo.reduce_vector("int32", "MIN", u) == -1
    assert gbo.reduce_vector("int32", "MAX", gbo.Vec(4, "int32")) == -2**31
    assert gbo.reduce_vector("uint32", "PLUS", gbo.Vec(3, "uint32", {0: 2**32 - 1, 1: 2})) == 1
    A = gbo.Mat(3, 3, "fp64", {(0, 1): 2.0, (0, 2): 3.0, (2, 0): -1.0})
    assert gbo.reduce_rows(gbo.Vec(3, "fp64"), None, None, "PLUS", A).e == {0: 5.0, 2: -1.0}
    assert gbo.reduce_matrix("fp64", "MAX", A) == 3.0


def test_mxm_masked_plus_pair_is_triangle_wedge_count():
    g = oracle.csr_from_tuples(gen.rmat(6, 6, seed=2))
    h = oracle.relabel(g, oracle.degree_order(g))
    L = np.tril(dense_adj(h), -1)
    Lm = gbo.Mat(h.n, h.n, "uint32", {(int(i), int(j)): 1 for i, j in zip(*np.nonzero(L))})
    C = gbo.mxm(gbo.Mat(h.n, h.n, "uint32"), Lm, None, "PLUS_PAIR", Lm, Lm, structural=True)
    D = (L @ L) * L
    for (i, j), c in C.e.items():
        assert c == D[i, j]
    assert sum(C.e.values()) == oracle.tc(h)


def test_running_example_masked_vxm():
    f = read_golden("running_example.txt")
    n = int(f["n"])
    edges = [tuple(map(int, e.split("-"))) for e in f["edges"].split()]
    A = gbo.Mat(n, n, "bool", {e: True for e in edges})
    assert len(A.e) == int(f["nnz"])
    fr = [int(x) for x in f["frontier"].split()]
    vis = [int(x) for x in f["visited"].split()]
    u = gbo.Vec(n, "bool", {i: True for i in fr})
    v = gbo.Vec(n, "bool", {i: True for i in vis})
    nb = gbo.vxm(gbo.Vec(n, "bool"), None, None, "LOR_LAND", u, A)
    assert sorted(nb.e) == [int(x) for x in f["neighbours_of_frontier"].split()]
    nxt = gbo.vxm(gbo.Vec(n, "bool"), v, None, "LOR_LAND", u, A, scmp=True)
    assert sorted(nxt.e) == [int(x) for x in f["next_frontier"].split()]
    # Table 8 costs: SpMSpV reads the columns of the frontier, the mask-first
    # SpMV reads the rows (of A^T) of the unvisited vertices, GEMV reads n^2
    assert sum(1 for (i, j) in edges if i in fr) == int(f["spmspv_loads"])
    unvisited = set(range(n)) - set(vis)
    assert sum(1 for (i, j) in edges if j in unvisited) == int(f["masked_spmv_loads"])
    assert n * n == int(f["gemv_loads"])
    # the same step as a BFS transition of the oracle on the undirected
    # version is not asserted: the figure's graph is directed
