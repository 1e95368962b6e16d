"""GPU parity: matrix build (CSR/CSC) and direction-optimised BFS against
the oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1908_01407_gb300 as gb

pytestmark = pytest.mark.gpu


def make(ctx, t, weights=False, flags=gb.SYMMETRIC):
    g = oracle.csr_from_tuples(t)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w if weights else None, type_=gb.UINT32, flags=flags)
    return g, A


# ------------------------------------------------------------------ build
@pytest.mark.parametrize("scale,ef", [(10, 8), (14, 16)])
def test_build_csr_matches_oracle(ctx, scale, ef):
    t = gen.rmat(scale, ef, seed=scale, wmax=255)
    g, A = make(ctx, t, weights=True, flags=gb.BUILD_DEFAULT)
    rp, ci, v = A.export_csr(with_vals=True)
    assert A.nvals == g.m
    assert np.array_equal(rp.astype(np.uint64), g.rowptr)
    assert np.array_equal(ci, g.colidx)
    assert np.array_equal(v, g.vals)
    cp, ri, cv = A.export_csc(with_vals=True)
    rows = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.rowptr).astype(np.int64))
    gt = oracle.csr_build(g.n, g.colidx, rows, g.vals)
    assert np.array_equal(cp.astype(np.uint64), gt.rowptr)
    assert np.array_equal(ri, gt.colidx)
    assert np.array_equal(cv, gt.vals)
    A.free()


@pytest.mark.parametrize("dup,odup", [(gb.PLUS, oracle.DUP_PLUS), (gb.MIN, oracle.DUP_MIN), (gb.MAX, oracle.DUP_MAX),
                                      (gb.FIRST, oracle.DUP_FIRST), (gb.SECOND, oracle.DUP_SECOND)])
def test_build_dup_operators_and_rectangular(ctx, dup, odup):
    rng = np.random.default_rng(3)
    nr, nc, nt = 777, 1234, 60000      # ragged sizes, many duplicates
    r = rng.integers(0, nr, nt).astype(np.uint32)
    c = rng.integers(0, nc, nt).astype(np.uint32)
    v = rng.integers(0, 1 << 20, nt).astype(np.uint32)
    A = gb.Matrix(ctx, gb.UINT32, nr, nc)
    A.build(torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), torch.from_numpy(v).cuda(), dup=dup)
    g = oracle.csr_build(nr, r, c, v, odup, ncols=nc)
    rp, ci, vv = A.export_csr(with_vals=True)
    assert np.array_equal(rp.astype(np.uint64), g.rowptr)
    assert np.array_equal(ci, g.colidx)
    assert np.array_equal(vv, g.vals)
    A.free()


def test_build_errors_and_empty(ctx):
    A = gb.Matrix(ctx, gb.UINT32, 10, 10)
    with pytest.raises(gb.GBError) as e:
        A.build(np.array([1, 10], np.uint32), np.array([0, 0], np.uint32))
    assert e.value.code == gb.INVALID_INDEX
    A.build(np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert A.nvals == 0
    rp, ci = A.export_csr()
    assert np.all(rp == 0)
    A.free()


# -------------------------------------------------------------------- BFS
def check_bfs(ctx, g, A, src, desc=None):
    lv, par, st = gb.bfs(ctx, A, src, desc=desc)
    torch.cuda.synchronize()
    lv, par = lv.cpu().numpy(), par.cpu().numpy()
    want = oracle.bfs(g, src)
    assert np.array_equal(lv, want)
    assert oracle.bfs_parent_violations(g, src, lv, par) == 0
    assert st["status"] == 0
    assert st["vertices_reached"] == int((want >= 0).sum())
    assert st["depth"] == int(want.max()) + 1
    return st


def test_bfs_rmat_s14_max_degree_source(ctx):
    """R-MAT scale 14, edge factor 16, seed 1, source = max-degree vertex."""
    t = gen.rmat(14, 16, seed=1)
    g, A = make(ctx, t)
    deg = g.degrees()
    src = int(np.flatnonzero(deg == deg.max())[0])
    st = check_bfs(ctx, g, A, src)
    assert st["push_levels"] >= 1
    for s in gen.sources(t, 8, seed=1):
        check_bfs(ctx, g, A, int(s))
    A.free()


@pytest.mark.parametrize("direction", [gb.PUSH, gb.PULL, gb.AUTO])
def test_bfs_directions_agree(ctx, direction):
    t = gen.rmat(13, 16, seed=7)
    g, A = make(ctx, t)
    d = gb.Descriptor(direction=direction)
    for s in gen.sources(t, 4, seed=3):
        st = check_bfs(ctx, g, A, int(s), d)
        if direction == gb.PUSH:
            assert st["pull_levels"] == 0
        if direction == gb.PULL:
            assert st["push_levels"] == 0
    d.free()
    A.free()


@pytest.mark.parametrize("beta", [1, 4, 10, 40, 1000])
def test_bfs_switch_threshold_does_not_change_levels(ctx, beta):
    t = gen.rmat(12, 16, seed=11)
    g, A = make(ctx, t)
    d = gb.Descriptor(beta=beta)
    check_bfs(ctx, g, A, int(gen.sources(t, 1, seed=2)[0]), d)
    A.free()


def test_bfs_closed_form_graphs_and_edge_cases(ctx):
    cases = [
        gen.from_edges(37, [(i, i + 1) for i in range(36)]),                 # path, ragged n
        gen.from_edges(70, [(0, i) for i in range(1, 70)]),                  # star
        gen.from_edges(6, [(0, 1), (1, 2), (3, 4), (4, 5)]),                # two components
        gen.grid(33, 31, 0.0, seed=1),                                       # full grid
        gen.grid(64, 64, 0.1, seed=3),                                       # grid with deletions
        gen.from_edges(1, []),                                               # a single vertex
        gen.from_edges(5, [(1, 2)]),                                         # isolated source
    ]
    for t in cases:
        g, A = make(ctx, t)
        for src in sorted({0, t.n // 2, t.n - 1}):
            for direction in (gb.AUTO, gb.PUSH, gb.PULL):
                d = gb.Descriptor(direction=direction)
                check_bfs(ctx, g, A, src, d)
                d.free()
        A.free()


def test_bfs_csr_only_and_host_buffers(ctx):
    t = gen.rmat(11, 8, seed=5)
    g = oracle.csr_from_tuples(t)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.CSR_ONLY)
    src = int(gen.sources(t, 1, seed=9)[0])
    lv = np.empty(t.n, np.int32)
    par = np.empty(t.n, np.int32)
    _, _, st = gb.bfs(ctx, A, src, lv, par)          # push only (no CSC)
    assert st["pull_levels"] == 0
    assert np.array_equal(lv, oracle.bfs(g, src))
    assert oracle.bfs_parent_violations(g, src, lv, par) == 0
    with pytest.raises(gb.GBError) as e:
        gb.bfs(ctx, A, t.n, lv, par)
    assert e.value.code == gb.INVALID_INDEX
    A.free()


def test_bfs_directed_matrix_uses_csr_and_csc(ctx):
    """A non-symmetric matrix: BFS follows edges i -> j (f' = f A)."""
    rng = np.random.default_rng(5)
    n = 3000
    r = rng.integers(0, n, 20000).astype(np.uint32)
    c = rng.integers(0, n, 20000).astype(np.uint32)
    A = gb.Matrix.from_tuples(ctx, n, r, c)
    g = oracle.csr_build(n, r, c)
    for direction in (gb.AUTO, gb.PUSH, gb.PULL):
        d = gb.Descriptor(direction=direction)
        lv, par, st = gb.bfs(ctx, A, 7, desc=d)
        lv = lv.cpu().numpy()
        assert np.array_equal(lv, oracle.bfs(g, 7))
        d.free()
    A.free()


@pytest.mark.slow
def test_bfs_rmat_s22_full_size_sampled_sources(ctx):
    """R-MAT scale 22, edge factor 16, seed 2: the benchmark graph, in the
    benchmark's launch configuration, three of its 64 sources."""
    t = gen.rmat(22, 16, seed=2)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    g = oracle.csr_from_tuples(t)
    assert A.nvals == g.m
    srcs = gen.sources(t, 64, seed=1)
    for s in srcs[:3]:
        st = check_bfs(ctx, g, A, int(s))
        assert st["pull_levels"] >= 1
    A.free()


def test_bfs_autotune_picks_a_candidate_and_keeps_results(ctx):
    t = gen.rmat(13, 16, seed=12)
    g, A = make(ctx, t)
    beta, ms = gb.bfs_autotune(ctx, A, gen.sources(t, 4, seed=99))
    assert beta in (4, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64, 96, 128, 192, 256) and ms > 0
    w, b = gb.bfs_get_shape(A)
    assert w in (1, 2, 4) and b in (0, 1)
    for s in gen.sources(t, 4, seed=1):
        check_bfs(ctx, g, A, int(s))          # default descriptor: the tuned beta and shape
    A.free()


@pytest.mark.parametrize("case", ["rmat14", "grid", "layered"])
def test_bfs_every_tile_shape_matches_the_oracle(ctx, case):
    """Every tile shape the autotuner can pick (pull candidates per lane x
    blocks per SM), with the default descriptor and forced pull: levels
    bit-exact, parents valid."""
    if case == "layered":
        t, src0 = layered_graph()
    else:
        t = {"rmat14": lambda: gen.rmat(14, 16, seed=3), "grid": lambda: gen.grid(70, 61, 0.1, seed=2)}[case]()
        src0 = int(gen.sources(t, 1, seed=5)[0])
    g, A = make(ctx, t)
    srcs = [src0] + [int(s) for s in gen.sources(t, 2, seed=7)]
    pull = gb.Descriptor(direction=gb.PULL)
    for w in (1, 2, 4):
        for b in (0, 1, 2, 3, 4):
            gb.bfs_set_shape(A, w, b)
            assert gb.bfs_get_shape(A) == (w, b)
            for s in srcs:
                check_bfs(ctx, g, A, s)
                check_bfs(ctx, g, A, s, pull)
    gb.bfs_set_shape(A, 0, 0)
    assert gb.bfs_get_shape(A) == (2, 0)
    for bad in ((3, 0), (8, 0), (2, 5)):
        with pytest.raises(gb.GBError) as e:
            gb.bfs_set_shape(A, *bad)
        assert e.value.code == gb.INVALID_VALUE
    pull.free()
    A.free()


def layered_graph(wide=300, nwide=4, clique=40, isolated=5000, seed=4):
    """src - W1 - b1 - W2 - b2 - ...: every W is a clique joined completely
    to the single vertices before and after it, so the frontier alternates
    between many out-edges (a W) and few (a b); plus a separate clique
    (reachable by a pull never) and vertices without edges. Vertex ids are
    permuted. Returns (tuples, source)."""
    edges = []
    nxt, prev = 1, [0]
    for _ in range(nwide):
        W = list(range(nxt, nxt + wide))
        nxt += wide
        edges += [(u, v) for u in prev for v in W] + [(W[i], W[j]) for i in range(wide) for j in range(i)]
        b = nxt
        nxt += 1
        edges += [(u, b) for u in W]
        prev = [b]
    c0 = nxt
    edges += [(c0 + i, c0 + j) for i in range(clique) for j in range(i)]
    nxt += clique + isolated
    perm = np.random.default_rng(seed).permutation(nxt)
    return gen.from_edges(nxt, [(int(perm[u]), int(perm[v])) for u, v in edges]), int(perm[0])


def test_bfs_pull_push_pull_keeps_candidates(ctx):
    """Directions alternate push, pull, push, pull, ...: each pull starts
    from the candidates the previous pull left, some of which a push has
    claimed in between; the clique component stays a candidate throughout."""
    t, src = layered_graph()
    g, A = make(ctx, t)
    d = gb.Descriptor(beta=10)
    st = check_bfs(ctx, g, A, src, d)
    dirs = "".join("P" if x["dir"] == "pull" else "s" for x in st["trace"])
    assert dirs == "sPsPsPsP", dirs     # b4 ends the component: its level is not expanded
    d.free()
    # the same graph with the pulls only
    d = gb.Descriptor(direction=gb.PULL)
    check_bfs(ctx, g, A, src, d)
    d.free()
    A.free()


@pytest.mark.parametrize("case", ["rmat14", "rmat18", "grid", "path", "star", "two", "single", "isolated_src"])
def test_bfs_single_cluster_schedule(ctx, case):
    """The single-cluster schedule gives the same levels (and valid parents)
    as the oracle; rmat18's middle frontiers overflow the CTAs' shared lists
    into the global list, the star's hub row is expanded warp-cooperatively,
    the path has 300 levels."""
    t = {"rmat14": lambda: gen.rmat(14, 16, seed=1),
         "rmat18": lambda: gen.rmat(18, 16, seed=5),
         "grid": lambda: gen.grid(200, 150, 0.1, seed=3),
         "path": lambda: gen.from_edges(300, [(i, i + 1) for i in range(299)]),
         "star": lambda: gen.from_edges(5000, [(0, i) for i in range(1, 5000)]),
         "two": lambda: gen.from_edges(6, [(0, 1), (1, 2), (3, 4), (4, 5)]),
         "single": lambda: gen.from_edges(1, []),
         "isolated_src": lambda: gen.from_edges(70, [(1, 2), (2, 3)])}[case]()
    g, A = make(ctx, t)
    d = gb.Descriptor(schedule=gb.SCHED_CLUSTER)
    srcs = [0, t.n - 1] if t.n > 1 else [0]
    if case.startswith("rmat"):
        srcs = [int(s) for s in gen.sources(t, 3, seed=4)]
    for src in srcs:
        st = check_bfs(ctx, g, A, src, d)
        assert st["schedule"] == gb.SCHED_CLUSTER
    d.free()
    A.free()


def test_bfs_autotune_chooses_a_high_diameter_schedule_for_a_long_path(ctx):
    """A 3000-vertex path has 3000 levels of one vertex each: the cluster or
    the barrier-free schedule wins over the persistent grid and becomes the
    matrix's default; the results and the statistics are the same."""
    t = gen.from_edges(3000, [(i, i + 1) for i in range(2999)])
    g, A = make(ctx, t)
    gb.bfs_autotune(ctx, A, np.array([0, 1500], np.uint32))
    st = check_bfs(ctx, g, A, 0)
    assert st["schedule"] in (gb.SCHED_CLUSTER, gb.SCHED_ASYNC)
    d = gb.Descriptor(schedule=gb.SCHED_GRID)      # the descriptor overrides the tuned choice
    st = check_bfs(ctx, g, A, 0, d)
    assert st["schedule"] == gb.SCHED_GRID
    d.free()
    A.free()


@pytest.mark.parametrize("schedule", [gb.SCHED_GRID, gb.SCHED_CLUSTER, gb.SCHED_ASYNC])
@pytest.mark.parametrize("out", ["pinned", "numpy", "device", "levels_only"])
def test_bfs_batch_rows_match_the_oracle(ctx, schedule, out):
    """gb_bfs_batch: row q is the BFS from source q (levels exactly, parents a
    valid BFS tree), with host outputs through the two alternating device
    buffers (odd k, so both buffers and the last half-filled pair are used)."""
    t = gen.rmat(15, 16, seed=2)
    g, A = make(ctx, t)
    srcs = [int(s) for s in gen.sources(t, 7, seed=11)]
    srcs[3] = srcs[1]                                  # a repeated source
    k, n = len(srcs), t.n
    d = gb.Descriptor(schedule=schedule)
    if out == "pinned":
        lv = torch.empty((k, n), dtype=torch.int32).pin_memory()
        par = torch.empty((k, n), dtype=torch.int32).pin_memory()
    elif out == "numpy":
        lv, par = np.empty((k, n), np.int32), np.empty((k, n), np.int32)
    elif out == "levels_only":
        lv, par = np.empty((k, n), np.int32), False
    else:
        lv, par = None, None
    lv, par = gb.bfs_batch(ctx, A, np.array(srcs, np.uint32), lv, par, desc=d)
    torch.cuda.synchronize()
    lv = lv.cpu().numpy() if isinstance(lv, torch.Tensor) else lv
    if par is not None:
        par = par.cpu().numpy() if isinstance(par, torch.Tensor) else par
    for q, s in enumerate(srcs):
        want = oracle.bfs(g, s)
        assert np.array_equal(lv[q], want), q
        if par is not None:
            assert oracle.bfs_parent_violations(g, s, lv[q], par[q]) == 0, q
    d.free()
    A.free()


def test_bfs_batch_errors(ctx):
    t = gen.rmat(10, 8, seed=3)
    g, A = make(ctx, t)
    lv = np.empty((2, t.n), np.int32)
    with pytest.raises(gb.GBError) as e:
        gb.bfs_batch(ctx, A, np.array([0, t.n], np.uint32), lv, False)
    assert e.value.code == gb.INVALID_INDEX
    with pytest.raises(gb.GBError) as e:
        gb.bfs_batch(ctx, A, np.array([], np.uint32), lv, False)
    assert e.value.code == gb.INVALID_VALUE
    A.free()


def test_bfs_stays_in_pull_when_few_candidates_are_left(ctx):
    """src - 200 hubs (a clique) - 50 leaves each, 5 leaves with one child,
    and a separate 150-clique. With beta = 4, Table 9's rule pushes the
    level of the 10,000 leaves (|E_f| * 4 < |E|), but the first pull left
    only the 5 children and the clique (155 candidates, 22,355 in-edges),
    fewer reads than the push plus building its list: that level pulls. The
    next level (the 5 children, one of which has a child; the clique still
    left) pushes, and the level of that grandchild, which completes the
    component, is not expanded."""
    edges, nxt = [], 1
    hubs = list(range(nxt, nxt + 200))
    nxt += 200
    edges += [(0, h) for h in hubs] + [(hubs[i], hubs[j]) for i in range(200) for j in range(i)]
    leaves = []
    for h in hubs:
        edges += [(h, nxt + k) for k in range(50)]
        leaves += list(range(nxt, nxt + 50))
        nxt += 50
    for k in range(5):
        edges.append((leaves[k * 997], nxt))
        nxt += 1
    edges.append((nxt - 1, nxt))
    nxt += 1
    c0 = nxt
    edges += [(c0 + i, c0 + j) for i in range(150) for j in range(i)]
    nxt += 150 + 64
    perm = np.random.default_rng(7).permutation(nxt)
    t = gen.from_edges(nxt, [(int(perm[u]), int(perm[v])) for u, v in edges])
    g, A = make(ctx, t)
    d = gb.Descriptor(beta=4)
    st = check_bfs(ctx, g, A, int(perm[0]), d)
    dirs = "".join("P" if x["dir"] == "pull" else "s" for x in st["trace"])
    assert dirs == "sPPs", dirs
    d.free()
    A.free()


def test_bfs_stops_once_the_component_is_reached(ctx):
    """The build keeps each vertex's component size on the matrix; a BFS that
    has reached its source's whole component leaves its last frontier
    unexpanded (one traced level fewer than the depth) while levels,
    parents, depth and reached count still match the oracle: sources in the
    giant component, in a small one, and an isolated source."""
    t = gen.rmat(14, 16, seed=1)
    g, A = make(ctx, t)
    lab = oracle.cc(g)
    size = np.bincount(lab, minlength=t.n)[lab]
    deg = g.degrees()
    giant = [int(s) for s in gen.sources(t, 3, seed=5)]
    small = [int(np.flatnonzero((size > 1) & (size < 10))[0])]
    isolated = [int(np.flatnonzero(deg == 0)[0])]
    d = gb.Descriptor(schedule=gb.SCHED_GRID)
    for s in giant + small + isolated:
        st = check_bfs(ctx, g, A, s, d)
        assert len(st["trace"]) == st["depth"] - 1, (s, st["depth"], len(st["trace"]))
    d.free()
    A.free()


def test_bfs_with_self_loops_and_a_directed_build(ctx):
    """A matrix built from tuples with self-loops (no symmetric flag: CSR and
    CSC): a self-loop never makes a vertex its own parent or moves its level,
    in any direction; the component early stop still holds."""
    rows = np.array([0, 0, 1, 1, 2, 2, 3, 3, 4, 5, 5, 6], np.uint32)
    cols = np.array([0, 1, 0, 2, 1, 3, 2, 3, 4, 6, 5, 5], np.uint32)
    n = 8
    g = oracle.csr_build(n, rows, cols)
    A = gb.Matrix.from_tuples(ctx, n, rows, cols)
    for direction in (gb.AUTO, gb.PUSH, gb.PULL):
        d = gb.Descriptor(direction=direction)
        for src in (0, 3, 4, 5, 7):
            lv, par, st = gb.bfs(ctx, A, src, desc=d)
            torch.cuda.synchronize()
            lv, par = lv.cpu().numpy(), par.cpu().numpy()
            assert np.array_equal(lv, oracle.bfs(g, src)), (direction, src)
            assert oracle.bfs_parent_violations(g, src, lv, par) == 0
            assert par[src] == src
        d.free()
    A.free()


def test_bfs_batch_single_vertex_graph(ctx):
    t = gen.from_edges(1, [])
    g, A = make(ctx, t)
    lv, par = gb.bfs_batch(ctx, A, np.zeros(3, np.uint32), np.empty((3, 1), np.int32), np.empty((3, 1), np.int32))
    assert lv.tolist() == [[0], [0], [0]] and par.tolist() == [[0], [0], [0]]
    A.free()


@pytest.mark.parametrize("case", ["rmat_even", "rmat_odd", "directed", "csr_only", "isolated", "single", "many"])
def test_bfs_batch_device_rows_match_the_oracle(ctx, case):
    """gb_bfs_batch with device outputs: each row equals the oracle's BFS
    (levels exactly, parents valid), for an even and an odd number of runs, a
    directed matrix (pulls over its CSC), a CSR-only matrix (push only),
    isolated sources among others, one run, and 75 runs with repeated and
    isolated sources; a second batch on the same workspace gives the same
    rows."""
    if case in ("directed", "csr_only"):
        rng = np.random.default_rng(17)
        n = 5000
        r = rng.integers(0, n, 60000).astype(np.uint32)
        c = rng.integers(0, n, 60000).astype(np.uint32)
        A = gb.Matrix.from_tuples(ctx, n, r, c, flags=gb.CSR_ONLY if case == "csr_only" else gb.BUILD_DEFAULT)
        g = oracle.csr_build(n, r, c)
        srcs = [3, 11, 4999, 250, 7]
    else:
        t = gen.rmat(14, 16, seed=21)
        g, A = make(ctx, t)
        n = t.n
        srcs = [int(s) for s in gen.sources(t, {"rmat_even": 8, "rmat_odd": 9, "isolated": 4, "single": 1,
                                                 "many": 65}[case], seed=5)]
        if case == "many":
            deg = np.diff(g.rowptr.astype(np.int64))
            iso = [int(v) for v in np.flatnonzero(deg == 0)[:5]]
            srcs = srcs[:30] + iso + srcs[:5] + srcs[30:]
        if case == "isolated":
            deg = np.diff(g.rowptr.astype(np.int64))
            iso = [int(v) for v in np.flatnonzero(deg == 0)[:2]]
            srcs = [iso[0], srcs[0], iso[1], srcs[1], srcs[2]]
    k = len(srcs)
    for _ in range(2):
        lv = torch.full((k, n), 9, dtype=torch.int32, device="cuda")
        par = torch.full((k, n), 9, dtype=torch.int32, device="cuda")
        gb.bfs_batch(ctx, A, np.array(srcs, np.uint32), lv, par)
        torch.cuda.synchronize()
        lv, par = lv.cpu().numpy(), par.cpu().numpy()
        for q, s in enumerate(srcs):
            assert np.array_equal(lv[q], oracle.bfs(g, s)), (case, q)
            assert oracle.bfs_parent_violations(g, s, lv[q], par[q]) == 0, (case, q)
    A.free()
