"""GPU parity of the barrier-free schedule (GB_SCHED_ASYNC, gb_cc_async):
SSSP distances bit-exact against Dijkstra for every distance-bucket width,
BFS levels bit-exact against the queue BFS with valid parents (each the
smallest in-neighbour one level up), component labels bit-exact against
union-find; small, ragged, directed, disconnected and degenerate graphs and
the 4096 x 4096 grid at full size."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1908_01407_gb300 as gb

pytestmark = pytest.mark.gpu


def graphs(ctx, case):
    """(oracle CSR, matrix, n, sources) of one test graph."""
    if case == "directed":
        rng = np.random.default_rng(11)
        n = 2500
        r = rng.integers(0, n, 12000).astype(np.uint32)
        c = rng.integers(0, n, 12000).astype(np.uint32)
        w = rng.integers(1, 300, 12000).astype(np.uint32)
        return oracle.csr_build(n, r, c, w), gb.Matrix.from_tuples(ctx, n, r, c, w, type_=gb.UINT32), n, [0, 7, 2499]
    t = {"grid": lambda: gen.grid(150, 131, 0.1, seed=5, wmax=1000),
         "rmat12": lambda: gen.rmat(12, 16, seed=21, wmax=255),
         "path": lambda: gen.from_edges(2049, [(i, i + 1) for i in range(2048)], [1 + i % 13 for i in range(2048)]),
         "star": lambda: gen.from_edges(3001, [(0, i) for i in range(1, 3001)],
                                        [1 + (i * 37) % 900 for i in range(1, 3001)]),
         "pieces": lambda: gen.grid(70, 45, 0.45, seed=8, wmax=50),
         "single": lambda: gen.from_edges(1, [], []),
         "pair": lambda: gen.from_edges(2, [], [])}[case]()
    w = t.w if t.w is not None else np.ones_like(t.src)
    g = oracle.csr_from_tuples(gen.Tuples(t.n, t.src, t.dst, w, t.name))
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, w, type_=gb.UINT32, flags=gb.SYMMETRIC)
    srcs = sorted({0, t.n // 3, t.n - 1}) if t.n > 1 else [0]
    return g, A, t.n, srcs


CASES = ["grid", "rmat12", "path", "star", "pieces", "directed", "single", "pair"]


@pytest.mark.parametrize("case", CASES)
def test_async_sssp_matches_dijkstra_for_every_bucket_width(ctx, case):
    g, A, n, srcs = graphs(ctx, case)
    for delta in (0, 1, 7, 300, 2**31 - 1):
        d = gb.Descriptor(schedule=gb.SCHED_ASYNC, sssp_delta=delta)
        for src in srcs:
            dist = np.empty(n, np.uint32)
            _, it, st = gb.sssp(ctx, A, src, dist, d, stats=True)
            assert np.array_equal(dist, oracle.sssp(g, src)), (case, delta, src)
            assert st["schedule"] == gb.SCHED_ASYNC and st["status"] == 0
            assert it >= 1
        d.free()
    A.free()


@pytest.mark.parametrize("case", CASES)
def test_async_bfs_levels_and_parents(ctx, case):
    g, A, n, srcs = graphs(ctx, case)
    d = gb.Descriptor(schedule=gb.SCHED_ASYNC)
    for src in srcs:
        lv = np.empty(n, np.int32)
        par = np.empty(n, np.int32)
        _, _, st = gb.bfs(ctx, A, src, lv, par, desc=d)
        want = oracle.bfs(g, src)
        assert np.array_equal(lv, want), (case, src)
        assert st["schedule"] == gb.SCHED_ASYNC and st["status"] == 0
        assert st["depth"] == int(want.max()) + 1 and st["vertices_reached"] == int((want >= 0).sum())
        assert oracle.bfs_parent_violations(g, src, lv, par) == 0
        # each parent is the smallest in-neighbour one level up
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.rowptr.astype(np.int64)))
        cols = g.colidx.astype(np.int64)
        ok = (want[rows] >= 0) & (want[cols] == want[rows] + 1)
        exp = np.full(n, np.iinfo(np.int64).max, np.int64)
        np.minimum.at(exp, cols[ok], rows[ok])
        exp[src] = src
        exp[want < 0] = -1
        assert np.array_equal(par.astype(np.int64), exp), (case, src)
        # device outputs, no parents
        dl = torch.empty(n, dtype=torch.int32, device="cuda")
        gb.bfs(ctx, A, src, dl, False, desc=d, stats=False)
        torch.cuda.synchronize()
        assert np.array_equal(dl.cpu().numpy(), want)
    d.free()
    A.free()


@pytest.mark.parametrize("case", ["grid", "rmat12", "path", "star", "pieces", "single", "pair"])
def test_async_cc_matches_union_find(ctx, case):
    """Barrier-free min-label components equal union-find's canonical labels
    for every label-bucket width: the automatic one, narrow buckets (many
    phases), a width that leaves a ragged last bucket, and one bucket."""
    g, A, n, _ = graphs(ctx, case)
    want = oracle.cc(g)
    lab = np.empty(n, np.uint32)
    for bucket in (0, 5, 333, 2**32 - 1):
        _, st = gb.cc_async(ctx, A, lab, stats=True, bucket=bucket)
        assert np.array_equal(lab, want), (case, bucket)
        assert st["status"] == 0 and st["schedule"] == gb.SCHED_ASYNC
    # twice in a row on device memory: the launch leaves nothing behind
    dl = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(2):
        gb.cc_async(ctx, A, dl)
        torch.cuda.synchronize()
        assert np.array_equal(dl.cpu().numpy().view(np.uint32), want)
    A.free()


def test_async_stats_count_the_work(ctx):
    """Items, edges and bytes reported by the barrier-free SSSP follow from
    its definition: every reachable vertex is relaxed at least once, each
    relaxation reads its whole row, and the algorithmic bytes are the stated
    sum of those counts."""
    t = gen.grid(120, 97, 0.1, seed=4, wmax=1000)
    g = oracle.csr_from_tuples(t)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
    src = gen.first_nonisolated(t)
    d = gb.Descriptor(schedule=gb.SCHED_ASYNC)
    dist = np.empty(t.n, np.uint32)
    _, it, st = gb.sssp(ctx, A, src, dist, d, stats=True)
    want = oracle.sssp(g, src)
    assert np.array_equal(dist, want)
    reach = want != np.iinfo(np.uint32).max
    deg = np.diff(g.rowptr.astype(np.int64))
    assert st["vertices_reached"] >= reach.sum()
    assert st["edges_examined"] >= deg[reach].sum()
    assert st["depth"] == it >= 1
    d.free()
    A.free()


@pytest.mark.slow
def test_async_grid_4096_full_size(ctx):
    """The 4096 x 4096 grid with 10% of its edges deleted (seed 3), weights
    in [1, 1000]: barrier-free SSSP, BFS and components against Dijkstra,
    queue BFS and union-find."""
    t = gen.grid(4096, 4096, 0.1, seed=3, wmax=1000)
    g = oracle.csr_from_tuples(t)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
    src = gen.first_nonisolated(t)
    d = gb.Descriptor(schedule=gb.SCHED_ASYNC)
    dist = torch.empty(t.n, dtype=torch.int32, device="cuda")
    gb.sssp(ctx, A, src, dist, d)
    assert np.array_equal(dist.cpu().numpy().view(np.uint32), oracle.sssp(g, src))
    lv = torch.empty(t.n, dtype=torch.int32, device="cuda")
    par = torch.empty(t.n, dtype=torch.int32, device="cuda")
    gb.bfs(ctx, A, src, lv, par, desc=d)
    lvh = lv.cpu().numpy()
    assert np.array_equal(lvh, oracle.bfs(g, src))
    assert oracle.bfs_parent_violations(g, src, lvh, par.cpu().numpy()) == 0
    lab = torch.empty(t.n, dtype=torch.int32, device="cuda")
    gb.cc_async(ctx, A, lab)
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), oracle.cc(g))
    d.free()
    A.free()
