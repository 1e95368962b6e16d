"""The serving loop: every result of a concurrent BFS/SSSP/PageRank mix is
the same as the result of the same request run alone (BFS levels and SSSP
distances bit-exact, PageRank bit-identical), concurrent BFS requests on one
graph are batched into multi-source launches, admission by the HBM budget,
and the error paths."""
import concurrent.futures as cf

import numpy as np
import pytest

import gen
import oracle
import paper_1908_01407_gb300 as gb

pytestmark = pytest.mark.gpu


def graphs(ctx):
    out = []
    for scale, seed in ((10, 1001), (12, 1002), (13, 1003)):
        t = gen.rmat(scale, 16, seed=seed, wmax=255)
        A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
        out.append((t, A))
    return out


def alone(ctx, t, A, kind, src):
    if kind == gb.REQ_BFS:
        lv = np.empty(t.n, np.int32)
        gb.bfs(ctx, A, src, lv, False, stats=False)
        return lv
    if kind == gb.REQ_SSSP:
        d = np.empty(t.n, np.uint32)
        gb.sssp(ctx, A, src, d)
        return d
    r = np.empty(t.n, np.float32)
    gb.pagerank(ctx, A, 0.85, 50, r, residuals=False)
    return r


def test_results_same_alone_and_in_the_mix(ctx):
    G = graphs(ctx)
    S = gb.Server(ctx, max_inflight=4, batch_window_us=300)
    ids = [S.add_graph(A) for _, A in G]
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(160):
        g = int(rng.integers(len(G)))
        kind = [gb.REQ_BFS] * 6 + [gb.REQ_SSSP] * 3 + [gb.REQ_PAGERANK]
        kind = kind[int(rng.integers(10))]
        t = G[g][0]
        src = int(gen.sources(t, 50, seed=7)[int(rng.integers(50))])
        reqs.append((g, kind, src))
    # submit from several threads at once so requests arrive while others run
    def submit(r):
        g, kind, src = r
        return S.submit(kind, ids[g], src)
    with cf.ThreadPoolExecutor(8) as ex:
        tickets = list(ex.map(submit, reqs))
    results = []
    for tk, (g, kind, src) in zip(tickets, reqs):
        res = S.wait(tk, 120000)
        assert res.status == gb.SUCCESS
        results.append((S.fetch(tk, res.n, kind), res))
    st = S.stats()
    assert st["completed"] == len(reqs)
    assert st["batched_bfs"] > st["batches"] * 0 and st["p99_us"] >= st["p50_us"] > 0
    assert any(r.batch_size > 1 for _, r in results)        # BFS requests were packed
    for (got, res), (g, kind, src) in zip(results, reqs):
        t, A = G[g]
        want = alone(ctx, t, A, kind, src)
        if kind == gb.REQ_PAGERANK:
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
        else:
            assert np.array_equal(got.view(want.dtype), want)
    # and against the oracle for a sample
    for (got, res), (g, kind, src) in list(zip(results, reqs))[:20]:
        t, A = G[g]
        go = oracle.csr_from_tuples(t)
        if kind == gb.REQ_BFS:
            assert np.array_equal(got, oracle.bfs(go, src))
        elif kind == gb.REQ_SSSP:
            assert np.array_equal(got.view(np.uint32), oracle.sssp(go, src))
        else:
            p, _ = oracle.pagerank(go, 0.85, 50)
            assert np.abs(got.astype(np.float64) - p).sum() <= 1e-5
    S.destroy()
    for _, A in G:
        A.free()


def test_bfs_burst_is_batched(ctx):
    t = gen.rmat(12, 16, seed=3)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    S = gb.Server(ctx, max_inflight=2, batch_window_us=2000)
    gid = S.add_graph(A)
    srcs = gen.sources(t, 128, seed=2)
    tickets = [S.submit(gb.REQ_BFS, gid, int(s)) for s in srcs]
    g = oracle.csr_from_tuples(t)
    sizes = []
    for tk, s in zip(tickets, srcs):
        r = S.wait(tk)
        sizes.append(r.batch_size)
        assert np.array_equal(S.fetch(tk, r.n, gb.REQ_BFS), oracle.bfs(g, int(s)))
    st = S.stats()
    assert st["batches"] < len(srcs) and max(sizes) > 8
    S.destroy()
    A.free()


def test_admission_budget_and_errors(ctx):
    t = gen.rmat(11, 8, seed=4, wmax=9)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
    # a budget too small for any job: requests fail with OUT_OF_MEMORY, nothing hangs
    S = gb.Server(ctx, max_inflight=2, hbm_budget_bytes=1024)
    gid = S.add_graph(A)
    tk = S.submit(gb.REQ_SSSP, gid, 0)
    r = S.wait(tk)
    assert r.status == gb.OUT_OF_MEMORY
    with pytest.raises(gb.GBError):
        S.fetch(tk, r.n, gb.REQ_SSSP)
    with pytest.raises(gb.GBError) as e:
        S.submit(gb.REQ_BFS, gid + 5, 0)
    assert e.value.code == gb.INVALID_INDEX
    with pytest.raises(gb.GBError) as e:
        S.submit(gb.REQ_BFS, gid, t.n)
    assert e.value.code == gb.INVALID_INDEX
    with pytest.raises(gb.GBError) as e:
        S.wait(987654321, 10)
    assert e.value.code == gb.INVALID_INDEX
    S.destroy()
    # a budget that fits one job at a time still completes everything
    S = gb.Server(ctx, max_inflight=4, hbm_budget_bytes=4 * (t.n * 68 + (1 << 20)) // 3)
    gid = S.add_graph(A)
    tks = [S.submit(gb.REQ_SSSP, gid, int(s)) for s in gen.sources(t, 12, seed=1)]
    g = oracle.csr_from_tuples(t)
    for tk, s in zip(tks, gen.sources(t, 12, seed=1)):
        r = S.wait(tk)
        assert r.status == gb.SUCCESS
        assert np.array_equal(S.fetch(tk, r.n, gb.REQ_SSSP), oracle.sssp(g, int(s)))
    assert S.stats()["hbm_peak"] <= 4 * (t.n * 68 + (1 << 20)) // 3
    S.destroy()
    # structural graph: SSSP is refused at submit time
    B = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    S = gb.Server(ctx, max_inflight=1)
    gid = S.add_graph(B)
    with pytest.raises(gb.GBError) as e:
        S.submit(gb.REQ_SSSP, gid, 0)
    assert e.value.code == gb.DOMAIN_MISMATCH
    S.destroy()
    A.free()
    B.free()
