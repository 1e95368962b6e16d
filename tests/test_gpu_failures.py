"""Failure handling without a GPU fault: bounded device waits end with
GB_TIMEOUT and leave the context usable, allocation failures injected in
the memory pool come back as GB_OUT_OF_MEMORY, and a server wait that
runs out of time returns GB_TIMEOUT while the request still completes."""
import numpy as np
import pytest

import gen
import oracle
import paper_1908_01407_gb300 as gb

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_stays_usable(ctx):
    for limit_us in (1000, 20000):
        assert ctx.selftest_wait(limit_us) == gb.TIMEOUT
    # the persistent kernels' barriers still work afterwards
    t = gen.rmat(10, 8, seed=21)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    lv = np.empty(t.n, np.int32)
    _, _, st = gb.bfs(ctx, A, int(gen.sources(t, 1, seed=1)[0]), lv, False)
    assert st["status"] == 0
    assert np.array_equal(lv, oracle.bfs(oracle.csr_from_tuples(t), int(gen.sources(t, 1, seed=1)[0])))
    A.free()


def test_injected_allocation_failures(ctx):
    t = gen.rmat(10, 8, seed=22)
    ctx.inject_alloc_failures(1)
    with pytest.raises(gb.GBError) as e:
        gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    assert e.value.code == gb.OUT_OF_MEMORY
    # the next build is served normally and is correct
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    assert A.nvals == oracle.csr_from_tuples(t).m
    # a failure inside an algorithm's scratch allocation comes back as a code too
    d = np.empty(t.n, np.int32)
    ctx.inject_alloc_failures(1)
    with pytest.raises(gb.GBError) as e:
        gb.pagerank(ctx, A, 0.85, 5, d.view(np.float32), residuals=False)
    assert e.value.code == gb.OUT_OF_MEMORY
    ctx.inject_alloc_failures(0)
    gb.pagerank(ctx, A, 0.85, 5, d.view(np.float32), residuals=False)
    A.free()


def test_server_wait_times_out_then_completes(ctx):
    t = gen.rmat(16, 16, seed=23)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    S = gb.Server(ctx, max_inflight=1, batch_window_us=0)
    gid = S.add_graph(A)
    # one slot, a queue of PageRank jobs: the last one cannot be done at once
    tickets = [S.submit(gb.REQ_PAGERANK, gid) for _ in range(6)]
    with pytest.raises(gb.GBError) as e:
        S.wait(tickets[-1], 0)
    assert e.value.code == gb.TIMEOUT
    for tk in tickets:
        r = S.wait(tk, 120000)
        assert r.status == gb.SUCCESS
    S.destroy()
    A.free()


def test_bfs_timeout_without_waiting_is_reported_by_synchronize(ctx):
    """gb_bfs with device outputs and no stats returns without waiting; when
    its bounded barrier wait runs out (a test hook makes one block withhold
    its arrival; no fault), the next synchronise reports GB_TIMEOUT once, a
    waiting call reports it at once, and the context stays usable."""
    import os
    import torch
    t = gen.rmat(12, 16, seed=24)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    g = oracle.csr_from_tuples(t)
    s = int(gen.sources(t, 1, seed=1)[0])
    lv = torch.empty(t.n, dtype=torch.int32, device="cuda")
    ctx.synchronize()
    os.environ["GBX_TEST_WITHHOLD_BARRIER_US"] = "2000"
    try:
        gb.bfs(ctx, A, s, lv, False, stats=False)          # does not wait
        with pytest.raises(gb.GBError) as e:
            ctx.synchronize()
        assert e.value.code == gb.TIMEOUT
        ctx.synchronize()                                   # reported once
        with pytest.raises(gb.GBError) as e:                # a waiting call reports it itself
            gb.bfs(ctx, A, s, lv, False, stats=True)
        assert e.value.code == gb.TIMEOUT
        ctx.synchronize()
    finally:
        del os.environ["GBX_TEST_WITHHOLD_BARRIER_US"]
    _, _, st = gb.bfs(ctx, A, s, lv, False, stats=True)
    assert st["status"] == 0
    assert np.array_equal(lv.cpu().numpy(), oracle.bfs(g, s))
    A.free()


def test_barrier_free_traversal_timeout_is_reported_and_the_next_run_is_correct(ctx):
    """The barrier-free schedule bounds its whole traversal (and every wait
    in it); a test hook shrinks that bound to a few microseconds, so the run
    stops with GB_TIMEOUT (no fault, no hang), and the next run on the same
    context, with its own fresh ring and state, gives Dijkstra's distances
    and the union-find labels."""
    import os
    t = gen.grid(400, 400, 0.1, seed=6, wmax=1000)
    g = oracle.csr_from_tuples(t)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
    src = gen.first_nonisolated(t)
    d = gb.Descriptor(schedule=gb.SCHED_ASYNC)
    dist = np.empty(t.n, np.uint32)
    lab = np.empty(t.n, np.uint32)
    os.environ["GBX_TEST_ASYNC_LIMIT_US"] = "5"
    try:
        with pytest.raises(gb.GBError) as e:
            gb.sssp(ctx, A, src, dist, d)
        assert e.value.code == gb.TIMEOUT
        with pytest.raises(gb.GBError) as e:
            gb.cc_async(ctx, A, lab)
        assert e.value.code == gb.TIMEOUT
    finally:
        del os.environ["GBX_TEST_ASYNC_LIMIT_US"]
    gb.sssp(ctx, A, src, dist, d)
    assert np.array_equal(dist, oracle.sssp(g, src))
    gb.cc_async(ctx, A, lab)
    assert np.array_equal(lab, oracle.cc(g))
    d.free()
    A.free()
