"""gb_bfs_noalloc, the BFS entry point that allocates no device memory. It
is for callers that cannot allocate device memory when they run a query:
their memory belongs to another allocator (a framework's caching allocator
or a fixed arena), or cudaFree's device-wide synchronisation would stall a
latency-critical loop, or the deployment forbids allocation after start-up.

Each case enqueues two calls back to back on one stream (they share the
library's built-in scratch) before a single synchronise, and checks both
results against the oracle's queue BFS and against gb_bfs, the entry point
that allocates. The failure path is driven without a GPU fault: a test hook
makes one block withhold its barrier arrival, the bounded wait of the others
runs out, and the caller's status word must say GB_TIMEOUT. This file is
collected last on purpose."""
import os

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1908_01407_gb300 as gb

pytestmark = pytest.mark.gpu


def padded_device(a: np.ndarray) -> torch.Tensor:
    # 16 readable bytes past the end, as the entry point requires
    p = np.zeros(a.shape[0] + 4, dtype=np.uint32)
    p[: a.shape[0]] = a
    return torch.from_numpy(p.view(np.int32)).cuda()


def directed_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, m).astype(np.uint32), rng.integers(0, n, m).astype(np.uint32)


def make_case(ctx, case):
    """(gbx matrix, oracle graph, device CSR, device CSC or None, sources)"""
    if case == "directed":
        n = 3001                                   # not a multiple of 32: a ragged last bitmap word
        r, c = directed_graph(n, 24000, seed=31)
        A = gb.Matrix.from_tuples(ctx, n, r, c)
        g = oracle.csr_build(n, r, c)
        srcs = [7, 2999]
    else:
        scale = {"symmetric": 14, "push_only": 12, "no_parents": 14, "max_n": 18}[case]
        t = gen.rmat(scale, 16, seed=1)
        A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
        g = oracle.csr_from_tuples(t)
        srcs = [int(s) for s in gen.sources(t, 2, seed=1)]
    rp, ci = A.export_csr()
    csr = (torch.from_numpy(rp.view(np.int32)).cuda(), padded_device(ci))
    if case == "push_only":
        csc = None
    elif case == "directed":
        cp, ri = A.export_csc()
        csc = (torch.from_numpy(cp.view(np.int32)).cuda(), padded_device(ri))
    else:
        csc = csr                                  # symmetric: the CSR serves as the CSC
    return A, g, csr, csc, srcs


@pytest.mark.parametrize("case", ["symmetric", "directed", "push_only", "no_parents", "max_n"])
def test_noalloc_two_calls_on_one_stream_match_the_oracle(ctx, case):
    A, g, csr, csc, srcs = make_case(ctx, case)
    n, nnz = A.nrows, A.nvals
    if case == "max_n":
        assert n == gb.NOALLOC_MAX_VERTICES
    assert csr[1].data_ptr() % 16 == 0
    with_parents = case != "no_parents"
    outs = []
    stream = torch.cuda.current_stream()
    for s in srcs:                                 # both enqueued before one synchronise
        lv = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        pa = torch.full((n,), 7, dtype=torch.int32, device="cuda") if with_parents else None
        status = torch.full((1,), -5, dtype=torch.int32, device="cuda")
        gb.bfs_noalloc(csr[0], csr[1], csc[0] if csc else None, csc[1] if csc else None, n, nnz, s, lv, pa,
                       status=status, stream=stream)
        outs.append((s, lv, pa, status))
    torch.cuda.synchronize()
    for s, lv, pa, status in outs:
        assert int(status.item()) == 0
        lv = lv.cpu().numpy()
        want = oracle.bfs(g, s)
        assert np.array_equal(lv, want)
        ref_lv, _, _ = gb.bfs(ctx, A, s, parents=False)      # the allocating entry point agrees
        assert np.array_equal(lv, ref_lv.cpu().numpy())
        if with_parents:
            # parents are not unique: each must be a valid BFS parent
            assert oracle.bfs_parent_violations(g, s, lv, pa.cpu().numpy()) == 0
    A.free()


def test_noalloc_reports_a_timeout_to_the_caller(ctx):
    t = gen.rmat(12, 16, seed=1)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    g = oracle.csr_from_tuples(t)
    rp, ci = A.export_csr()
    rp_d, ci_d = torch.from_numpy(rp.view(np.int32)).cuda(), padded_device(ci)
    n, nnz = A.nrows, A.nvals
    s = int(gen.sources(t, 1, seed=1)[0])
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    os.environ["GBX_TEST_WITHHOLD_BARRIER_US"] = "2000"
    try:
        gb.bfs_noalloc(rp_d, ci_d, rp_d, ci_d, n, nnz, s, lv, status=status)
        torch.cuda.synchronize()
    finally:
        del os.environ["GBX_TEST_WITHHOLD_BARRIER_US"]
    assert int(status.item()) == gb.TIMEOUT
    # the next call on the same scratch runs normally and says so
    gb.bfs_noalloc(rp_d, ci_d, rp_d, ci_d, n, nnz, s, lv, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(lv.cpu().numpy(), oracle.bfs(g, s))
    A.free()


def test_noalloc_bfs_rejects_graphs_above_its_limit(ctx):
    n = gb.NOALLOC_MAX_VERTICES + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(4, dtype=torch.int32, device="cuda")
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.GBError) as e:
        gb.bfs_noalloc(rp, ci, rp, ci, n, 0, 0, lv)
    assert e.value.code == gb.INVALID_VALUE
    assert "scratch" in str(e.value)
