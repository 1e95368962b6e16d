"""gb_bfs_noalloc, the BFS entry point that allocates no device memory
(for callers that cannot allocate on the call path), against gb_bfs: the
same levels and valid parents, on two calls in a row that share the
built-in scratch. This file is collected last on purpose."""
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


def test_noalloc_bfs_matches_gb_bfs_on_two_calls(ctx):
    t = gen.rmat(14, 16, seed=1)
    g = oracle.csr_from_tuples(t)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    rp, ci = A.export_csr()
    rp_d = torch.from_numpy(rp.view(np.int32)).cuda()
    ci_d = padded_device(ci)
    assert ci_d.data_ptr() % 16 == 0
    n, nnz = A.nrows, A.nvals
    srcs = [int(s) for s in gen.sources(t, 2, seed=1)]
    for s in srcs:                      # two calls in a row on the shared scratch
        lv = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        pa = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        gb.bfs_noalloc(rp_d, ci_d, rp_d, ci_d, n, nnz, s, lv, pa)
        torch.cuda.synchronize()
        ref_lv, ref_pa, _ = gb.bfs(ctx, A, s)
        torch.cuda.synchronize()
        lv, pa = lv.cpu().numpy(), pa.cpu().numpy()
        assert np.array_equal(lv, ref_lv.cpu().numpy())
        # parents are not unique: both must be valid BFS parents
        assert oracle.bfs_parent_violations(g, s, lv, pa) == 0
        assert oracle.bfs_parent_violations(g, s, ref_lv.cpu().numpy(), ref_pa.cpu().numpy()) == 0
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
