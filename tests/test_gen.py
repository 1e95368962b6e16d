"""The seeded input generators: determinism and the structural properties
the paper's datasets have (undirected, no self-loops; Table 11 caption)."""
import numpy as np

import gen


def test_rmat_deterministic_symmetric_no_self_loops():
    a = gen.rmat(12, 16, seed=1, wmax=255)
    b = gen.rmat(12, 16, seed=1, wmax=255)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst) and np.array_equal(a.w, b.w)
    c = gen.rmat(12, 16, seed=2)
    assert not np.array_equal(a.src, c.src)
    assert np.all(a.src != a.dst)
    assert a.ntuples % 2 == 0 and a.ntuples <= 2 * 16 * 4096
    # both directions with equal weights
    assert np.array_equal(a.src[0::2], a.dst[1::2]) and np.array_equal(a.w[0::2], a.w[1::2])
    assert a.w.min() >= 1 and a.w.max() <= 255
    key = a.src.astype(np.uint64) << np.uint64(32) | a.dst
    rkey = a.dst.astype(np.uint64) << np.uint64(32) | a.src
    assert np.array_equal(np.sort(key), np.sort(rkey))


def test_rmat_is_skewed():
    t = gen.rmat(14, 16, seed=1)
    deg = np.bincount(t.src, minlength=t.n)
    # scale-free: a few hubs, many low-degree and isolated vertices
    assert deg.max() > 50 * deg.mean()
    assert (deg == 0).sum() > 0.1 * t.n


def test_grid_counts_and_structure():
    t = gen.grid(64, 64, 0.1, seed=3, wmax=1000)
    full = 2 * (64 * 63 * 2)
    assert 0.85 * full < t.ntuples < 0.95 * full
    diff = np.abs(t.src.astype(np.int64) - t.dst.astype(np.int64))
    assert np.all((diff == 1) | (diff == 64))
    assert t.w.min() >= 1 and t.w.max() <= 1000
    t0 = gen.grid(8, 8, 0.0, seed=3)
    assert t0.ntuples == 2 * (8 * 7 * 2)


def test_sources_distinct_nonisolated_and_permutation():
    t = gen.rmat(12, 16, seed=2)
    s = gen.sources(t, 64, seed=1)
    assert s.size == 64 and np.unique(s).size == 64
    has = gen.touched(t)
    assert np.all(has[s] == 1)
    p = gen.permutation(1000, 5)
    assert np.array_equal(np.sort(p), np.arange(1000))
