"""GPU parity of the exact triangle path (mlt_triangle_trace): per-probe int64
moments bit-exact against the oracle, and the control-variate estimate equal to
the oracle's to the last bit (same integer sums, same double-precision steps)."""
import math

import numpy as np
import pytest

from paper_2103_10516_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    from paper_2103_10516_gb300 import build, mlt
    build.build()
    return mlt


@pytest.mark.parametrize("d,p,nprobes", [(500, 0.03, 300), (64, 0.5, 1), (2000, 0.004, 129)])
def test_random_graph_bit_exact(L, O, d, p, nprobes):
    g = synth.random_graph(d, p, seed=d)
    x = np.zeros((nprobes, 3), dtype=np.int64)
    with L.Matrix(g) as G:
        est, se = G.triangles(5, 17, nprobes, use_cv=True, x=x)
        est0, se0 = G.triangles(5, 17, nprobes, use_cv=False)
    xr = O.triangle_moments(g, 5, 17, nprobes)
    assert np.array_equal(x, xr)
    er, sr, _, _ = O.triangle_estimate(xr, g.nnz, True)
    assert est == er and (se == sr or (math.isnan(se) and math.isnan(sr)))
    er0, sr0, _, _ = O.triangle_estimate(xr, g.nnz, False)
    assert est0 == er0 and (se0 == sr0 or (math.isnan(se0) and math.isnan(sr0)))


def test_rmat_scale14_and_truth(L, O):
    g = synth.rmat_adjacency(14, 16, seed=0)
    x = np.zeros((512, 3), dtype=np.int64)
    with L.Matrix(g) as G:
        est, se = G.triangles(0, 0, 512, x=x)
    assert np.array_equal(x, O.triangle_moments(g, 0, 0, 512))
    T = O.triangle_count(g)
    assert abs(est - T) < 5 * se


def test_exhaustive_signs_give_exact_count(L, O):
    """Every sign vector of a 10-vertex graph, taken from the GPU's own probes:
    16,384 probe ids cover all 2^10 sign patterns (checked); averaging the GPU's
    moments over one probe per pattern averages over the whole sign space, so
    mean x3 = 6T, mean x2 = nnz and mean x1 = 0 hold exactly, in integers."""
    g = synth.random_graph(10, 0.5, seed=11)
    n = 16384
    x = np.zeros((n, 3), dtype=np.int64)
    with L.Matrix(g) as G:
        G.triangles(3, 0, n, x=x)
    first = {}
    for p in range(n):
        key = tuple(O.rademacher(3, p, 10).astype(int))
        first.setdefault(key, p)
    assert len(first) == 1 << 10
    rows = x[sorted(first.values())]
    assert np.array_equal(rows, O.triangle_moments(g, 3, 0, n)[sorted(first.values())])
    T = O.triangle_count(g)
    assert int(rows[:, 2].sum()) == 6 * T * (1 << 10)
    assert int(rows[:, 1].sum()) == g.nnz * (1 << 10)
    assert int(rows[:, 0].sum()) == 0


@pytest.mark.parametrize("cv", ["none", "fit", "cheb"])
def test_estimates_from_gpu_moments_bit_exact(L, O, cv):
    """The library's estimate from the GPU's integers, for every control-variate
    form of Section 5.4 (none, fitted, a priori from the Chebyshev expansion of
    x^3 on [-max degree, max degree]), equals the oracle's from its own
    integers to the last bit."""
    g = synth.rmat_adjacency(13, 16, seed=2)
    x = np.zeros((700, 3), dtype=np.int64)
    with L.Matrix(g) as G:
        L.mlt_triangle_trace(G.handle, 8, 123, 700, x=x)
    xr = O.triangle_moments(g, 8, 123, 700)
    assert np.array_equal(x, xr)
    dmax = float(np.max(np.diff(g.rowptr)))
    est, se, a1, a2 = L.mlt_triangle_estimate(x, g.nnz, cv, -dmax, dmax)
    if cv == "cheb":
        ra1, ra2 = O.triangle_cv_cheb(-dmax, dmax)
        er, sr = O.triangle_estimate_fixed(xr, g.nnz, ra1, ra2)
        assert (a1, a2) == (ra1, ra2)
    else:
        er, sr, _, _ = O.triangle_estimate(xr, g.nnz, cv == "fit")
    assert est == er and se == sr


def test_device_output(L, O):
    import torch
    g = synth.random_graph(300, 0.05, seed=2)
    xd = torch.zeros((200, 3), dtype=torch.int64, device="cuda")
    with L.Matrix(g) as G:
        est, _ = G.triangles(1, 0, 200, x=xd)
    assert np.array_equal(xd.cpu().numpy(), O.triangle_moments(g, 1, 0, 200))


def test_rejects_bad_inputs(L):
    with L.Matrix(synth.grid_laplacian_2d(5)) as M:      # has values
        with pytest.raises(L.MLTError) as e:
            M.triangles(0, 0, 10)
        assert e.value.code == L.MLT_EINVAL
    loop = synth.CSR(3, 3, np.array([0, 2, 3, 4]), np.array([0, 1, 0, 2]))
    with L.Matrix(loop) as M:
        with pytest.raises(L.MLTError) as e:
            M.triangles(0, 0, 10)
        assert e.value.code == L.MLT_EINVAL
    g = synth.random_graph(20, 0.3, seed=0)
    with L.Matrix(g) as M:
        for blk in (64, 192, 512):
            with pytest.raises(L.MLTError):
                L.mlt_triangle_trace(M.handle, 0, 0, 10, block=blk)
        with pytest.raises(L.MLTError):
            M.triangles(0, 0, 0)


def test_block_128_bit_exact(L, O):
    """Blocks of 128 probes, as Section 5.4's triangle workload states them,
    give the oracle's integers and the oracle's estimate bit for bit, and the
    same results as blocks of 256, over a ragged probe count."""
    g = synth.rmat_adjacency(12, 16, seed=4)
    x128 = np.zeros((300, 3), dtype=np.int64)
    x256 = np.zeros((300, 3), dtype=np.int64)
    with L.Matrix(g) as G:
        e128, s128 = L.mlt_triangle_trace(G.handle, 5, 77, 300, block=128, use_cv=True, x=x128)
        e256, s256 = L.mlt_triangle_trace(G.handle, 5, 77, 300, block=256, use_cv=True, x=x256)
    xr = O.triangle_moments(g, 5, 77, 300)
    assert np.array_equal(x128, xr) and np.array_equal(x256, xr)
    er, sr, _, _ = O.triangle_estimate(xr, g.nnz, True)
    assert e128 == er and s128 == sr and e256 == er and s256 == sr


def test_full_size_rmat20_sampled(L, O):
    # the R-MAT scale-20 triangle workload at full size: 1024 probes in blocks
    # of 256; a sample of probes (first, half and block edges, last) against the
    # oracle
    g = synth.rmat_adjacency(20, 16, seed=0)
    x = np.zeros((1024, 3), dtype=np.int64)
    with L.Matrix(g) as G:
        est, se = G.triangles(0, 0, 1024, x=x)
    for p in (0, 3, 127, 128, 131, 255, 256, 1023):
        assert np.array_equal(x[p], O.triangle_moments(g, 0, p, 1)[0]), p
    er, sr, _, _ = O.triangle_estimate(x, g.nnz, True)   # same sums -> same bits
    assert est == er and se == sr
    assert np.all(x[:, 1] > 0)


@pytest.mark.parametrize("make", [lambda: synth.complete_graph(1500),
                                  lambda: synth.rmat_adjacency(16, 16, seed=3)])
def test_long_rows_split_across_chunks(L, O, make):
    # rows longer than a work chunk are cut and their counts merged atomically
    g = make()
    x = np.zeros((130, 3), dtype=np.int64)
    with L.Matrix(g) as G:
        est, se = G.triangles(9, 1000, 130, x=x)
    assert np.array_equal(x, O.triangle_moments(g, 9, 1000, 130))
    er, sr, _, _ = O.triangle_estimate(x, g.nnz, True)
    assert est == er and se == sr


def test_empty_and_tiny_graphs(L, O):
    empty = synth.CSR(3, 3, np.array([0, 0, 0, 0]), np.array([], dtype=np.int32))
    x = np.ones((5, 3), dtype=np.int64)
    with L.Matrix(empty) as G:
        est, se = G.triangles(0, 0, 5, x=x)
    assert np.all(x == 0) and est == 0.0
    tri = synth.complete_graph(3)
    x = np.zeros((200, 3), dtype=np.int64)
    with L.Matrix(tri) as G:
        est, se = G.triangles(2, 64, 200, x=x)
    assert np.array_equal(x, O.triangle_moments(tri, 2, 64, 200))


def _undirected(d, u, v):
    """Symmetric 0/1 CSR from undirected edges (u, v), duplicates and loops dropped."""
    u, v = np.asarray(u, dtype=np.int64), np.asarray(v, dtype=np.int64)
    keep = u != v
    a, b = np.minimum(u, v)[keep], np.maximum(u, v)[keep]
    key = np.unique(a * d + b)
    a, b = key // d, key % d
    return synth._from_coo(d, d, np.concatenate([a, b]), np.concatenate([b, a]), None)


def test_degree_classes_and_huge_rows(L, O):
    # every storage class of y in one graph: two adjacent hubs of degree
    # > 32767 (int32 rows, edges into them on the pair list, one hub-to-hub
    # pair), a 300-clique (int16 rows) and sparse leaves (int8 rows)
    rng = np.random.default_rng(7)
    d = 40_002
    h1, h2 = d - 2, d - 1
    l1 = rng.choice(40_000, 34_000, replace=False)
    l2 = rng.choice(40_000, 34_000, replace=False)
    clique = rng.choice(40_000, 300, replace=False)
    cu, cv = np.triu_indices(300, 1)
    su, sv = rng.integers(0, 40_000, 60_000), rng.integers(0, 40_000, 60_000)
    g = _undirected(d, np.concatenate([[h1], np.full(l1.size, h1), np.full(l2.size, h2), clique[cu], su]),
                    np.concatenate([[h2], l1, l2, clique[cv], sv]))
    deg = np.diff(g.rowptr)
    assert deg[h1] > 32767 and deg[h2] > 32767 and deg.max() > 127 and np.sum((deg > 127) & (deg <= 32767)) >= 300
    x = np.zeros((160, 3), dtype=np.int64)
    with L.Matrix(g) as G:
        est, se = G.triangles(4, 250, 160, x=x)
    assert np.array_equal(x, O.triangle_moments(g, 4, 250, 160))
    er, sr, _, _ = O.triangle_estimate(x, g.nnz, True)
    assert est == er and se == sr


def test_pooled_memory_reuse(L, O):
    # handles take their memory from the library's pool: a handle built in the
    # blocks a destroyed handle (another graph, stale contents) left behind
    # gives the same moments, and returning the cache to the driver is clean
    ga = synth.rmat_adjacency(13, 16, seed=4)
    gb = synth.random_graph(3000, 0.004, seed=9)
    xs = []
    for g in (ga, gb, ga):
        x = np.zeros((256, 3), dtype=np.int64)
        with L.Matrix(g) as G:
            G.triangles(2, 7, 256, x=x)
        xs.append(x)
    assert np.array_equal(xs[0], xs[2])
    assert np.array_equal(xs[0], O.triangle_moments(ga, 2, 7, 256))
    assert np.array_equal(xs[1], O.triangle_moments(gb, 2, 7, 256))
    L.mlt_release_cached()
    x = np.zeros((256, 3), dtype=np.int64)
    with L.Matrix(gb) as G:
        G.triangles(2, 7, 256, x=x)
    assert np.array_equal(x, xs[1])
