"""The allocation-free moment entry point, for callers that cannot call
cudaMalloc (inside a stream capture they do not own, in loops that cannot take
the synchronisation an allocation may cause, or under a host memory pool that
owns the device memory).  Its output must equal the regular mlt_moments path's
within the FP64 moment tolerance (1e-10 d), on two calls in a row that share
the library's fixed scratch array, and inside a CUDA graph capture; and it must
equal the CPU oracle's moments on the same probes within the same tolerance.
The spectrum interval comes from the host (the oracle's Gershgorin bound), so no
library call chooses the interval both sides use.  This file is collected last
on purpose."""
import numpy as np
import pytest

from paper_2103_10516_gb300 import synth

pytestmark = pytest.mark.gpu
TOL64 = 1e-10


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    from paper_2103_10516_gb300 import build, mlt
    build.build()
    return mlt


def _dev(m):
    import torch
    rp = torch.from_numpy(m.rowptr).cuda()
    col = torch.from_numpy(m.col).cuda()
    val = None if m.val is None else torch.from_numpy(m.val).cuda()
    return rp, col, val


def test_noalloc_matches_regular_path_twice(L, O):
    import torch
    calls = [
        (synth.grid_laplacian_2d(32, shift=0.1), 1.0, (0.1, 8.1), 3, 0,
         np.array([8] * 40 + [32] * 20 + [64] * 5, dtype=np.int32)),
        (synth.rmat_adjacency(10, 8, seed=5), 0.05, None, 11, 1000,
         (np.arange(100) % 37).astype(np.int32)),
    ]
    for m, scale, ab, seed, off, deg in calls:
        a, b = ab if ab else O.interval(m, scale)
        with L.Matrix(m, scale=scale) as M:
            ref = M.moments(a, b, seed, off, deg)
        orc = O.moments(m, a, b, seed, off, deg, scale=scale)
        rp, col, val = _dev(m)
        mu = torch.full((deg.size, ref.shape[1] + 3), 5.0, dtype=torch.float64, device="cuda")
        L.mlt_moments_noalloc(m.nrows, m.nnz, rp, col, val, scale, a, b, seed, off, deg, mu)
        got = mu.cpu().numpy()
        assert np.max(np.abs(got[:, :ref.shape[1]] - ref)) <= TOL64 * m.nrows
        assert np.max(np.abs(got[:, :ref.shape[1]] - orc)) <= TOL64 * m.nrows
        assert np.all(got[:, ref.shape[1]:] == 0.0)


def test_noalloc_rejects_oversize_and_bad_input(L):
    import torch
    big = synth.grid_laplacian_2d(200, shift=0.1)          # 40,000 rows
    rp, col, val = _dev(big)
    mu = torch.zeros((512, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(L.MLTError) as e:                    # 2 * 40,000 * 512 doubles > 32 MiB
        L.mlt_moments_noalloc(big.nrows, big.nnz, rp, col, val, 1.0, 0.1, 8.1, 0, 0, [8] * 512, mu)
    assert e.value.code == L.MLT_ERANGE
    small = synth.grid_laplacian_2d(4, shift=0.1)
    rp, col, val = _dev(small)
    col[3] = 99
    with pytest.raises(L.MLTError) as e:
        L.mlt_moments_noalloc(small.nrows, small.nnz, rp, col, val, 1.0, 0.1, 8.1, 0, 0, [4], mu[:1])
    assert e.value.code == L.MLT_EINVAL


def test_noalloc_inside_graph_capture(L, O):
    """A call captured into a CUDA graph (after one uncaptured call has looked
    up the scratch array) replays to the same moments, twice; captured with a
    column out of range it yields NaN rows instead of an error code."""
    import torch
    m = synth.grid_laplacian_2d(24, shift=0.1)
    deg = np.array([16] * 30 + [40] * 10, dtype=np.int32)
    with L.Matrix(m) as M:
        ref = M.moments(0.1, 8.1, 7, 50, deg)
    orc = O.moments(m, 0.1, 8.1, 7, 50, deg)
    rp, col, val = _dev(m)
    warm = torch.zeros((deg.size, ref.shape[1]), dtype=torch.float64, device="cuda")
    L.mlt_moments_noalloc(m.nrows, m.nnz, rp, col, val, 1.0, 0.1, 8.1, 7, 50, deg, warm)
    mu = torch.full((deg.size, ref.shape[1]), 5.0, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        L.mlt_moments_noalloc(m.nrows, m.nnz, rp, col, val, 1.0, 0.1, 8.1, 7, 50, deg, mu,
                              stream=torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        mu.fill_(5.0)
        g.replay()
        torch.cuda.synchronize()
        assert np.max(np.abs(mu.cpu().numpy() - ref)) <= TOL64 * m.nrows
        assert np.max(np.abs(mu.cpu().numpy() - orc)) <= TOL64 * m.nrows
    bad_col = col.clone()
    bad_col[5] = m.nrows + 3
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=side):
        L.mlt_moments_noalloc(m.nrows, m.nnz, rp, bad_col, val, 1.0, 0.1, 8.1, 7, 50, deg, mu,
                              stream=torch.cuda.current_stream().cuda_stream)
    g2.replay()
    torch.cuda.synchronize()
    assert torch.isnan(mu).all()
