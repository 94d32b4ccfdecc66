"""GPU parity of the block polynomial application (mlt_poly_apply, Clenshaw's
recurrence) and of Hutch++ (mlt_hutchpp_estimate, the variance reduction
Section 5.3 proposes for the Estrada index) against the oracle on the same
inputs and probes.

Tolerances: Y = p(At) X is a sum of n + 1 c-weighted Chebyshev terms of
vectors bounded by max|X|, so |Y_gpu - Y_oracle| <= 1e-10 * sum|c| * max|X|
(FP64 rounding is about n * 2^-52 of that).  A quadratic form v^T p(At) v of a
unit or remainder vector v is bounded by sum|c| * |v|^2, giving the tolerance
1e-10 * sum|c| * |v|^2 for the sketch trace and the remainder samples."""
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


def _gershgorin(m, scale=1.0):
    v = np.ones(m.nnz) if m.val is None else np.abs(np.asarray(m.val, dtype=np.float64))
    rows = np.repeat(np.arange(m.nrows), np.diff(m.rowptr))
    r = np.bincount(rows, weights=v, minlength=m.nrows)
    return scale * float(r.max())


def _cases():
    g = synth.rmat_adjacency(12, 16, seed=3)            # hub rows longer than a step's segment
    rg = _gershgorin(g, 0.02)
    lap = synth.grid_laplacian_2d(20, shift=0.1)
    return [("laplacian-log", lap, "log", 0.1, 8.1, 64, 5, False, 1.0),
            ("rmat-exp", g, "exp", -rg, rg, 40, 16, False, 0.02),
            ("rmat-cube", g, "cube", -rg, rg, 3, 3, False, 0.02)]


@pytest.mark.parametrize("case", range(3))
def test_poly_apply_matches_oracle(L, O, case):
    name, m, fn, a, b, n, ncols, gram, scale = _cases()[case]
    c = O.cheb_coeffs(fn, a, b, n)
    X = np.random.default_rng(case).standard_normal((m.nrows, ncols))
    want = O.poly_apply(m, a, b, c, X, scale=scale)
    with L.Matrix(m, scale=scale) as M:
        got = L.mlt_poly_apply(M.handle, a, b, c, np.ascontiguousarray(X))
    assert np.max(np.abs(got - want)) <= 1e-10 * np.sum(np.abs(c)) * np.max(np.abs(X)), name


def test_poly_apply_gram_device_tensors(L, O):
    import torch
    X = synth.sparse_gaussian(300, 120, 0.05, seed=4)
    D = 0.5 * X.to_dense()
    b = float(np.linalg.eigvalsh(D.T @ D)[-1]) * 1.01
    c = O.cheb_coeffs("sqrt", 0.0, b, 48)
    V = np.random.default_rng(7).standard_normal((120, 9))
    want = O.poly_apply(X, 0.0, b, c, V, gram=True, scale=0.5)
    with L.Matrix(X, gram=True, scale=0.5) as M:
        Vt = torch.from_numpy(V).cuda()
        got = L.mlt_poly_apply(M.handle, 0.0, b, c, Vt).cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-10 * np.sum(np.abs(c)) * np.max(np.abs(V))


def _hutchpp_pair(L, O, m, a, b, c, seed, off, s, g, gram=False, scale=1.0):
    ref = O.hutchpp(m, a, b, c, seed, off, s, g, gram=gram, scale=scale)
    samples = np.zeros(g)
    with L.Matrix(m, gram=gram, scale=scale) as M:
        r = L.mlt_hutchpp_estimate(M.handle, a, b, c, seed, off, s, g, samples=samples)
    return ref, r, samples


def test_hutchpp_matches_oracle_laplacian(L, O):
    m = synth.grid_laplacian_2d(16, shift=0.1)
    c = O.cheb_coeffs("log", 0.1, 8.1, 32)
    ref, r, samples = _hutchpp_pair(L, O, m, 0.1, 8.1, c, seed=5, off=100, s=8, g=16)
    sc = np.sum(np.abs(c))
    assert r.rank == ref["rank"] == 8
    assert abs(r.t_sketch - ref["t_sketch"]) <= 1e-10 * sc * 8
    assert np.max(np.abs(samples - ref["samples"])) <= 1e-10 * sc * m.nrows
    assert abs(r.estimate - ref["estimate"]) <= 1e-10 * sc * m.nrows
    assert abs(r.std_error - ref["stderr"]) <= 1e-6 * ref["stderr"]
    assert r.matvecs == 8 * 32 + 24 * 16


def test_hutchpp_matches_oracle_graph_and_gram(L, O):
    g = synth.random_graph(300, 0.03, seed=6)
    rg = _gershgorin(g, 0.25)
    c = O.cheb_coeffs("exp", -rg, rg, 24)
    ref, r, samples = _hutchpp_pair(L, O, g, -rg, rg, c, seed=2, off=0, s=5, g=7, scale=0.25)
    sc = np.sum(np.abs(c))
    assert r.rank == ref["rank"] == 5
    assert abs(r.t_sketch - ref["t_sketch"]) <= 1e-10 * sc * 5
    assert np.max(np.abs(samples - ref["samples"])) <= 1e-10 * sc * g.nrows
    X = synth.sparse_gaussian(200, 80, 0.08, seed=8)
    D = X.to_dense()
    bb = float(np.linalg.eigvalsh(D.T @ D)[-1]) * 1.01
    c2 = O.cheb_coeffs("sqrt", 0.0, bb, 20)
    ref, r, samples = _hutchpp_pair(L, O, X, 0.0, bb, c2, seed=9, off=7, s=6, g=5, gram=True)
    sc = np.sum(np.abs(c2))
    assert r.rank == ref["rank"] == 6
    assert abs(r.t_sketch - ref["t_sketch"]) <= 1e-10 * sc * 6
    assert np.max(np.abs(samples - ref["samples"])) <= 1e-10 * sc * X.ncols


def test_hutchpp_full_and_oversized_sketch_is_exact(L, O):
    # s >= d: Q spans everything (dependent columns dropped), the estimate is
    # tr p(At) and the remainder vanishes
    d = 40
    g = synth.random_graph(d, 0.2, seed=12)
    A = g.to_dense()
    lam = np.linalg.eigvalsh(A)
    a, b = lam[0] - 0.3, lam[-1] + 0.3
    c = O.cheb_coeffs("exp", a, b, 30)
    t = (2 * lam - (a + b)) / (b - a)
    exact = math.fsum(O.cheb_eval(c, t).tolist())
    for s in (d, 48):
        samples = np.zeros(3)
        with L.Matrix(g) as M:
            r = L.mlt_hutchpp_estimate(M.handle, a, b, c, 1, 0, s, 3, samples=samples)
        assert r.rank == d
        assert abs(r.estimate - exact) <= 1e-9 * abs(exact)
        assert np.max(np.abs(samples)) <= 1e-9 * abs(exact)


def test_hutchpp_sketch_only_and_remainder_only(L, O):
    m = synth.grid_laplacian_2d(12, shift=0.1)
    c = O.cheb_coeffs("log", 0.1, 8.1, 16)
    with L.Matrix(m) as M:
        r0 = L.mlt_hutchpp_estimate(M.handle, 0.1, 8.1, c, 3, 0, 0, 6)      # plain Hutchinson
        r1 = L.mlt_hutchpp_estimate(M.handle, 0.1, 8.1, c, 3, 0, 4, 0)      # sketch term alone
    mu = O.moments(m, 0.1, 8.1, 3, 0, [16] * 6)
    assert abs(r0.estimate - float(np.mean(mu @ c))) <= 1e-10 * np.sum(np.abs(c)) * m.nrows
    assert r0.rank == 0 and r1.rank == 4 and math.isnan(r1.std_error)
    ref = O.hutchpp(m, 0.1, 8.1, c, 3, 0, 4, 0)
    assert abs(r1.estimate - ref["t_sketch"]) <= 1e-10 * np.sum(np.abs(c)) * 4


def test_hutchpp_rejects_bad_arguments(L, O):
    m = synth.grid_laplacian_2d(6, shift=0.1)
    c = O.cheb_coeffs("log", 0.1, 8.1, 8)
    with L.Matrix(m) as M:
        for args in ((0.1, 8.1, c, 0, 0, 129, 4), (0.1, 8.1, c, 0, 0, 4, 1025), (0.1, 8.1, c, 0, 0, 0, 0),
                     (8.1, 0.1, c, 0, 0, 4, 4), (0.1, 8.1, c, 0, (1 << 32) - 3, 2, 2)):
            with pytest.raises(L.MLTError):
                L.mlt_hutchpp_estimate(M.handle, *args)
        with pytest.raises(L.MLTError):
            L.mlt_poly_apply(M.handle, 0.1, 8.1, c[:1], np.ones((m.nrows, 2)))


def test_hutchpp_fp32_sketch(L, O):
    # the sketch in FP32 only moves span(Q): a full sketch is still exact, and on
    # a well-conditioned problem every part stays within FP32 rounding of the
    # all-FP64 oracle (sketch error ~1e-7 relative moves span(Q) by as much)
    d = 40
    g = synth.random_graph(d, 0.2, seed=12)
    lam = np.linalg.eigvalsh(g.to_dense())
    a, b = lam[0] - 0.3, lam[-1] + 0.3
    c = O.cheb_coeffs("exp", a, b, 30)
    exact = math.fsum(O.cheb_eval(c, (2 * lam - (a + b)) / (b - a)).tolist())
    with L.Matrix(g) as M:
        r = L.mlt_hutchpp_estimate(M.handle, a, b, c, 1, 0, d, 3, precision="fp32")
    assert r.rank == d and abs(r.estimate - exact) <= 1e-9 * abs(exact)
    m = synth.grid_laplacian_2d(16, shift=0.1)
    c = O.cheb_coeffs("log", 0.1, 8.1, 32)
    ref = O.hutchpp(m, 0.1, 8.1, c, 5, 100, 8, 16)
    samples = np.zeros(16)
    with L.Matrix(m) as M:
        r = L.mlt_hutchpp_estimate(M.handle, 0.1, 8.1, c, 5, 100, 8, 16, precision="fp32", samples=samples)
        with pytest.raises(L.MLTError):
            L.mlt_hutchpp_estimate(M.handle, 0.1, 8.1, c, 5, 100, 8, 16, precision=2)
    sc = np.sum(np.abs(c))
    assert r.rank == 8
    assert abs(r.t_sketch - ref["t_sketch"]) <= 1e-5 * sc * 8
    assert np.max(np.abs(samples - ref["samples"])) <= 1e-5 * sc * m.nrows


def test_hutchpp_df64_moments(L, O):
    # double-float moments keep the FP64 tolerances of the remainder samples and
    # the sketch trace (the FP32 sketch only moves span(Q): a full sketch is exact)
    d = 40
    g = synth.random_graph(d, 0.2, seed=12)
    lam = np.linalg.eigvalsh(g.to_dense())
    a, b = lam[0] - 0.3, lam[-1] + 0.3
    c = O.cheb_coeffs("exp", a, b, 30)
    exact = math.fsum(O.cheb_eval(c, (2 * lam - (a + b)) / (b - a)).tolist())
    with L.Matrix(g) as M:
        r = L.mlt_hutchpp_estimate(M.handle, a, b, c, 1, 0, d, 3, precision="df64")
    assert r.rank == d and abs(r.estimate - exact) <= 1e-9 * abs(exact)
    m = synth.grid_laplacian_2d(12, shift=0.1)
    c = O.cheb_coeffs("log", 0.1, 8.1, 16)
    with L.Matrix(m) as M:
        r0 = L.mlt_hutchpp_estimate(M.handle, 0.1, 8.1, c, 3, 0, 0, 6, precision="df64")   # remainder only
    mu = O.moments(m, 0.1, 8.1, 3, 0, [16] * 6)
    assert abs(r0.estimate - float(np.mean(mu @ c))) <= 1e-10 * np.sum(np.abs(c)) * m.nrows


def test_hutchpp_multi_tile_gram_schmidt(L, O):
    """A sketch wider than one 64-column tile (s = 100) takes the Gram-Schmidt
    path without Cholesky QR, over two Q tiles, and the 130 remainder probes
    span three G tiles in the block deflation; all against the oracle."""
    m = synth.grid_laplacian_2d(30, shift=0.1)
    c = O.cheb_coeffs("log", 0.1, 8.1, 24)
    ref, r, samples = _hutchpp_pair(L, O, m, 0.1, 8.1, c, seed=4, off=50, s=100, g=130)
    sc = np.sum(np.abs(c))
    assert r.rank == ref["rank"] == 100
    assert abs(r.t_sketch - ref["t_sketch"]) <= 1e-10 * sc * 100
    assert np.max(np.abs(samples - ref["samples"])) <= 1e-10 * sc * m.nrows
    assert abs(r.estimate - ref["estimate"]) <= 1e-10 * sc * m.nrows
    assert abs(r.std_error - ref["stderr"]) <= 1e-6 * ref["stderr"]
    assert r.matvecs == 100 * 24 + 230 * 12
