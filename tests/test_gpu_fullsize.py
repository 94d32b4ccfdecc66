"""Parity of the moment engine at the full sizes the FP32 benchmarks time, in
the same launch configuration (probe count, degree, precision, autotuned
probe-group width), on sampled outputs the oracle computes one by one, and
on properties that hold for every output.

Tolerance.  FP32 vectors: each of the deg/2 steps rounds V to 2^-24 of its
size and these errors add up along the recurrence; the tests allow
max(64, deg/2) * 2^-24 * d, the bound the smaller FP32 tests use up to degree
128.  Emulating the FP32 recurrence on the CPU gives 0.1 of it on the 3D
stencil and 0.02 on the Gram operator and the scaled R-MAT graph.  Every moment of a spectrum inside
[a, b] also satisfies |mu_j| <= d.

The sampled probes stay at low degree: the oracle sums in long double, which is
quad precision in software on aarch64, about 10^8 multiply-adds a few seconds
there.  The bound above is checked on every moment of every probe."""
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


def _tol32(deg, d):
    return max(64, deg // 2) * 2.0 ** -24 * d


def _check_all(got, degs, d, tol):
    # mu_0 = z.z = d, and |mu_j| <= d for every moment of every probe
    assert np.max(np.abs(got[:, 0] - d)) <= tol
    for p, dg in enumerate(degs):
        assert np.max(np.abs(got[p, :dg + 1])) <= d + tol, p


def _check_sampled(O, m, a, b, seed, offset, got, samples, tol, **kw):
    for p, dg in samples:
        ref = O.moments(m, a, b, seed, offset + p, [dg], **kw)[0]
        err = np.max(np.abs(got[p, :dg + 1] - ref))
        assert err <= tol, (p, dg, err, tol)


def test_stencil3d_fp32_full_size(L, O):
    # the 100^3 diffusion operator, 128 probes to degree 128 in FP32; two probes
    # checked to degree 8 (2 x 8 operator applications of 6.9M entries)
    m = synth.diffusion_3d(100, sigma=1.0, shift=0.1, seed=0)
    a, b = 0.1, O.gershgorin(m)[1]
    deg = np.full(128, 128, dtype=np.int32)
    with L.Matrix(m) as M:
        L.mlt_autotune(M.handle, "fp32", 4)
        got = M.moments(a, b, 0, 4096, deg, precision="fp32")
    tol = _tol32(128, m.nrows)
    _check_all(got, deg, m.nrows, tol)
    _check_sampled(O, m, a, b, 0, 4096, got, [(0, 8), (127, 8)], tol)


def test_nuclear_gram_fp32_full_size(L, O):
    # X^T X with X 2^18 x 2^16 (density 1e-4), 512 probes to degree 512 in FP32;
    # the interval's upper end is ||X||_1 ||X||_inf >= ||X||_2^2; one probe of the
    # last group checked to degree 32
    X = synth.sparse_gaussian(1 << 18, 1 << 16, 1e-4, seed=0)
    absv = np.abs(np.asarray(X.val, dtype=np.float64))
    rows = np.repeat(np.arange(X.nrows), np.diff(X.rowptr))
    b = float(np.bincount(rows, weights=absv).max()) * float(np.bincount(X.col, weights=absv).max())
    deg = np.full(512, 512, dtype=np.int32)
    with L.Matrix(X, gram=True) as M:
        L.mlt_autotune(M.handle, "fp32", 4)
        got = M.moments(0.0, b, 0, 0, deg, precision="fp32")
    tol = _tol32(512, X.ncols)
    _check_all(got, deg, X.ncols, tol)
    _check_sampled(O, X, 0.0, b, 0, 0, got, [(511, 32)], tol, gram=True)


def test_estrada_rmat22_fp32_full_size(L, O):
    # the R-MAT scale-22 adjacency scaled into [-10, 10] (by its largest degree,
    # a Gershgorin bound), 256 probes to degree 128 in FP32: two probe groups;
    # one probe of the second group checked to degree 2 (128M entries a step)
    g = synth.rmat_adjacency(22, 16, seed=1)
    scale = 10.0 / float(np.max(np.diff(g.rowptr)))
    deg = np.full(256, 128, dtype=np.int32)
    with L.Matrix(g, scale=scale) as M:
        L.mlt_autotune(M.handle, "fp32", 4)
        got = M.moments(-10.0, 10.0, 0, 0, deg, precision="fp32")
    tol = _tol32(128, g.nrows)
    _check_all(got, deg, g.nrows, tol)
    _check_sampled(O, g, -10.0, 10.0, 0, 0, got, [(255, 2)], tol, scale=scale)

