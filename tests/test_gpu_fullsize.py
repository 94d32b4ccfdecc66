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

The oracle sums in long double, which is quad precision in software on
aarch64; with fewer probes than host threads it spreads each product's rows
over the threads (the same arithmetic), so a few probes per test reach the
degrees the benchmarks use: degree 64 on the stencil and the Gram operator,
degree 16 on the scale-22 graph (the moments the learned level consumes).
FP64 and double-float runs are held to the FP64 tolerance 1e-10 d.  The bound
|mu_j| <= d (+ tol) is checked on every moment of every probe."""
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


def _spread(nprobes, k):
    """k probe indices spread over [0, nprobes): first, last and between, so
    that several probe groups are sampled."""
    return sorted(set(int(round(i * (nprobes - 1) / (k - 1))) for i in range(k)))


def test_stencil3d_fp32_full_size(L, O):
    # the 100^3 diffusion operator, 128 probes to degree 128 in FP32; four probes
    # checked to degree 64
    m = synth.diffusion_3d(100, sigma=1.0, shift=0.1, seed=0)
    a, b = 0.1, O.gershgorin(m)[1]
    deg = np.full(128, 128, dtype=np.int32)
    with L.Matrix(m) as M:
        L.mlt_autotune(M.handle, "fp32", 4)
        got = M.moments(a, b, 0, 4096, deg, precision="fp32")
    tol = _tol32(128, m.nrows)
    _check_all(got, deg, m.nrows, tol)
    _check_sampled(O, m, a, b, 0, 4096, got, [(p, 64) for p in _spread(128, 4)], tol)


def test_stencil3d_fp64_full_size(L, O):
    # the same operator in FP64, 128 probes to degree 64: four probes to degree 64
    # at the FP64 tolerance
    m = synth.diffusion_3d(100, sigma=1.0, shift=0.1, seed=0)
    a, b = 0.1, O.gershgorin(m)[1]
    deg = np.full(128, 64, dtype=np.int32)
    with L.Matrix(m) as M:
        got = M.moments(a, b, 0, 8192, deg, precision="fp64")
    tol = 1e-10 * m.nrows
    _check_all(got, deg, m.nrows, tol)
    _check_sampled(O, m, a, b, 0, 8192, got, [(p, 64) for p in _spread(128, 4)], tol)


def test_nuclear_gram_fp32_full_size(L, O):
    # X^T X with X 2^18 x 2^16 (density 1e-4), 512 probes to degree 512 in FP32;
    # the interval's upper end is ||X||_1 ||X||_inf >= ||X||_2^2; four probes
    # from different groups checked to degree 64
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
    _check_sampled(O, X, 0.0, b, 0, 0, got, [(p, 64) for p in _spread(512, 4)], tol, gram=True)


@pytest.fixture(scope="module")
def rmat22():
    g = synth.rmat_adjacency(22, 16, seed=1)
    return g, 10.0 / float(np.max(np.diff(g.rowptr)))


def test_estrada_rmat22_fp32_full_size(L, O, rmat22):
    # the R-MAT scale-22 adjacency scaled into [-10, 10] (by its largest degree,
    # a Gershgorin bound), 256 probes to degree 128 in FP32: two probe groups;
    # four probes across both groups checked to degree 16
    g, scale = rmat22
    deg = np.full(256, 128, dtype=np.int32)
    with L.Matrix(g, scale=scale) as M:
        L.mlt_autotune(M.handle, "fp32", 4)
        got = M.moments(-10.0, 10.0, 0, 0, deg, precision="fp32")
    tol = _tol32(128, g.nrows)
    _check_all(got, deg, g.nrows, tol)
    _check_sampled(O, g, -10.0, 10.0, 0, 0, got, [(p, 16) for p in _spread(256, 4)], tol, scale=scale)


def test_estrada_rmat22_df64_full_size_reordered(L, O, rmat22):
    # the default benchmark's configuration: the graph relabelled by degree
    # (MLT_REORDER), double-float moments of 128 probes to degree 128 at the
    # autotuned group width; four probes checked to degree 16 at the FP64
    # tolerance
    g, scale = rmat22
    deg = np.full(128, 128, dtype=np.int32)
    with L.Matrix(g, scale=scale, reorder=True) as M:
        L.mlt_autotune(M.handle, "df64", 4)
        got = M.moments(-10.0, 10.0, 0, 0, deg, precision="df64")
    tol = 1e-10 * g.nrows
    _check_all(got, deg, g.nrows, tol)
    _check_sampled(O, g, -10.0, 10.0, 0, 0, got, [(p, 16) for p in _spread(128, 4)], tol, scale=scale)


def test_diffusion64_batched_fp64_full_size(L, O):
    """The 64 diffusion operators of the batched workload (grids 10^3 .. 100^3,
    sum of d about 9.6e6) as one persistent batch in FP64, each matrix's
    ragged levels as the benchmark runs them; for every matrix its first
    probe (degree 16) in full and its last probe (degree 256) through degree
    16 against the oracle, and |mu_j| <= d for every moment."""
    import torch
    mats, jobs, outs, Ms = [], [], [], []
    try:
        for i in range(64):
            side = int(round(10 * 10 ** (i / 63)))
            sh = float(np.random.default_rng(1000 + i).uniform(0.01, 1.0))
            m = synth.diffusion_3d(side, sigma=1.0, shift=sh, seed=i)
            lv, mm = ([16, 64, 256], [64, 16, 4]) if i % 2 == 0 else ([16, 48, 128, 256], [64, 32, 8, 4])
            deg = np.repeat(np.array(lv, dtype=np.int32), mm)
            b = float(np.max(np.add.reduceat(np.abs(m.val), m.rowptr[:-1])))   # Gershgorin (positive diagonal)
            M = L.Matrix(m)
            Ms.append(M)
            out = torch.zeros((deg.size, 257), dtype=torch.float64, device="cuda")
            outs.append(out)
            mats.append((m, sh, b, deg))
            jobs.append({"matrix": M.handle, "a": sh, "b": b, "seed": 7, "probe_offset": 3 * 128, "degrees": deg,
                         "out": out})
        with L.Batch(jobs) as B:
            B.run(0)
            torch.cuda.synchronize()
        tol = 1e-10
        for (m, sh, b, deg), out in zip(mats, outs):
            got = out.cpu().numpy()
            d = m.nrows
            _check_all(got, deg, d, tol * d)
            _check_sampled(O, m, sh, b, 7, 3 * 128, got, [(0, 16), (deg.size - 1, 16)], tol * d)
    finally:
        for M in Ms:
            M.close()
