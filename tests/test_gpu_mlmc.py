"""GPU parity of the multilevel estimator (mlt_mlmc_estimate) against the
oracle on the same probes: same levels and sample counts, and estimates within
1e-10 * sum|c_j| * d (each band is a c-weighted sum of moments with |mu_j| <= d).
Also the exact low-degree traces (mlt_low_traces) and the low-degree control
variates (MLT_LOW_CV) of Section 5.4."""
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


def test_c1_fixed_levels(L, O):
    m = synth.grid_laplacian_2d(64, shift=0.1)
    ref = O.mlmc_fixed(m, "log", 0.1, 8.1, 128, [8, 32, 128], [256, 64, 16], seed=0)
    with L.Matrix(m) as M:
        got = M.mlmc("log", 0.1, 8.1, 128, seed=0, levels=[8, 32, 128], m=[256, 64, 16])
    tol = 1e-10 * np.sum(np.abs(ref["coeffs"])) * m.nrows
    assert got["levels"] == [8, 32, 128] and got["m"] == [256, 64, 16]
    assert abs(got["estimate"] - ref["estimate"]) <= tol
    assert np.max(np.abs(np.array(got["level_mean"]) - ref["level_mean"])) <= tol
    assert abs(got["stderr"] - ref["stderr"]) <= 1e-6 * ref["stderr"]
    assert got["matvecs"] == 256 * 4 + 64 * 16 + 16 * 64
    # against the exact log-determinant (closed form) within 5 standard errors
    k = np.arange(1, 65)
    e = 2.0 - 2.0 * np.cos(k * np.pi / 65.0)
    logdet = float(np.sum(np.log((e[:, None] + e[None, :]).ravel() + 0.1)))
    assert abs(got["estimate"] - logdet) < 5 * got["stderr"]


@pytest.mark.parametrize("mode,target,max_levels", [("budget", 3000.0, 0), ("budget", 3000.0, 3),
                                                     ("variance", 4.0, 0)])
def test_auto_levels(L, O, mode, target, max_levels):
    m = synth.grid_laplacian_2d(24, shift=0.1)
    n = 48
    ref = O.mlmc_auto(m, "log", 0.1, 8.1, n, seed=2, m_pilot=10, mode=mode, target=target,
                      max_levels=max_levels)
    with L.Matrix(m) as M:
        got = M.mlmc("log", 0.1, 8.1, n, seed=2, m_pilot=10, mode=mode, target=target,
                     max_levels=max_levels)
    assert got["levels"] == ref["levels"]
    assert got["m"] == ref["m"]
    tol = 1e-10 * np.sum(np.abs(ref["coeffs"])) * m.nrows
    assert abs(got["estimate"] - ref["estimate"]) <= tol


def test_nuclear_norm_gram(L, O):
    X = synth.sparse_gaussian(400, 150, 0.03, seed=1)
    _, b = O.interval(X, gram=True)
    a = 1e-3 * b
    with L.Matrix(X, gram=True) as M:
        got = M.mlmc("sqrt", a, b, 40, seed=0, levels=[4, 12, 40], m=[40, 12, 6])
    ref = O.mlmc_fixed(X, "sqrt", a, b, 40, [4, 12, 40], [40, 12, 6], seed=0, gram=True)
    tol = 1e-10 * np.sum(np.abs(ref["coeffs"])) * 150
    assert abs(got["estimate"] - ref["estimate"]) <= tol


@pytest.mark.parametrize("kind", ["values", "pattern_scaled", "gram", "fp32_values"])
def test_low_traces_match_oracle(L, O, kind):
    gram, scale, vdt = False, 1.0, None
    if kind == "values":
        m = synth.grid_laplacian_2d(40, shift=0.3)
        a, b = 0.3, 8.3
    elif kind == "pattern_scaled":
        m = synth.rmat_adjacency(12, 8, seed=3)
        scale = 0.05
        a, b = -4.0, 4.0
    elif kind == "gram":
        m = synth.sparse_gaussian(500, 200, 0.02, seed=5)
        gram, scale = True, 0.8
        a, b = 0.0, 60.0
    else:
        m = synth.random_symmetric(700, 0.01, seed=4, diag_shift=2.0)
        m = synth.CSR(m.nrows, m.ncols, m.rowptr, m.col, m.val.astype(np.float32).astype(np.float64))
        vdt = np.float32
        a, b = -3.0, 7.0
    with L.Matrix(m, gram=gram, scale=scale, vals_dtype=vdt) as M:
        got = L.mlt_low_traces(M.handle, a, b)
    ref = O.exact_low_traces(m, a, b, gram, scale)
    assert len(got) == len(ref)
    # both sides add the same terms in different orders: the difference is a
    # few roundings of the magnitudes the sums carry
    alpha = 2.0 / (b - a)
    v = np.ones(m.nnz) if m.val is None else np.abs(m.val)
    mag = (m.ncols if gram else m.nrows) + abs(alpha) * scale * np.sum(v) + (alpha * scale) ** 2 * np.sum(v * v)
    assert np.max(np.abs(got - np.array(ref))) <= 1e-13 * mag * 8


def test_low_cv_mlmc_matches_oracle(L, O):
    # fixed and automatic levels with the low-degree control variates: same
    # levels, counts, estimates and level variances as the oracle, and no level
    # whose residual variance exceeds its plain variance (least squares)
    m = synth.random_symmetric(3000, 0.002, seed=11, diag_shift=1.0)
    lo, hi = O.interval(m)
    ref = O.mlmc_fixed(m, "exp", lo, hi, 24, [4, 24], [300, 40], seed=5, low_cv=True)
    plain = O.mlmc_fixed(m, "exp", lo, hi, 24, [4, 24], [300, 40], seed=5)
    with L.Matrix(m) as M:
        got = M.mlmc("exp", lo, hi, 24, seed=5, levels=[4, 24], m=[300, 40], low_cv=True)
        auto = M.mlmc("exp", lo, hi, 24, seed=6, m_pilot=12, mode="budget", target=2000.0, low_cv=True)
    tol = 1e-10 * np.sum(np.abs(ref["coeffs"])) * m.nrows
    assert got["m"] == [300, 40]
    assert abs(got["estimate"] - ref["estimate"]) <= tol
    assert np.max(np.abs(np.array(got["level_mean"]) - ref["level_mean"])) <= tol
    assert np.allclose(got["level_var"], ref["level_var"], rtol=1e-8)
    for k, mk in enumerate((300, 40)):
        assert got["level_var"][k] * (mk - 3) <= plain["level_var"][k] * (mk - 1) * (1 + 1e-9)
    aref = O.mlmc_auto(m, "exp", lo, hi, 24, seed=6, m_pilot=12, mode="budget", target=2000.0, low_cv=True)
    assert auto["levels"] == aref["levels"] and auto["m"] == aref["m"]
    assert abs(auto["estimate"] - aref["estimate"]) <= tol


def test_pilot_variances_from_gpu_moments_match_oracle(L, O):
    """The library's pilot variance table (Section 3.2.1), computed from pilot
    moments of the GPU engine, against the oracle's table from its own moments
    of the same probes, entry by entry.  A moment error e (|e| <= 1e-10 d) moves
    a band sample by at most dq = 1e-10 d sum|c|, so a sample variance moves by
    at most 2 dq (sqrt(V m / (m - 1)) + dq) m / (m - 1)."""
    m = synth.grid_laplacian_2d(24, shift=0.1)
    n, mp = 48, 12
    c = O.cheb_coeffs("log", 0.1, 8.1, n)
    with L.Matrix(m) as M:
        mu = M.moments(0.1, 8.1, 2, 0, [n] * mp)
    V = L.mlt_pilot_variances(c, mu)
    ref = O.pilot_variances(c, O.moments(m, 0.1, 8.1, 2, 0, [n] * mp))
    dq = 1e-10 * m.nrows * np.sum(np.abs(c))
    f = mp / (mp - 1.0)
    tol = 2.0 * dq * (np.sqrt(ref * f) + dq) * f
    assert np.all(np.abs(V - ref) <= tol + 1e-300)
    assert np.all(np.tril(V) == 0.0)


@pytest.mark.parametrize("auto", [True, False])
def test_sharded_path_one_rank_is_mlmc_estimate(L, O, auto):
    """The sharded driver on one process (no collective) makes the same moment
    calls as mlt_mlmc_estimate and combines with the same routines, so its
    estimate equals the library's to the last bit; both match the oracle."""
    from paper_2103_10516_gb300 import shard
    m = synth.grid_laplacian_2d(24, shift=0.1)
    n = 48
    kw = dict(m_pilot=10, mode="budget", target=3000.0) if auto else dict(levels=[8, 24, 48], m=[60, 20, 6])
    with L.Matrix(m) as M:
        lib = M.mlmc("log", 0.1, 8.1, n, seed=2, **kw)
        sh = shard.mlmc_sharded(shard.library_moments(M.handle, 0.1, 8.1, 2), "log", 0.1, 8.1, n, **kw)
    for f in ("estimate", "stderr", "levels", "m", "level_mean", "level_var", "probes", "matvecs"):
        np.testing.assert_array_equal(np.asarray(sh[f]), np.asarray(lib[f]), err_msg=f)   # NaN == NaN
    ref = O.mlmc_auto(m, "log", 0.1, 8.1, n, seed=2, **kw) if auto else \
        O.mlmc_fixed(m, "log", 0.1, 8.1, n, kw["levels"], kw["m"], seed=2)
    assert abs(sh["estimate"] - ref["estimate"]) <= 1e-10 * np.sum(np.abs(ref["coeffs"])) * m.nrows
