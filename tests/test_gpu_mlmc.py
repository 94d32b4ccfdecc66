"""GPU parity of the multilevel estimator (mlt_mlmc_estimate) against the
oracle on the same probes: same levels and sample counts, and estimates within
1e-10 * sum|c_j| * d (each band is a c-weighted sum of moments with |mu_j| <= d)."""
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
    with L.Matrix(X, gram=True) as M:
        a, b = M.bounds()
        a = 1e-3 * b
        got = M.mlmc("sqrt", a, b, 40, seed=0, levels=[4, 12, 40], m=[40, 12, 6])
    ref = O.mlmc_fixed(X, "sqrt", a, b, 40, [4, 12, 40], [40, 12, 6], seed=0, gram=True)
    tol = 1e-10 * np.sum(np.abs(ref["coeffs"])) * 150
    assert abs(got["estimate"] - ref["estimate"]) <= tol
