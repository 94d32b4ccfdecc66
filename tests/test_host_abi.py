"""The library's host-side multilevel and triangle arithmetic through the C ABI,
without a GPU: pilot variances (Section 3.2.1), level selection and sample
counts (Theorem levels, Eqs. optSamples / optMu), band samples (Eq.
def:qlevels), the combination (Eq. multiEstimator) and the triangle estimates
of Section 5.4, each against the oracle on the same inputs."""
import itertools

import numpy as np
import pytest

from paper_2103_10516_gb300 import synth


@pytest.fixture(scope="module")
def L():
    from paper_2103_10516_gb300 import build, mlt
    build.build()
    return mlt


def _pilot(O, n=24, m=9, seed=5):
    g = synth.grid_laplacian_2d(10, shift=0.1)
    c = O.cheb_coeffs("log", 0.1, 8.1, n)
    return c, O.moments(g, 0.1, 8.1, seed, 0, [n] * m)


def test_pilot_variances_match_oracle(L, O):
    c, mu = _pilot(O)
    V = L.mlt_pilot_variances(c, mu)
    ref = O.pilot_variances(c, mu)
    assert np.all((V == 0) == (ref == 0))
    nz = ref > 0
    assert np.max(np.abs(V[nz] - ref[nz]) / ref[nz]) < 1e-12


def test_pilot_variances_exhaustive_closed_form(L, O):
    """The library's table against the Hutchinson variance of each band's
    matrix over all 2^d sign vectors (the same pin as the oracle's)."""
    d, n = 6, 8
    m = synth.random_symmetric(d, 0.6, seed=4, diag_shift=1.0)
    lam, Q = np.linalg.eigh(m.to_dense())
    a, b = float(lam[0]) - 0.2, float(lam[-1]) + 0.3
    c = O.cheb_coeffs("exp", a, b, n)
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=d)))
    mu = O.moments_z(m, a, b, Z, n)
    V = L.mlt_pilot_variances(c, mu)
    th = np.arccos(np.clip((2 * lam - (a + b)) / (b - a), -1, 1))
    N = Z.shape[0]
    for lo in range(n):
        for hi in range(lo + 1, n + 1):
            B = (Q * sum(c[j] * np.cos(j * th) for j in range(lo + 1, hi + 1))) @ Q.T
            exact = 2.0 * (np.sum(B * B) - np.sum(np.diag(B) ** 2)) * N / (N - 1)
            assert abs(V[lo, hi] - exact) < 1e-9 * exact
    assert np.all(np.tril(V) == 0)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("kw", [dict(cost_model="symmetric", m_pilot=0, mode="budget", target=3000.0),
                                dict(cost_model="linear", m_pilot=6, mode="budget", target=900.0),
                                dict(cost_model="symmetric", m_pilot=6, mode="variance", target=0.05),
                                dict(cost_model="symmetric", m_pilot=6, mode="budget", target=2000.0,
                                     max_levels=3)])
def test_select_levels_match_oracle(L, O, seed, kw):
    rng = np.random.default_rng(seed)
    n = 30
    terms = rng.standard_normal((12, n + 1)) * np.exp(-0.15 * np.arange(n + 1))[None, :]
    V = O.pilot_variances(np.ones(n + 1), terms)
    levels, m = L.mlt_select_levels(V, **kw)
    ref_levels = O.select_levels(V, kw["cost_model"], kw["m_pilot"], kw["mode"], kw["target"],
                                 kw.get("max_levels", 0))
    ref_m = O.allocate(ref_levels, V, kw["cost_model"], kw["mode"], kw["target"], kw["m_pilot"])
    assert levels == ref_levels and m == ref_m


def test_select_levels_rejects_bad_input(L):
    V = np.zeros((5, 5))
    for kw in (dict(target=0.0), dict(mode=7), dict(cost_model=9), dict(m_pilot=-1)):
        args = dict(cost_model="symmetric", m_pilot=0, mode="budget", target=10.0)
        args.update(kw)
        with pytest.raises(L.MLTError) as e:
            L.mlt_select_levels(V, **args)
        assert e.value.code == L.MLT_EINVAL
    V[0, 2] = -1.0
    with pytest.raises(L.MLTError):
        L.mlt_select_levels(V, target=10.0)


def test_band_samples_and_combine_match_oracle(L, O):
    c, mu = _pilot(O, n=32, m=11)
    for lo, hi in ((-1, 4), (4, 17), (17, 32), (-1, 32)):
        got = L.mlt_band_samples(c, lo, hi, mu)
        ref = O.band(c, mu, lo, hi)
        assert np.max(np.abs(got - ref)) <= 1e-14 * np.sum(np.abs(c)) * 100
    # the combination of fixed levels against the oracle's estimator on the same probes
    g = synth.grid_laplacian_2d(10, shift=0.1)
    levels, m = [4, 17, 32], [20, 8, 3]
    ref = O.mlmc_fixed(g, "log", 0.1, 8.1, 32, levels, m, seed=3)
    parts, off, lo = [], 0, -1
    for l, mk in zip(levels, m):
        rows = O.moments(g, 0.1, 8.1, 3, off, [l] * mk)
        parts.append(L.mlt_band_samples(ref["coeffs"], lo, l, rows))
        off, lo = off + mk, l
    got = L.mlt_mlmc_combine(levels, m, np.concatenate(parts))
    tol = 1e-12 * np.sum(np.abs(ref["coeffs"])) * g.nrows
    assert abs(got["estimate"] - ref["estimate"]) <= tol
    assert abs(got["stderr"] - ref["stderr"]) <= 1e-10 * ref["stderr"]
    assert got["levels"] == levels and got["m"] == m
    assert np.allclose(got["level_var"], ref["level_var"], rtol=1e-10, atol=0)
    with pytest.raises(L.MLTError):
        L.mlt_mlmc_combine([4], [0], np.zeros(0))


@pytest.mark.parametrize("cv", ["none", "fit", "cheb"])
def test_triangle_estimate_bit_exact(L, O, cv):
    """Same integers in, same formula and operation order: the library's
    estimate and standard error equal the oracle's to the last bit."""
    g = synth.random_graph(150, 0.06, seed=8)
    x = O.triangle_moments(g, 4, 0, 97)
    dmax = float(np.max(np.diff(g.rowptr)))
    est, se, a1, a2 = L.mlt_triangle_estimate(x, g.nnz, cv, -dmax, dmax)
    if cv == "cheb":
        ra1, ra2 = O.triangle_cv_cheb(-dmax, dmax)
        er, sr = O.triangle_estimate_fixed(x, g.nnz, ra1, ra2)
        assert (a1, a2) == (ra1, ra2)
    else:
        er, sr, ra1, ra2 = O.triangle_estimate(x, g.nnz, cv == "fit")
        if cv == "fit":
            assert (a1, a2) == (ra1, ra2)
    assert est == er and se == sr


def test_triangle_estimate_rejects_bad_input(L):
    x = np.zeros((4, 3), dtype=np.int64)
    for cv, a, b in (("cheb", 1.0, 1.0), (7, 0.0, 1.0)):
        with pytest.raises(L.MLTError) as e:
            L.mlt_triangle_estimate(x, 10, cv, a, b)
        assert e.value.code == L.MLT_EINVAL
