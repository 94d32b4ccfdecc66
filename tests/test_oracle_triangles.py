"""Pins of the oracle's triangle path (Section 2.1 Example: triangles = tr(A^3)/6;
Section 5.4: control variates with tr A = 0, tr A^2 = nnz(A))."""
import itertools
import math

import numpy as np
import pytest

from paper_2103_10516_gb300 import synth


@pytest.mark.parametrize("d,p,seed", [(40, 0.2, 0), (80, 0.1, 1), (25, 0.6, 2)])
def test_bruteforce_count_matches_networkx(O, d, p, seed):
    nx = pytest.importorskip("networkx")
    g = synth.random_graph(d, p, seed=seed)
    G = nx.from_numpy_array(g.to_dense())
    assert O.triangle_count(g) == sum(nx.triangles(G).values()) // 3


@pytest.mark.parametrize("d", [3, 4, 9, 20])
def test_complete_graph(O, d):
    assert O.triangle_count(synth.complete_graph(d)) == math.comb(d, 3)


def test_moments_match_dense_powers(O):
    g = synth.random_graph(50, 0.15, seed=3)
    A = g.to_dense().astype(np.int64)
    x = O.triangle_moments(g, 5, 10, 4)
    for p in range(4):
        z = O.rademacher(5, 10 + p, 50).astype(np.int64)
        y = A @ z
        assert x[p, 0] == z @ y
        assert x[p, 1] == y @ y
        assert x[p, 2] == y @ (A @ y)
    # the trace identity on the dense matrix: tr(A^3) = 6 T
    assert np.trace(A @ A @ A) == 6 * O.triangle_count(g)


def test_exhaustive_signs_exact(O):
    d = 10
    g = synth.random_graph(d, 0.5, seed=11)
    Z = np.array(list(itertools.product([-1, 1], repeat=d)), dtype=np.int8)
    x = O.triangle_moments_z(g, Z)
    T = O.triangle_count(g)
    n = Z.shape[0]
    assert int(x[:, 2].sum()) == 6 * T * n      # E[z^T A^3 z] = tr A^3 = 6T
    assert int(x[:, 1].sum()) == g.nnz * n      # E[z^T A^2 z] = tr A^2 = nnz
    assert int(x[:, 0].sum()) == 0              # E[z^T A z] = tr A = 0


def test_control_variate_regression(O):
    g = synth.random_graph(120, 0.08, seed=5)
    x = O.triangle_moments(g, 0, 0, 64)
    est, se, a1, a2 = O.triangle_estimate(x, g.nnz, use_cv=True)
    # a1, a2 are the ordinary least-squares slopes of x3 on (1, x1, x2)
    M = np.column_stack([np.ones(64), x[:, 0], x[:, 1]]).astype(np.float64)
    coef = np.linalg.lstsq(M, x[:, 2].astype(np.float64), rcond=None)[0]
    assert abs(a1 - coef[1]) < 1e-9 * (1 + abs(coef[1]))
    assert abs(a2 - coef[2]) < 1e-9 * (1 + abs(coef[2]))
    xf = x.astype(np.float64)
    direct = (xf[:, 2] - a2 * (xf[:, 1] - g.nnz) - a1 * xf[:, 0]).mean() / 6.0
    assert abs(est - direct) < 1e-9 * abs(direct)
    resid = xf[:, 2] - a1 * xf[:, 0] - a2 * xf[:, 1]
    assert abs(se - math.sqrt(resid.var(ddof=3) / 64) / 6.0) < 1e-9 * se
    # without control variates: the plain Hutchinson mean
    est0, se0, _, _ = O.triangle_estimate(x, g.nnz, use_cv=False)
    assert est0 == (float(x[:, 2].sum()) / 64.0) / 6.0
    assert abs(se0 - math.sqrt(xf[:, 2].var(ddof=1) / 64) / 6.0) < 1e-9 * se0
    # the regression cannot raise the residual spread above the plain one
    assert se <= se0 * math.sqrt(63.0 / 61.0) + 1e-12
    T = O.triangle_count(g)
    assert abs(est - T) < 5 * se


def _offdiag_sq(B):
    return float(np.sum(B * B) - np.sum(np.diag(B) ** 2))


@pytest.mark.parametrize("shift", [None, (1.0, 2.5)])
def test_apriori_cv_coefficients_from_cheb_expansion(O, shift):
    """a1, a2 of Section 5.4 chosen a priori from x^3 = (3 T_1 + T_3)/4 on the
    mapped spectrum: A^3 - a2 A^2 - a1 A is (r^3/4) T_3(At) plus a multiple of I,
    with T_3 evaluated through the eigendecomposition as cos(3 arccos x)."""
    g = synth.random_graph(30, 0.2, seed=7)
    A = g.to_dense()
    lam, Q = np.linalg.eigh(A)
    if shift is None:      # the Gershgorin interval [-max degree, max degree]
        a, b = -float(np.max(np.diff(g.rowptr))), float(np.max(np.diff(g.rowptr)))
    else:                  # an asymmetric interval around the spectrum (c != 0)
        a, b = float(lam[0]) - shift[0], float(lam[-1]) + shift[1]
    a1, a2 = O.triangle_cv_cheb(a, b)
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    lt = (lam - c) / r
    T3 = (Q * np.cos(3 * np.arccos(np.clip(lt, -1, 1)))) @ Q.T
    lhs = A @ A @ A - a2 * (A @ A) - a1 * A - (r ** 3 / 4) * T3
    const = c ** 3 - 0.75 * c * r * r
    assert np.max(np.abs(lhs - const * np.eye(30))) < 1e-9 * (r ** 3 + abs(c) ** 3)


def test_apriori_cv_exhaustive_signs(O):
    """Over all 2^d sign vectors the a-priori estimate is the triangle count
    exactly (no fit, so no bias), and its residual variance is the Hutchinson
    variance 2 sum_{i != k} B_ik^2 of B = (r^3/4) T_3(At) (a multiple of I adds
    none); the sample variance over the 2^d vectors has divisor 2^d - 1."""
    d = 10
    g = synth.random_graph(d, 0.5, seed=11)
    A = g.to_dense()
    Z = np.array(list(itertools.product([-1, 1], repeat=d)), dtype=np.int8)
    x = O.triangle_moments_z(g, Z)
    T = O.triangle_count(g)
    lam, Q = np.linalg.eigh(A)
    a, b = float(lam[0]) - 0.5, float(lam[-1]) + 0.25
    a1, a2 = O.triangle_cv_cheb(a, b)
    est, se = O.triangle_estimate_fixed(x, g.nnz, a1, a2)
    assert abs(est - T) < 1e-9 * max(T, 1)
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    T3 = (Q * np.cos(3 * np.arccos(np.clip((lam - c) / r, -1, 1)))) @ Q.T
    N = Z.shape[0]
    pop_var = 2.0 * _offdiag_sq((r ** 3 / 4) * T3)
    got_pop_var = (se * 6.0) ** 2 * N * (N - 1) / N
    assert abs(got_pop_var - pop_var) < 1e-8 * pop_var
    # the plain estimator's spread on the same vectors is larger
    _, se0, _, _ = O.triangle_estimate(x, g.nnz, use_cv=False)
    assert se < se0


def test_fixed_coefficients_reduce_to_plain_and_regression(O):
    """With a1 = a2 = 0 the fixed-coefficient form is the plain mean (same
    variance divisor); with the fitted slopes its estimate is the regression
    estimate (the variance divisors differ: m - 1 against m - 3)."""
    g = synth.random_graph(120, 0.08, seed=5)
    x = O.triangle_moments(g, 0, 0, 64)
    est0, se0, _, _ = O.triangle_estimate(x, g.nnz, use_cv=False)
    e, s = O.triangle_estimate_fixed(x, g.nnz, 0.0, 0.0)
    assert e == est0 and abs(s - se0) <= 1e-15 * se0
    estr, ser, a1, a2 = O.triangle_estimate(x, g.nnz, use_cv=True)
    e, s = O.triangle_estimate_fixed(x, g.nnz, a1, a2)
    assert abs(e - estr) < 1e-12 * abs(estr)
    assert abs(s - ser * math.sqrt(61.0 / 63.0)) < 1e-6 * ser
