"""Pins of the oracle's polynomial application and Hutch++ (the variance
reduction Section 5.3 proposes for the Estrada index): p(At) X against a dense
eigendecomposition and an exact cube, the full-sketch case that leaves no
remainder, exhaustive remainder signs that make the estimate exact, and
unbiasedness and variance reduction over seeds."""
import itertools
import math

import numpy as np

from paper_2103_10516_gb300 import synth


def _mapped_eigs(A, a, b):
    lam, V = np.linalg.eigh(A)
    return (2 * lam - (a + b)) / (b - a), V


def test_poly_apply_matches_dense_eigendecomposition(O):
    cases = [(synth.random_symmetric(60, 0.08, seed=3, diag_shift=3.0), "exp", 40, 0.2),
             (synth.grid_laplacian_2d(8, shift=0.1), "log", 48, 0.0)]
    for m, fn, n, pad in cases:
        A = m.to_dense()
        lam = np.linalg.eigvalsh(A)
        a, b = lam[0] - pad if fn == "exp" else 0.1, lam[-1] + 0.2
        c = O.cheb_coeffs(fn, a, b, n)
        X = np.random.default_rng(0).standard_normal((m.nrows, 7))
        t, V = _mapped_eigs(A, a, b)
        want = V @ np.diag(O.cheb_eval(c, t)) @ V.T @ X     # p through cos(j arccos t)
        got = O.poly_apply(m, a, b, c, X)
        assert np.max(np.abs(got - want)) < 1e-11 * np.sum(np.abs(c)) * np.max(np.abs(X)), fn


def test_poly_apply_cube_is_exact_power(O):
    # x^3 interpolated at degree 5 is x^3 itself: p(At) = A^3 on the original scale
    m = synth.random_symmetric(30, 0.2, seed=5, diag_shift=1.0)
    A = m.to_dense()
    X = np.random.default_rng(1).standard_normal((30, 3))
    c = O.cheb_coeffs("cube", -6.0, 9.0, 5)
    got = O.poly_apply(m, -6.0, 9.0, c, X)
    want = A @ (A @ (A @ X))
    assert np.max(np.abs(got - want)) < 1e-10 * np.max(np.abs(want))


def test_poly_apply_gram_and_scale(O):
    X = synth.sparse_gaussian(25, 12, 0.3, seed=2)
    D = 0.5 * X.to_dense()
    A = D.T @ D
    lam = np.linalg.eigvalsh(A)
    a, b = max(lam[0], 0.0) + 1e-3, lam[-1] + 0.1
    c = O.cheb_coeffs("sqrt", 0.0, b, 24)
    V = np.random.default_rng(2).standard_normal((12, 4))
    t, E = _mapped_eigs(A, 0.0, b)
    want = E @ np.diag(O.cheb_eval(c, t)) @ E.T @ V
    got = O.poly_apply(X, 0.0, b, c, V, gram=True, scale=0.5)
    assert np.max(np.abs(got - want)) < 1e-11 * np.sum(np.abs(c)) * np.max(np.abs(V))


def _exact_trace(O, A, a, b, c):
    t, _ = _mapped_eigs(A, a, b)
    return math.fsum(O.cheb_eval(c, t).tolist())


def test_full_sketch_leaves_no_remainder(O):
    # s >= d: Q spans the whole space, t1 is tr p(At) and every remainder is zero
    d = 24
    m = synth.random_graph(d, 0.3, seed=7)
    A = m.to_dense()
    lam = np.linalg.eigvalsh(A)
    a, b = lam[0] - 0.5, lam[-1] + 0.5
    c = O.cheb_coeffs("exp", a, b, 30)
    r = O.hutchpp(m, a, b, c, seed=3, probe_offset=0, s=d, g=4)
    exact = _exact_trace(O, A, a, b, c)
    assert r["rank"] == d
    assert abs(r["t_sketch"] - exact) < 1e-10 * abs(exact)
    assert np.max(np.abs(r["samples"])) < 1e-10 * abs(exact)
    assert abs(r["estimate"] - exact) < 1e-10 * abs(exact)


def test_exhaustive_remainder_signs_make_it_exact(O):
    # for any fixed Q, the mean of g'^T p g' over all 2^d sign vectors g is
    # tr((I - QQ^T) p (I - QQ^T)), and t1 + that is tr p(At)
    d = 10
    m = synth.random_symmetric(d, 0.4, seed=8, diag_shift=2.0)
    A = m.to_dense()
    lam = np.linalg.eigvalsh(A)
    a, b = lam[0] - 0.3, lam[-1] + 0.3
    c = O.cheb_coeffs("exp", a, b, 16)
    S = np.stack([O.rademacher(4, i, d) for i in range(3)], axis=1).astype(np.float64)
    G = np.array(list(itertools.product([-1.0, 1.0], repeat=d))).T
    t1, samples, rank = O.hutchpp_parts(m, a, b, c, S, G)
    assert rank == 3
    exact = _exact_trace(O, A, a, b, c)
    assert abs(t1 + math.fsum(samples.tolist()) / samples.size - exact) < 1e-11 * d * np.sum(np.abs(c))
    # and t1 alone is the trace over span(Q): below the total for this positive p
    assert 0.0 < t1 < exact


def test_dependent_sketch_columns_are_dropped(O):
    # repeated sketch columns: the copies add nothing to span(Q)
    d = 20
    m = synth.random_symmetric(d, 0.3, seed=9, diag_shift=2.0)
    lam = np.linalg.eigvalsh(m.to_dense())
    a, b = lam[0] - 0.3, lam[-1] + 0.3
    c = O.cheb_coeffs("exp", a, b, 12)
    z = O.rademacher(1, 0, d).astype(np.float64)
    S = np.stack([z, O.rademacher(1, 1, d), z, 2.0 * z], axis=1).astype(np.float64)
    G = np.stack([O.rademacher(1, 10 + i, d) for i in range(5)], axis=1).astype(np.float64)
    t1, samples, rank = O.hutchpp_parts(m, a, b, c, S, G)
    t1b, samplesb, rankb = O.hutchpp_parts(m, a, b, c, S[:, :2], G)
    assert rank == 2 and rankb == 2
    assert abs(t1 - t1b) < 1e-10 * abs(t1b)
    assert np.max(np.abs(samples - samplesb)) < 1e-9 * np.max(np.abs(samplesb))


def test_unbiased_and_lower_variance_than_hutchinson(O):
    # a spectrum dominated by a few large eigenvalues (exp of a scaled graph),
    # where deflation pays: over many seeds the Hutch++ mean is within 4 sigma of
    # tr p, and its spread is below plain Hutchinson's at the same matvec count
    d = 60
    m = synth.random_graph(d, 0.15, seed=11)
    A = m.to_dense()
    lam = np.linalg.eigvalsh(A)
    a, b = lam[0] - 0.2, lam[-1] + 0.2
    n = 24
    c = O.cheb_coeffs("exp", a, b, n)
    exact = _exact_trace(O, A, a, b, c)
    s, g = 4, 4
    est = []
    for seed in range(120):
        est.append(O.hutchpp(m, a, b, c, seed=seed, probe_offset=0, s=s, g=g)["estimate"])
    est = np.array(est)
    assert abs(est.mean() - exact) < 4 * est.std(ddof=1) / math.sqrt(est.size)
    # plain Hutchinson with the same operator applications: s sketch columns
    # cost n (p(At) S) + n/2 (their moments), a remainder probe n/2
    k = int(round((s * 1.5 * n + g * 0.5 * n) / (0.5 * n)))
    plain = []
    for seed in range(120):
        mu = O.moments(m, a, b, seed, 0, [n] * k)
        plain.append(float(np.mean(mu @ c)))
    assert est.std(ddof=1) < 0.5 * np.std(plain, ddof=1)
