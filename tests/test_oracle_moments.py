"""Pins of the oracle's Chebyshev moments mu_j = z^T T_j(At) z (Section 2.2,
recurrence Eq. recurrence, affine map to [-1, 1]) against a dense
eigendecomposition, where T_j(x) = cos(j arccos x) needs no recurrence."""
import itertools

import numpy as np
import pytest

from paper_2103_10516_gb300 import synth


def _spectral_moments(A, a, b, z, deg):
    lam, Q = np.linalg.eigh(A)
    lt = (2.0 * lam - (a + b)) / (b - a)
    assert np.all(np.abs(lt) <= 1.0 + 1e-12)
    th = np.arccos(np.clip(lt, -1, 1))
    w = (Q.T @ z) ** 2
    return np.array([np.sum(w * np.cos(j * th)) for j in range(deg + 1)])


@pytest.mark.parametrize("seed", [0, 1])
def test_moments_match_eigendecomposition(O, seed):
    m = synth.random_symmetric(40, 0.15, seed=seed, diag_shift=0.0)
    A = m.to_dense()
    lam = np.linalg.eigvalsh(A)
    a, b = lam[0] - 0.05, lam[-1] + 0.05
    deg = 60
    mu = O.moments(m, a, b, 3, 5, [deg, deg])
    for p in range(2):
        z = O.rademacher(3, 5 + p, 40).astype(np.float64)
        ref = _spectral_moments(A, a, b, z, deg)
        assert np.max(np.abs(mu[p] - ref)) < 1e-11 * 40


def test_moments_gram_operator(O):
    X = synth.sparse_gaussian(30, 12, 0.3, seed=4)
    A = X.to_dense().T @ X.to_dense()
    lam = np.linalg.eigvalsh(A)
    a, b = 0.0, lam[-1] * 1.01
    mu = O.moments(X, a, b, 9, 0, [33], gram=True)
    z = O.rademacher(9, 0, 12).astype(np.float64)
    ref = _spectral_moments(A, a, b, z, 33)
    assert np.max(np.abs(mu[0] - ref)) < 1e-11 * 12


def test_pattern_scale(O):
    g = synth.random_graph(30, 0.2, seed=2)
    A = g.to_dense() * 0.25
    lam = np.linalg.eigvalsh(A)
    a, b = lam[0] - 0.1, lam[-1] + 0.1
    mu = O.moments(g, a, b, 0, 0, [20], scale=0.25)
    z = O.rademacher(0, 0, 30).astype(np.float64)
    assert np.max(np.abs(mu[0] - _spectral_moments(A, a, b, z, 20))) < 1e-11 * 30


def test_invariants_and_ragged_degrees(O):
    m = synth.grid_laplacian_2d(8, shift=0.1)
    degs = [0, 1, 2, 17, 5]
    mu = O.moments(m, 0.1, 8.1, 0, 0, degs)
    assert mu.shape == (5, 18)
    assert np.all(mu[:, 0] == 64.0)                      # mu_0 = z.z = d exactly
    assert np.all(np.abs(mu) <= 64.0 * (1 + 1e-12))      # |T_j| <= 1 on the spectrum
    for p, dg in enumerate(degs):
        assert np.all(mu[p, dg + 1:] == 0.0)
    # a probe's moments do not depend on the other probes or its degree
    full = O.moments(m, 0.1, 8.1, 0, 3, [17])
    assert np.array_equal(full[0], mu[3])
    short = O.moments(m, 0.1, 8.1, 0, 4, [5])
    assert np.array_equal(short[0][:6], mu[4][:6])


def test_exhaustive_sign_average_is_trace(O):
    # Theorem 2.1 made exact: averaging z^T p_n(At) z over all 2^d sign vectors
    # gives tr p_n(At) = sum_i p_n(lambda~_i)
    d = 10
    m = synth.random_symmetric(d, 0.4, seed=7, diag_shift=1.0)
    A = m.to_dense()
    lam = np.linalg.eigvalsh(A)
    a, b = lam[0] - 0.2, lam[-1] + 0.2
    n = 12
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=d)))
    mu = O.moments_z(m, a, b, Z, n)
    c = O.cheb_coeffs("exp", a, b, n)
    per_probe = mu @ c
    lt = (2.0 * lam - (a + b)) / (b - a)
    assert abs(per_probe.mean() - np.sum(O.cheb_eval(c, lt))) < 1e-11 * np.sum(np.abs(c)) * d
    # each moment's average is tr T_j(At)
    th = np.arccos(np.clip(lt, -1, 1))
    for j in range(n + 1):
        assert abs(mu[:, j].mean() - np.sum(np.cos(j * th))) < 1e-11 * d


def test_row_parallel_products_change_no_bit(O):
    """With fewer probes than threads the oracle spreads each product's rows
    over the threads instead of spreading the probes; each row is still summed
    alone in entry order, so every moment is the same to the last bit."""
    import os
    g = synth.rmat_adjacency(11, 16, seed=6)
    sc = 0.02
    a, b = O.interval(g, scale=sc)
    many = O.moments(g, a, b, 3, 0, [30] * (2 * (os.cpu_count() or 1) + 2), scale=sc)
    for p in (0, 5):
        one = O.moments(g, a, b, 3, p, [30], scale=sc)
        assert np.array_equal(one[0], many[p])
