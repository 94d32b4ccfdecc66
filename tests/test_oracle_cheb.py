"""Pins of the oracle's Chebyshev interpolant (Section 2.2, Eq. chebSeries and the
extrema nodes x_j = cos(j pi / n)) against closed forms."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("n", [3, 4, 7, 16])
def test_cube_reproduced_exactly(O, n):
    # x^3 = (3 T_1 + T_3) / 4: an interpolant of degree >= 3 reproduces it
    c = O.cheb_coeffs("cube", -1.0, 1.0, n)
    expect = np.zeros(n + 1)
    expect[1] = 0.75
    expect[3] = 0.25
    assert np.max(np.abs(c - expect)) < 1e-15


@pytest.mark.parametrize("k,n", [(0, 5), (2, 5), (5, 5), (7, 12), (12, 12)])
def test_chebyshev_polynomial_gives_unit_vector(O, k, n):
    f = lambda t, p: math.cos(k * math.acos(max(-1.0, min(1.0, t))))
    c = O.cheb_coeffs(f, -1.0, 1.0, n)
    e = np.zeros(n + 1)
    e[k] = 1.0
    assert np.max(np.abs(c - e)) < 1e-14


def _bessel_i(k, x, terms=120):
    # I_k(x) = sum_m (x/2)^(2m+k) / (m! (m+k)!), terms built by their ratio
    h = x / 2.0
    t = 1.0
    for i in range(1, k + 1):
        t *= h / i
    out = []
    for m in range(terms):
        out.append(t)
        t *= h * h / ((m + 1) * (m + 1 + k))
    return math.fsum(out)


@pytest.mark.parametrize("a,b,n", [(-10.0, 10.0, 64), (-10.0, 10.0, 128), (0.5, 6.5, 40)])
def test_exp_matches_bessel_series(O, a, b, n):
    # exp on [a, b]: e^{beta + alpha t} = e^beta [I_0(alpha) + 2 sum_k I_k(alpha) T_k(t)],
    # alpha = (b-a)/2, beta = (a+b)/2; aliasing is below 1e-16 relative for n >= 2 alpha + 20
    alpha, beta = (b - a) / 2.0, (a + b) / 2.0
    c = O.cheb_coeffs("exp", a, b, n)
    exact = np.array([(1.0 if k == 0 else 2.0) * math.exp(beta) * _bessel_i(k, alpha)
                      for k in range(n + 1)])
    scale = np.sum(np.abs(exact))
    assert np.max(np.abs(c - exact)) < 2e-15 * scale
    # the power series itself agrees with the library's modified Bessel function
    sp = pytest.importorskip("scipy.special")
    assert abs(_bessel_i(3, alpha) - sp.iv(3, alpha)) < 1e-13 * sp.iv(3, alpha)


@pytest.mark.parametrize("fn,a,b,n", [("log", 0.1, 8.1, 128), ("sqrt", 0.01, 4.0, 50),
                                       ("inv", 1.0, 3.0, 30), ("exp", -2.0, 3.0, 25)])
def test_interpolates_at_nodes(O, fn, a, b, n):
    c = O.cheb_coeffs(fn, a, b, n)
    f = O.FUNCTIONS[fn]
    for j in range(n + 1):
        x = math.cos(j * math.pi / n)
        t = 0.5 * ((b - a) * x + (a + b))
        assert abs(O.cheb_eval(c, x) - f(t, 0.0)) < 1e-12 * max(1.0, abs(f(t, 0.0)))


def test_log_converges_geometrically(O):
    # log is analytic on [0.1, 8.1]; max error of p_n on a fine grid falls with n
    xs = np.linspace(-1, 1, 2001)
    t = 0.5 * (8.0 * xs + 8.2)
    errs = []
    for n in (16, 32, 64, 128):
        c = O.cheb_coeffs("log", 0.1, 8.1, n)
        errs.append(np.max(np.abs(O.cheb_eval(c, xs) - np.log(t))))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-7
