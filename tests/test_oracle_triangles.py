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
