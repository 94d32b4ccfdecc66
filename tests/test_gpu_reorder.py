"""GPU parity of the relabelled operator (MLT_REORDER): the moment engine runs
on P A P^T with rows in order of decreasing degree and each probe entry taken
at its original row id, so every moment must equal the oracle's moment of the
original operator and probe, within the tolerance of its precision.  Covers a
power-law pattern graph whose hub rows are cut into segments, a valued matrix
with equal degrees (ties keep increasing ids), direct and doubling modes, FP32,
double-float and mixed precision, several probe groups, a multilevel estimate,
and the rejection of a Gram handle."""
import numpy as np
import pytest

from paper_2103_10516_gb300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    from paper_2103_10516_gb300 import build, mlt
    build.build()
    return mlt


@pytest.mark.parametrize("precision,flags,tol", [("fp64", 0, TOL64), ("fp64", 1, TOL64), ("df64", 0, TOL64),
                                                 ("fp32", 0, 64 * 2.0 ** -24)])
def test_reordered_rmat_matches_oracle(L, O, precision, flags, tol):
    g = synth.rmat_adjacency(12, 16, seed=2)           # hubs: rows cut into segments
    sc = 0.02
    a, b = O.interval(g, scale=sc)
    deg = np.array([64] * 40 + [17] * 9 + [0, 1, 2], dtype=np.int32)
    with L.Matrix(g, scale=sc, reorder=True) as M:
        got = M.moments(a, b, 4, 9, deg, precision=precision, flags=flags)
    ref = O.moments(g, a, b, 4, 9, deg, scale=sc)
    assert np.max(np.abs(got - ref)) <= tol * g.nrows
    assert np.all(got[:, 0] == g.nrows)


def test_reordered_valued_and_many_groups(L, O):
    m = synth.random_symmetric(400, 0.03, seed=6, diag_shift=0.5)
    lo, hi = O.gershgorin(m)
    deg = (np.arange(1500) % 29).astype(np.int32)
    with L.Matrix(m, reorder=True) as M:
        got = M.moments(lo, hi, 3, 77, deg)
        mixed = M.moments(lo, hi, 3, 77, deg[:50], precision=L.mixed_at(4))
    ref = O.moments(m, lo, hi, 3, 77, deg)
    assert np.max(np.abs(got - ref)) <= TOL64 * m.nrows
    assert np.max(np.abs(mixed - ref[:50, :mixed.shape[1]])) <= 64 * 2.0 ** -24 * m.nrows
    grid = synth.grid_laplacian_2d(30, shift=0.1)       # every interior degree equal: ties by id
    with L.Matrix(grid, reorder=True) as M:
        got = M.moments(0.1, 8.1, 1, 0, [40] * 33)
    assert np.max(np.abs(got - O.moments(grid, 0.1, 8.1, 1, 0, [40] * 33))) <= TOL64 * grid.nrows


def test_reordered_mlmc_and_triangles_unchanged(L, O):
    g = synth.rmat_adjacency(11, 16, seed=3)
    sc = 0.03
    a, b = O.interval(g, scale=sc)
    ref = O.mlmc_fixed(g, "exp", a, b, 40, [6, 20, 40], [60, 20, 6], seed=5, scale=sc)
    with L.Matrix(g, scale=sc, reorder=True) as M:
        got = M.mlmc("exp", a, b, 40, seed=5, levels=[6, 20, 40], m=[60, 20, 6])
    assert abs(got["estimate"] - ref["estimate"]) <= 1e-10 * np.sum(np.abs(ref["coeffs"])) * g.nrows
    # the triangle path keeps the original arrays: its integers are untouched
    x = np.zeros((130, 3), dtype=np.int64)
    with L.Matrix(g, reorder=True) as M:
        L.mlt_triangle_trace(M.handle, 2, 0, 130, x=x)
    assert np.array_equal(x, O.triangle_moments(g, 2, 0, 130))


def test_reorder_rejects_gram(L):
    X = synth.sparse_gaussian(50, 20, 0.1, seed=1)
    with pytest.raises(L.MLTError) as e:
        L.Matrix(X, gram=True, reorder=True)
    assert e.value.code == L.MLT_EINVAL
