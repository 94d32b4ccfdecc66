"""GPU parity of the Chebyshev moment engine (mlt_moments) against the CPU
oracle on the same seeded probes.  Tolerance: |mu_gpu - mu_oracle| <= 1e-10 * d
for FP64 (|mu_j| <= d, so this is 1e-10 relative to the largest possible
moment); FP32 vectors use a bound derived from single-precision rounding."""
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


def _c1_degrees():
    # the 64x64 log-det workload: 256 probes at degree 8, 64 at 32, 16 at 128
    return np.array([8] * 256 + [32] * 64 + [128] * 16, dtype=np.int32)


def test_c1_logdet_moments_fp64(L, O):
    m = synth.grid_laplacian_2d(64, shift=0.1)
    deg = _c1_degrees()
    with L.Matrix(m) as M:
        got = M.moments(0.1, 8.1, 0, 0, deg)
    ref = O.moments(m, 0.1, 8.1, 0, 0, deg)
    assert got.shape == ref.shape
    err = np.max(np.abs(got - ref))
    assert err <= TOL64 * m.nrows, err
    assert np.all(got[:, 0] == m.nrows)


def test_direct_mode_matches(L, O):
    m = synth.grid_laplacian_2d(20, shift=0.1)
    deg = np.array([0, 1, 2, 3, 17, 40, 41, 5] * 5, dtype=np.int32)
    with L.Matrix(m) as M:
        got = M.moments(0.1, 8.1, 7, 100, deg, flags=L.MLT_DIRECT)
        dbl = M.moments(0.1, 8.1, 7, 100, deg)
    ref = O.moments(m, 0.1, 8.1, 7, 100, deg)
    assert np.max(np.abs(got - ref)) <= TOL64 * m.nrows
    assert np.max(np.abs(dbl - ref)) <= TOL64 * m.nrows


@pytest.mark.parametrize("nprobes", [1, 5, 37, 130])
def test_ragged_random_degrees(L, O, nprobes):
    rng = np.random.default_rng(nprobes)
    m = synth.random_symmetric(300, 0.02, seed=nprobes, diag_shift=0.0)
    lo, hi = O.gershgorin(m)
    deg = rng.integers(0, 70, size=nprobes).astype(np.int32)
    with L.Matrix(m) as M:
        got = M.moments(lo, hi, 11, 3, deg)
    ref = O.moments(m, lo, hi, 11, 3, deg)
    assert np.max(np.abs(got - ref)) <= TOL64 * m.nrows


def test_many_groups(L, O):
    # more probes than one group holds: groups are formed and results land in
    # the caller's order
    m = synth.grid_laplacian_2d(8, shift=0.5)
    deg = (np.arange(2100) % 23).astype(np.int32)
    with L.Matrix(m) as M:
        got = M.moments(0.5, 8.5, 1, 0, deg)
    ref = O.moments(m, 0.5, 8.5, 1, 0, deg)
    assert np.max(np.abs(got - ref)) <= TOL64 * m.nrows


def test_gram_operator(L, O):
    X = synth.sparse_gaussian(700, 240, 0.02, seed=3)
    deg = np.array([64] * 20 + [9] * 13, dtype=np.int32)
    a, b = O.interval(X, gram=True)          # host interval: no oracle input from the GPU
    with L.Matrix(X, gram=True) as M:
        ga, gb = M.bounds()
        assert ga == 0.0 and gb > 0
        got = M.moments(a, b, 5, 0, deg)
    ref = O.moments(X, a, b, 5, 0, deg, gram=True)
    assert np.max(np.abs(got - ref)) <= TOL64 * 240


def test_pattern_with_scale(L, O):
    g = synth.rmat_adjacency(10, 8, seed=2)
    sc = 0.05
    a, b = O.interval(g, scale=sc)
    with L.Matrix(g, scale=sc) as M:
        ga, gb = M.bounds()                   # the library's Gershgorin interval, checked
        got = M.moments(a, b, 4, 9, [30] * 40)
    assert abs(ga - a) < 1e-12 and abs(gb - b) < 1e-12
    ref = O.moments(g, a, b, 4, 9, [30] * 40, scale=sc)
    assert np.max(np.abs(got - ref)) <= TOL64 * g.nrows


def test_fp32_values_input(L, O):
    m = synth.grid_laplacian_2d(12, shift=0.1)
    with L.Matrix(m, vals_dtype=np.float32) as M:
        got = M.moments(0.1, 8.1, 0, 0, [20] * 9)
    # the oracle sees the FP32-rounded entries (4.1 is not exact in FP32)
    m32 = synth.CSR(m.nrows, m.ncols, m.rowptr, m.col, m.val.astype(np.float32).astype(np.float64))
    ref = O.moments(m32, 0.1, 8.1, 0, 0, [20] * 9)
    assert np.max(np.abs(got - ref)) <= TOL64 * m.nrows


def test_fp32_precision_mode(L, O):
    # FP32 vectors: each step adds relative rounding ~2^-24 to V; the doubled
    # moments carry |2 V_k.V_k| <= 2d, so after k steps the error stays below
    # ~ k * 2^-24 * 2d * (a small growth factor); 64 * eps32 * d bounds degree <= 128.
    m = synth.grid_laplacian_2d(64, shift=0.1)
    deg = _c1_degrees()
    with L.Matrix(m) as M:
        got = M.moments(0.1, 8.1, 0, 0, deg, precision="fp32")
    ref = O.moments(m, 0.1, 8.1, 0, 0, deg)
    err = np.max(np.abs(got - ref))
    assert err <= 64 * 2.0 ** -24 * m.nrows, err


def test_device_output_and_extra_columns(L, O):
    import torch
    m = synth.grid_laplacian_2d(10, shift=0.1)
    deg = np.array([5, 0, 9], dtype=np.int32)
    out = torch.full((3, 14), 7.0, dtype=torch.float64, device="cuda")
    host = np.full((3, 14), 7.0)
    with L.Matrix(m) as M:
        M.moments(0.1, 8.1, 2, 0, deg, out=out)
        M.moments(0.1, 8.1, 2, 0, deg, out=host)
    dev = out.cpu().numpy()
    assert np.array_equal(dev, host)
    ref = O.moments(m, 0.1, 8.1, 2, 0, deg)
    assert np.max(np.abs(host[:, :10] - ref)) <= TOL64 * m.nrows
    assert np.all(host[:, 10:] == 0.0) and host[1, 1] == 0.0 and host[0, 6] == 0.0


def test_degenerate_inputs(L, O):
    m = synth.grid_laplacian_2d(4, shift=0.1)
    with L.Matrix(m) as M:
        z = M.moments(0.1, 8.1, 0, 0, np.zeros(0, dtype=np.int32))
        assert z.shape[0] == 0
        zero = M.moments(0.1, 8.1, 0, 0, [0, 0])
        assert np.all(zero == 16.0)
        with pytest.raises(L.MLTError) as e:
            M.moments(1.0, 1.0, 0, 0, [3])
        assert e.value.code == L.MLT_EINVAL
        with pytest.raises(L.MLTError) as e:
            M.moments(0.1, 8.1, 0, 0, [-1])
        assert e.value.code == L.MLT_EINVAL
        with pytest.raises(L.MLTError) as e:     # spectrum far outside [a, b]
            M.moments(0.1, 0.2, 0, 0, [40])
        assert e.value.code == L.MLT_ERANGE
    # a 1x1 matrix and a matrix with empty rows
    one = synth.CSR(1, 1, np.array([0, 1]), np.array([0]), np.array([2.0]))
    with L.Matrix(one) as M:
        got = M.moments(1.0, 3.0, 0, 0, [6])
    assert np.max(np.abs(got - O.moments(one, 1.0, 3.0, 0, 0, [6]))) <= 1e-12
    e = synth.CSR(5, 5, np.array([0, 1, 1, 1, 2, 2]), np.array([0, 3]), np.array([1.0, 0.5]))
    with L.Matrix(e) as M:
        got = M.moments(-1.0, 1.5, 3, 0, [7, 3])
    assert np.max(np.abs(got - O.moments(e, -1.0, 1.5, 3, 0, [7, 3]))) <= 1e-12


def test_rejects_malformed_csr(L):
    rp = np.array([0, 2, 3], dtype=np.int64)
    for col in (np.array([0, 5, 1], dtype=np.int32),      # column out of range
                np.array([1, 0, 1], dtype=np.int32),      # not increasing in a row
                np.array([1, 1, 0], dtype=np.int32)):     # duplicate
        with pytest.raises(L.MLTError) as e:
            L.mlt_create_csr(2, 2, 3, rp, col, np.ones(3))
        assert e.value.code == L.MLT_EINVAL
    with pytest.raises(L.MLTError) as e:                 # rowptr not monotone
        L.mlt_create_csr(2, 2, 3, np.array([0, 4, 3], dtype=np.int64),
                         np.array([0, 1, 0], dtype=np.int32), np.ones(3))
    assert e.value.code == L.MLT_EINVAL


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("fp32", 64 * 2.0 ** -24), ("df64", TOL64)])
def test_long_rows_in_segments(L, O, precision, tol):
    # every row of K_300 is longer than a work chunk: segment products are
    # added in order by the second kernel
    g = synth.complete_graph(300)
    a, b = O.interval(g, scale=1.0 / 300)
    with L.Matrix(g, scale=1.0 / 300) as M:
        got = M.moments(a, b, 6, 0, [25, 10, 3], precision=precision)
    ref = O.moments(g, a, b, 6, 0, [25, 10, 3], scale=1.0 / 300)
    assert np.max(np.abs(got - ref)) <= tol * g.nrows


def test_reproducible_bits(L):
    g = synth.rmat_adjacency(12, 16, seed=4)
    with L.Matrix(g, scale=0.01) as M:
        a, b = M.bounds()
        r1 = M.moments(a, b, 1, 0, [40] * 70)
        r2 = M.moments(a, b, 1, 0, [40] * 70)
    assert np.array_equal(r1, r2)


@pytest.mark.parametrize("make,gram,sc", [
    (lambda: synth.grid_laplacian_2d(30, shift=0.1), False, 1.0),
    (lambda: synth.random_symmetric(400, 0.02, seed=3), False, 1.0),
    (lambda: synth.rmat_adjacency(11, 8, seed=2), False, 0.1),
    (lambda: synth.sparse_gaussian(600, 200, 0.03, seed=1), True, 1.0)])
def test_lanczos_interval_contains_spectrum(L, make, gram, sc):
    m = make()
    A = m.to_dense() * sc
    if gram:
        A = A.T @ A
    lam = np.linalg.eigvalsh(A)
    with L.Matrix(m, gram=gram, scale=sc) as M:
        a, b = L.mlt_spectrum_bounds(M.handle, L.MLT_BOUNDS_LANCZOS, 60, 1)
        ga, gb = M.bounds()
    assert a <= lam[0] and b >= lam[-1]
    # close at the top: Ritz value + residual, widened by 1%
    assert b <= lam[-1] + 0.05 * abs(lam[-1]) + 1e-9


def test_mixed_precision_switch(L, O):
    # FP32 for the first 16 steps (moments up to degree 32), FP64 after
    m = synth.grid_laplacian_2d(64, shift=0.1)
    deg = _c1_degrees()
    with L.Matrix(m) as M:
        f32 = M.moments(0.1, 8.1, 0, 0, deg, precision="fp32")
        mix = M.moments(0.1, 8.1, 0, 0, deg, precision=L.mixed_at(16))
    ref = O.moments(m, 0.1, 8.1, 0, 0, deg)
    assert np.array_equal(mix[:, :33], f32[:, :33])      # same FP32 steps, same bits
    assert np.max(np.abs(mix - ref)) <= 64 * 2.0 ** -24 * m.nrows
    # past the switch the drift no longer grows as in the all-FP32 run
    hi = slice(100, 129)
    assert np.max(np.abs(mix[:, hi] - ref[:, hi])) <= np.max(np.abs(f32[:, hi] - ref[:, hi])) + 1e-9


def test_batched_graph_matches_single_calls(L, O):
    # uneven matrices with ragged degrees in one graph launch; each job's
    # results equal the oracle's (and the single-call path's)
    mats = [synth.diffusion_3d(s, sigma=1.0, shift=0.05 * (i + 1), seed=i) for i, s in enumerate((4, 7, 10, 5))]
    handles = [L.Matrix(m) for m in mats]
    rng = np.random.default_rng(3)
    jobs, refs = [], []
    for i, (m, h) in enumerate(zip(mats, handles)):
        lo, hi = O.gershgorin(m)
        deg = rng.integers(0, 40, size=10 + 7 * i).astype(np.int32)
        out = np.zeros((deg.size, 40))
        jobs.append({"matrix": h.handle, "a": lo, "b": hi, "seed": i, "probe_offset": 100 * i,
                     "degrees": deg, "out": out})
        refs.append(O.moments(m, lo, hi, i, 100 * i, deg))
    L.mlt_moments_batched(jobs)
    for j, ref, m in zip(jobs, refs, mats):
        assert np.max(np.abs(j["out"][:, :ref.shape[1]] - ref)) <= TOL64 * m.nrows
    single = handles[2].moments(jobs[2]["a"], jobs[2]["b"], 2, 200, jobs[2]["degrees"], out=np.zeros((24, 40)))
    assert np.array_equal(single, jobs[2]["out"])
    with pytest.raises(L.MLTError):
        L.mlt_moments_batched([jobs[0], dict(jobs[0])])     # same handle twice
    for h in handles:
        h.close()


def test_autotune_picks_a_width(L, O):
    m = synth.grid_laplacian_2d(40, shift=0.1)
    with L.Matrix(m) as M:
        w = L.mlt_autotune(M.handle, "fp64", 4)
        assert w in (8, 16, 32, 64, 128)
        got = M.moments(0.1, 8.1, 0, 0, [12] * 50)
    assert np.max(np.abs(got - O.moments(m, 0.1, 8.1, 0, 0, [12] * 50))) <= TOL64 * m.nrows


# Double-float vectors (about 48 significant bits) keep the FP64 tolerance:
# their rounding, ~2^-47 of each value per operation over at most a few
# hundred steps, stays orders of magnitude below 1e-10 * d.
def test_df64_matches_fp64_tolerance(L, O):
    m = synth.grid_laplacian_2d(64, shift=0.1)
    deg = _c1_degrees()
    with L.Matrix(m) as M:
        got = M.moments(0.1, 8.1, 0, 0, deg, precision="df64")
        direct = M.moments(0.1, 8.1, 0, 0, deg[:40], precision="df64", flags=L.MLT_DIRECT)
    ref = O.moments(m, 0.1, 8.1, 0, 0, deg)
    assert np.max(np.abs(got - ref)) <= TOL64 * m.nrows
    assert np.max(np.abs(direct - ref[:40, :direct.shape[1]])) <= TOL64 * m.nrows
    assert np.all(got[:, 0] == m.nrows)
    g = synth.rmat_adjacency(12, 16, seed=2)      # pattern, scaled, hub rows in segments
    sc = 0.02
    a, b = O.interval(g, scale=sc)
    with L.Matrix(g, scale=sc) as M:
        got = M.moments(a, b, 4, 9, [128] * 40 + [17] * 9, precision="df64")
    ref = O.moments(g, a, b, 4, 9, [128] * 40 + [17] * 9, scale=sc)
    assert np.max(np.abs(got - ref)) <= TOL64 * g.nrows
    X = synth.sparse_gaussian(700, 240, 0.02, seed=3)   # Gram operator, FP64 values as pairs
    deg = np.array([64] * 20 + [9] * 13, dtype=np.int32)
    a, b = O.interval(X, gram=True)
    with L.Matrix(X, gram=True) as M:
        got = M.moments(a, b, 5, 0, deg, precision="df64")
    ref = O.moments(X, a, b, 5, 0, deg, gram=True)
    assert np.max(np.abs(got - ref)) <= TOL64 * 240


def test_df64_mlmc_matches_oracle(L, O):
    m = synth.grid_laplacian_2d(64, shift=0.1)
    ref = O.mlmc_fixed(m, "log", 0.1, 8.1, 128, [8, 32, 128], [256, 64, 16], seed=0)
    with L.Matrix(m) as M:
        got = M.mlmc("log", 0.1, 8.1, 128, seed=0, levels=[8, 32, 128], m=[256, 64, 16], precision="df64")
    assert abs(got["estimate"] - ref["estimate"]) <= 1e-10 * np.sum(np.abs(ref["coeffs"])) * m.nrows


def test_direct_mode_fp32_and_df64(L, O):
    # direct mode reads and writes single columns of the dot slots (FP32 slots
    # hold column pairs packed); ragged degrees retire probes step by step
    m = synth.grid_laplacian_2d(20, shift=0.1)
    deg = np.array([0, 1, 2, 3, 17, 40, 41, 5, 6] * 5, dtype=np.int32)
    ref = O.moments(m, 0.1, 8.1, 7, 100, deg)
    with L.Matrix(m) as M:
        f32 = M.moments(0.1, 8.1, 7, 100, deg, precision="fp32", flags=L.MLT_DIRECT)
        df = M.moments(0.1, 8.1, 7, 100, deg, precision="df64", flags=L.MLT_DIRECT)
    assert np.max(np.abs(f32 - ref)) <= 64 * 2.0 ** -24 * m.nrows
    assert np.max(np.abs(df - ref)) <= TOL64 * m.nrows


@pytest.mark.parametrize("nprobes", [1, 3, 9, 33, 64, 129])
@pytest.mark.parametrize("pattern", [False, True])
def test_fp32_group_widths_short_and_long_rows(L, O, nprobes, pattern):
    # FP32 lane groups of 1 to 32 lanes (1 to 129 live probes): groups of at
    # least eight lanes gather in predicated blocks of eight, narrower ones in
    # the plain loop.  Rows of 0 to 13 entries (not multiples of the block)
    # plus three hub rows longer than a work chunk, cut into segments.
    rng = np.random.default_rng(nprobes + 1000 * pattern)
    d = 400
    rows, cols = [], []
    for i in range(d):
        k = int(rng.integers(0, 7))
        for j in rng.choice(d, size=k, replace=False):
            if j != i:
                rows += [i, j]
                cols += [j, i]
    for h in (3, 150, 397):
        for j in range(d):
            if j != h:
                rows += [h, j]
                cols += [j, h]
    key = np.unique(np.array(rows, dtype=np.int64) * d + np.array(cols, dtype=np.int64))
    r, c = key // d, key % d
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=d), out=rowptr[1:])
    val = None if pattern else rng.uniform(0.5, 1.5, size=key.size)
    if val is not None:   # symmetric values
        vm = {}
        for t in range(key.size):
            a_, b_ = int(r[t]), int(c[t])
            vm.setdefault((min(a_, b_), max(a_, b_)), val[t])
            val[t] = vm[(min(a_, b_), max(a_, b_))]
    m = synth.CSR(d, d, rowptr, c.astype(np.int32), val)
    sc = 1.0 / 400.0
    a, b = O.interval(m, scale=sc)
    deg = rng.integers(0, 40, size=nprobes).astype(np.int32)
    deg[0] = 39
    with L.Matrix(m, scale=sc) as M:
        got = M.moments(a, b, 5, 17, deg, precision="fp32")
    ref = O.moments(m, a, b, 5, 17, deg, scale=sc)
    assert np.max(np.abs(got - ref)) <= 64 * 2.0 ** -24 * d


@pytest.mark.parametrize("precision,tol", [("fp32", 64 * 2.0 ** -24), ("df64", TOL64)])
def test_relabelled_graph_window_ordered_segments(L, O, precision, tol):
    # a power-law graph relabelled by degree, with hub rows cut into segments
    # that are dealt out in column-window order; the order must not change the
    # moments beyond rounding
    g = synth.rmat_adjacency(12, 16, seed=7)
    sc = 10.0 / float(np.max(np.diff(g.rowptr)))
    deg = np.array([33, 20, 7, 2] * 10, dtype=np.int32)
    with L.Matrix(g, scale=sc, reorder=True) as M:
        got = M.moments(-10.0, 10.0, 9, 4, deg, precision=precision)
        again = M.moments(-10.0, 10.0, 9, 4, deg, precision=precision)
    ref = O.moments(g, -10.0, 10.0, 9, 4, deg, scale=sc)
    assert np.array_equal(got, again)
    assert np.max(np.abs(got - ref)) <= tol * g.nrows
