"""Pins of the oracle's multilevel machinery: level bands (Eqs. def:qlevels,
decomposition), level selection (Theorem levels, Eq. costrecurrence, the top-level
sample constraint of Section 3.2.1), sample allocation (Eqs. optSamples, optMu,
totalCost) and the multilevel estimator (Eq. multiEstimator)."""
import itertools
import math

import numpy as np
import pytest

from paper_2103_10516_gb300 import synth


def test_bands_sum_to_quadratic_form(O):
    m = synth.grid_laplacian_2d(10, shift=0.1)
    n = 40
    c = O.cheb_coeffs("log", 0.1, 8.1, n)
    mu = O.moments(m, 0.1, 8.1, 0, 0, [n] * 3)
    for levels in ([n], [0, n], [3, 9, 27, n], list(range(0, n + 1))):
        lo = -1
        tot = np.zeros(3)
        for hi in levels:
            tot += O.band(c, mu, lo, hi)
            lo = hi
        assert np.allclose(tot, mu @ c, rtol=0, atol=1e-12 * np.sum(np.abs(c)) * 100)


def test_band_means_exact_under_exhaustive_signs(O):
    # E[Q_{l'l}] = sum_{j=l'+1..l} c_j tr T_j(At): exact over all 2^d sign vectors
    d = 9
    m = synth.random_symmetric(d, 0.5, seed=2, diag_shift=2.0)
    lam = np.linalg.eigvalsh(m.to_dense())
    a, b = lam[0] - 0.3, lam[-1] + 0.3
    n = 10
    c = O.cheb_coeffs("exp", a, b, n)
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=d)))
    mu = O.moments_z(m, a, b, Z, n)
    th = np.arccos((2 * lam - (a + b)) / (b - a))
    tr = [np.sum(np.cos(j * th)) for j in range(n + 1)]
    for lo, hi in ((-1, 2), (2, 5), (5, 10), (-1, 10)):
        exact = sum(c[j] * tr[j] for j in range(lo + 1, hi + 1))
        assert abs(O.band(c, mu, lo, hi).mean() - exact) < 1e-11 * d * np.sum(np.abs(c))


def _path_cost(V, levels, model):
    prev = [0] + levels[:-1]
    return sum(math.sqrt(V[lp, l] * O_cost(l, model)) for lp, l in zip(prev, levels))


def O_cost(l, model):
    return float(l) if model == "linear" else float((l + 1) // 2)


def _random_V(n, rng):
    # a plausible variance table: V[l', l] from random per-term spreads and
    # correlations, so that it is a genuine covariance-derived table
    terms = rng.standard_normal((25, n + 1)) * np.exp(-0.3 * np.arange(n + 1))[None, :]
    V = np.zeros((n + 1, n + 1))
    for lo in range(n):
        for hi in range(lo + 1, n + 1):
            V[lo, hi] = np.var(terms[:, lo + 1: hi + 1].sum(axis=1), ddof=1)
    return V


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("model", ["symmetric", "linear"])
def test_level_dp_matches_brute_force(O, seed, model):
    rng = np.random.default_rng(seed)
    n = 9
    V = _random_V(n, rng)
    levels = O.select_levels(V, model, m_pilot=0)
    best = min(_path_cost(V, list(s) + [n], model)
               for r in range(n) for s in itertools.combinations(range(1, n), r))
    assert levels[-1] == n and levels == sorted(set(levels))
    assert abs(_path_cost(V, levels, model) - best) < 1e-12 * best


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("max_levels", [0, 2, 3])
def test_constrained_dp_matches_brute_force(O, seed, max_levels):
    # the top-level constraint m_L = mu sqrt(V_L / C_L) >= m_pilot, budget mode,
    # mu = budget / sum sqrt(V_k C_k); optionally at most max_levels levels
    rng = np.random.default_rng(100 + seed)
    n = 9
    V = _random_V(n, rng)
    budget = float(rng.uniform(20, 400))
    m_pilot = 5
    levels = O.select_levels(V, "symmetric", m_pilot=m_pilot, mode="budget", target=budget,
                             max_levels=max_levels)
    cands = []
    for r in range(n):
        for s in itertools.combinations(range(1, n), r):
            lv = list(s) + [n]
            if max_levels and len(lv) > max_levels:
                continue
            S = _path_cost(V, lv, "symmetric")
            lp = lv[-2] if len(lv) > 1 else 0
            mL = budget / S * math.sqrt(V[lp, n] / O_cost(n, "symmetric"))
            if mL >= m_pilot:
                cands.append((S, lv))
    if not cands:
        assert levels == [n]
    else:
        best = min(S for S, _ in cands)
        assert abs(_path_cost(V, levels, "symmetric") - best) < 1e-12 * best


def test_allocation_is_kkt_optimal(O):
    # m_k = mu sqrt(V_k / C_k) minimises sum V_k / m_k subject to sum m_k C_k = C
    rng = np.random.default_rng(0)
    n = 30
    V = _random_V(n, rng)
    levels = [2, 7, 15, n]
    budget = 5000.0
    prev = [0] + levels[:-1]
    Vk = np.array([V[lp, l] for lp, l in zip(prev, levels)])
    Ck = np.array([O_cost(l, "symmetric") for l in levels])
    S = np.sum(np.sqrt(Vk * Ck))
    mstar = budget / S * np.sqrt(Vk / Ck)
    assert abs(np.sum(mstar * Ck) - budget) < 1e-9 * budget
    # total-cost identity (Eq. totalCost): variance eps^2 = S^2 / C at the optimum
    assert abs(np.sum(Vk / mstar) - S * S / budget) < 1e-12 * S * S / budget
    f0 = np.sum(Vk / mstar)
    for _ in range(200):
        dm = rng.standard_normal(len(levels))
        dm -= Ck * (dm @ Ck) / (Ck @ Ck)          # stay on the budget plane
        m2 = mstar + 0.05 * mstar.min() * dm / np.max(np.abs(dm))
        assert np.sum(Vk / m2) >= f0 * (1 - 1e-12)
    got = O.allocate(levels, V, "symmetric", "budget", budget)
    assert got == [max(1, math.ceil(v)) for v in mstar]
    # variance mode: mu = eps^-2 S gives variance sum V_k/m_k = eps^2
    eps2 = 1e-3 * S * S / budget
    mv = S / eps2 * np.sqrt(Vk / Ck)
    assert abs(np.sum(Vk / mv) - eps2) < 1e-12 * eps2
    assert O.allocate(levels, V, "symmetric", "variance", eps2) == \
        [max(1, math.ceil(v)) for v in mv]


def test_paper_level_table_arithmetic():
    # Table level_example: 18 levels of a typical nuclear-norm trial; with the
    # cost l per sample the samples add to 15,048 matvecs (caption: 15,070 for a
    # budget of 15,000), consistent with counts rounded up and the top level
    # holding at least m_pilot = 10 samples.
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "level_example.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    levels = [int(r[0]) for r in rows]
    samples = [int(r[1]) for r in rows]
    assert len(levels) == 18 and levels[-1] == 300
    assert sum(l * m for l, m in zip(levels, samples)) == 15048
    assert samples[-1] >= 10


def _c1_logdet_closed_form():
    # eigenvalues of the 64x64 Dirichlet 5-point Laplacian + 0.1 I
    k = np.arange(1, 65)
    e = 2.0 - 2.0 * np.cos(k * np.pi / 65.0)
    lam = (e[:, None] + e[None, :]).ravel() + 0.1
    return lam


def test_c1_closed_form_and_estimate(O):
    m = synth.grid_laplacian_2d(64, shift=0.1)
    assert m.nnz == 20224
    lo, hi = O.gershgorin(m)
    assert abs(lo - 0.1) < 1e-12 and abs(hi - 8.1) < 1e-12
    lam = _c1_logdet_closed_form()
    logdet = float(np.sum(np.log(lam)))
    assert abs(logdet - 5018.30909251356) < 1e-8
    sign, ld = np.linalg.slogdet(m.to_dense())
    assert sign == 1.0 and abs(ld - logdet) < 1e-9 * logdet
    n = 128
    c = O.cheb_coeffs("log", 0.1, 8.1, n)
    trp = float(np.sum(O.cheb_eval(c, (2 * lam - 8.2) / 8.0)))
    assert abs(trp - logdet) < 1e-3            # interpolation error of p_128
    out = O.mlmc_fixed(m, "log", 0.1, 8.1, n, [8, 32, 128], [256, 64, 16], seed=0)
    assert out["m"] == [256, 64, 16]
    assert abs(out["estimate"] - trp) < 5 * out["stderr"]
    # level means telescope to the estimate
    assert abs(sum(out["level_mean"]) - out["estimate"]) < 1e-9


def test_auto_mlmc_consistent(O):
    m = synth.grid_laplacian_2d(16, shift=0.1)
    n = 40
    out = O.mlmc_auto(m, "log", 0.1, 8.1, n, seed=1, m_pilot=10, mode="budget", target=4000.0)
    assert out["levels"][-1] == n
    assert out["m"][-1] >= 10
    spent = sum(mk * O_cost(l, "symmetric") for mk, l in zip(out["m"], out["levels"]))
    assert spent >= 4000.0 - 1e-9 and spent <= 4000.0 + sum(O_cost(l, "symmetric")
                                                             for l in out["levels"])
    lam = np.linalg.eigvalsh(m.to_dense())
    c = O.cheb_coeffs("log", 0.1, 8.1, n)
    trp = float(np.sum(O.cheb_eval(c, (2 * lam - 8.2) / 8.0)))
    assert abs(out["estimate"] - trp) < 5 * out["stderr"]


# ---- exact low-degree traces (closing remark of Section 5.4) -----------------

def _trace_cheb(lam, a, b, j):
    th = np.arccos(np.clip((2 * lam - (a + b)) / (b - a), -1.0, 1.0))
    return float(np.sum(np.cos(j * th)))


@pytest.mark.parametrize("kind", ["values", "pattern_scaled", "gram"])
def test_exact_low_traces_equal_exhaustive_mean_and_eigen(O, kind):
    # t_j must equal both the mean of mu_j over all 2^d sign vectors (which is
    # tr T_j exactly) and sum_i T_j(lambda_i) from a dense eigendecomposition
    gram, scale = False, 1.0
    if kind == "values":
        m = synth.random_symmetric(10, 0.5, seed=4, diag_shift=1.5)
        dense = m.to_dense()
    elif kind == "pattern_scaled":
        m = synth.random_graph(10, 0.4, seed=6)
        scale = 0.7
        dense = scale * m.to_dense()
    else:
        m = synth.sparse_gaussian(7, 9, 0.4, seed=3)
        gram, scale = True, 1.3
        X = scale * m.to_dense()
        dense = X.T @ X
    lam = np.linalg.eigvalsh(dense)
    a, b = lam[0] - 0.5, lam[-1] + 0.5
    t = O.exact_low_traces(m, a, b, gram, scale)
    assert len(t) == (2 if gram else 3)
    dim = dense.shape[0]
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=dim)))
    mu = O.moments_z(m, a, b, Z, 2, gram, scale)
    for j, tj in enumerate(t):
        assert abs(mu[:, j].mean() - tj) <= 1e-12 * dim
        assert abs(_trace_cheb(lam, a, b, j) - tj) <= 1e-10 * dim


def test_low_cv_level_regression_and_fallbacks(O):
    # the fitted control variates: the intercept and residual variance equal
    # the closed-form normal equations (centred 2x2 solve), the residual sum of
    # squares never exceeds the plain one, and the documented fallbacks hold
    rng = np.random.default_rng(0)
    m = 400
    t = [10.0, 0.3, -1.2]
    rows = np.column_stack([np.full(m, 10.0), 0.3 + rng.standard_normal(m), -1.2 + rng.standard_normal(m)])
    q = 5.0 + 2.0 * (rows[:, 1] - 0.3) - 0.7 * (rows[:, 2] + 1.2) + 0.1 * rng.standard_normal(m)
    mean, var = O.low_cv_level(q, rows, t)
    W = rows[:, 1:] - np.array(t[1:])
    Wc, qc = W - W.mean(0), q - q.mean()
    G = Wc.T @ Wc
    r = Wc.T @ qc
    det = G[0, 0] * G[1, 1] - G[0, 1] * G[1, 0]
    a = np.array([G[1, 1] * r[0] - G[0, 1] * r[1], G[0, 0] * r[1] - G[1, 0] * r[0]]) / det
    assert abs(mean - (q.mean() - a @ W.mean(0))) <= 1e-12 * abs(mean)
    res = qc - Wc @ a
    assert abs(var - res @ res / (m - 3)) <= 1e-10 * var
    assert var * (m - 3) <= np.var(q, ddof=1) * (m - 1)
    assert abs(a[0] - 2.0) < 0.05 and abs(a[1] + 0.7) < 0.05
    # fallbacks: degree 0 (no covariate), too few samples, degenerate covariates
    assert O.low_cv_level(q, rows[:, :1], t) == (pytest.approx(q.mean()), pytest.approx(np.var(q, ddof=1)))
    assert O.low_cv_level(q[:3], rows[:3], t)[0] == pytest.approx(q[:3].mean())
    flat = rows.copy()
    flat[:, 2] = -1.2 + 2.0 * (flat[:, 1] - 0.3)       # w_2 = 2 w_1: singular
    assert O.low_cv_level(q, flat, t)[0] == pytest.approx(q.mean())


def test_low_cv_mlmc_unbiased_and_not_worse(O):
    # with the fitted control variates the first level's residual variance never
    # exceeds its plain variance on the same probes, and the estimate stays
    # within a few standard errors of the exact trace (dense eigendecomposition)
    g = synth.random_symmetric(300, 0.05, seed=9, diag_shift=0.5)
    lam = np.linalg.eigvalsh(g.to_dense())
    a, b = lam[0] - 0.3, lam[-1] + 0.3
    c = O.cheb_coeffs("exp", a, b, 12)
    exact = sum(c[j] * _trace_cheb(lam, a, b, j) for j in range(13))
    for seed in (3, 4, 5):
        plain = O.mlmc_fixed(g, "exp", a, b, 12, [4, 12], [200, 50], seed=seed)
        cv = O.mlmc_fixed(g, "exp", a, b, 12, [4, 12], [200, 50], seed=seed, low_cv=True)
        assert cv["level_var"][0] * 197 <= plain["level_var"][0] * 199
        assert abs(cv["estimate"] - exact) < 5 * cv["stderr"]


def test_interval_contains_the_spectrum(O):
    # Gershgorin of scale * A, and [0, s^2 ||X||_1 ||X||_inf] for X^T X: both
    # contain every eigenvalue (dense eigvalsh), and the Gershgorin form is the
    # discs' extreme ends
    cases = [(synth.grid_laplacian_2d(12, shift=0.1), 1.0), (synth.rmat_adjacency(8, 8, seed=2), 0.05),
             (synth.random_symmetric(60, 0.1, seed=4, diag_shift=1.5), -0.5)]
    for m, sc in cases:
        a, b = O.interval(m, scale=sc)
        lam = np.linalg.eigvalsh(sc * m.to_dense())
        assert a <= lam[0] + 1e-12 and lam[-1] <= b + 1e-12
        D = sc * m.to_dense()
        r = np.sum(np.abs(D), axis=1) - np.abs(np.diag(D))
        assert abs(a - np.min(np.diag(D) - r)) < 1e-12 and abs(b - np.max(np.diag(D) + r)) < 1e-12
    X = synth.sparse_gaussian(90, 40, 0.1, seed=6)
    for sc in (1.0, 0.3):
        a, b = O.interval(X, scale=sc, gram=True)
        D = sc * X.to_dense()
        lam = np.linalg.eigvalsh(D.T @ D)
        assert a == 0.0 and lam[-1] <= b
        assert abs(b - np.abs(D).sum(axis=1).max() * np.abs(D).sum(axis=0).max()) < 1e-9 * b


# ---- pilot variances (Section 3.2.1) ----------------------------------------

def _exhaustive_pilot(O, d=6, n=8, seed=4):
    """All 2^d Rademacher vectors as the pilot sample of a small symmetric
    matrix: their moments, the coefficients of exp, and each band's matrix
    B_{lo,hi} = sum_{j=lo+1..hi} c_j T_j(At) from the eigendecomposition, with
    T_j(x) = cos(j arccos x) (no recurrence)."""
    m = synth.random_symmetric(d, 0.6, seed=seed, diag_shift=1.0)
    lam, Q = np.linalg.eigh(m.to_dense())
    a, b = float(lam[0]) - 0.2, float(lam[-1]) + 0.3
    c = O.cheb_coeffs("exp", a, b, n)
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=d)))
    mu = O.moments_z(m, a, b, Z, n)
    th = np.arccos(np.clip((2 * lam - (a + b)) / (b - a), -1, 1))

    def B(lo, hi):
        w = sum(c[j] * np.cos(j * th) for j in range(lo + 1, hi + 1))
        return (Q * w) @ Q.T
    return c, mu, B, Z.shape[0]


def _pilot_pin_error(V, B, N, n):
    """Largest relative gap between V[lo, hi] and the exact sample variance of
    z^T B z over all N = 2^d sign vectors: the Hutchinson variance
    2 (||B||_F^2 - sum_i B_ii^2) (Rademacher z) times N / (N - 1), since the
    sample variance divides by N - 1.  Entries with lo >= hi must be 0."""
    worst = 0.0
    for lo in range(n + 1):
        for hi in range(n + 1):
            if lo >= hi:
                if V[lo, hi] != 0.0:
                    return float("inf")
                continue
            Bm = B(lo, hi)
            exact = 2.0 * (np.sum(Bm * Bm) - np.sum(np.diag(Bm) ** 2)) * N / (N - 1)
            worst = max(worst, abs(V[lo, hi] - exact) / max(exact, 1e-300))
    return worst


def test_pilot_variances_exhaustive_closed_form(O):
    n = 8
    c, mu, B, N = _exhaustive_pilot(O, n=n)
    V = O.pilot_variances(c, mu)
    assert V.shape == (n + 1, n + 1)
    assert _pilot_pin_error(V, B, N, n) < 1e-9


def test_pilot_variance_pin_rejects_planted_mistakes(O):
    """The closed-form pin is sharp enough to catch the plausible slips of a
    pilot-variance routine: divisor m instead of m - 1, a band shifted by one
    term, the transposed table, and a band that starts at its own lower level."""
    n = 8
    c, mu, B, N = _exhaustive_pilot(O, n=n)
    terms = np.asarray(c)[None, :] * mu[:, : n + 1]

    def table(lo_off, hi_off, ddof, transpose=False):
        V = np.zeros((n + 1, n + 1))
        for lo in range(n):
            for hi in range(lo + 1, n + 1):
                q = terms[:, lo + lo_off: hi + hi_off].sum(axis=1)
                V[lo, hi] = np.var(q, ddof=ddof)
        return V.T.copy() if transpose else V

    assert _pilot_pin_error(table(1, 1, 1), B, N, n) < 1e-9        # the correct form
    for bad in (table(1, 1, 0), table(0, 0, 1), table(2, 1, 1), table(0, 1, 1), table(1, 1, 1, True)):
        assert _pilot_pin_error(bad, B, N, n) > 1e-3


def test_pilot_variances_band_by_band(O):
    """Each entry equals the sample variance (divisor m - 1) of the pinned band
    sums Q_{lo,hi} over the pilot rows (every band summed on its own)."""
    m = synth.grid_laplacian_2d(12, shift=0.1)
    n = 24
    c = O.cheb_coeffs("log", 0.1, 8.1, n)
    mu = O.moments(m, 0.1, 8.1, 9, 40, [n] * 7)
    V = O.pilot_variances(c, mu)
    for lo in range(n):
        for hi in range(lo + 1, n + 1):
            q = O.band(c, mu, lo, hi)
            ref = float(np.var(q, ddof=1))
            assert abs(V[lo, hi] - ref) <= 1e-12 * max(ref, 1e-30) + 1e-28, (lo, hi)
    assert np.all(np.tril(V) == 0.0)
    # a single pilot row has no sample variance: the table is all zeros
    assert np.all(O.pilot_variances(c, mu[:1]) == 0.0)


# ---- the three-level estimator with a learned coarse level -------------------

def test_learned_levels_exact_under_exhaustive_signs(O):
    """With every one of the 2^d sign vectors in each of the three groups, the
    estimate is tr p_n(At) exactly, whatever the network's outputs are (here an
    arbitrary nonlinear function of the features): the network's mean and the
    correction's mean cancel sample by sample."""
    d, n, l1 = 8, 12, 6
    m = synth.random_symmetric(d, 0.5, seed=3, diag_shift=1.0)
    lam = np.linalg.eigvalsh(m.to_dense())
    a, b = float(lam[0]) - 0.3, float(lam[-1]) + 0.2
    c = O.cheb_coeffs("exp", a, b, n)
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=d)))
    N = Z.shape[0]
    mu1 = O.moments_z(m, a, b, Z, n)
    mu = np.vstack([mu1, mu1, mu1])
    s = np.concatenate([np.sin(3 * mu1[:, 1]) + mu1[:, 2] ** 2] * 2)
    got = O.learned_estimate(c, mu, s, N, N, N, l1)
    th = np.arccos((2 * lam - (a + b)) / (b - a))
    exact = sum(c[j] * np.sum(np.cos(j * th)) for j in range(n + 1))
    assert abs(got["estimate"] - exact) < 1e-10 * np.sum(np.abs(c)) * d
    assert got["m"] == [N, N, N]


def test_learned_levels_special_cases(O):
    """S = 0 gives the plain two-level estimator (levels l1, n) plus an exact
    zero level; S equal to each probe's own P_l1 leaves a correction level of
    zero samples, and the estimate is the mean of S plus the top band."""
    m = synth.grid_laplacian_2d(10, shift=0.1)
    n, l1 = 30, 12
    c = O.cheb_coeffs("log", 0.1, 8.1, n)
    m_net, m_1, m_2 = 9, 14, 6
    deg = [l1] * (m_net + m_1) + [n] * m_2
    mu = O.moments(m, 0.1, 8.1, 5, 0, deg)
    zero = O.learned_estimate(c, mu, np.zeros(m_net + m_1), m_net, m_1, m_2, l1)
    plain = O.mlmc_fixed(m, "log", 0.1, 8.1, n, [l1, n], [m_1, m_2], seed=5, probe_offset=m_net)
    assert zero["level_mean"][0] == 0.0 and zero["level_var"][0] == 0.0
    assert abs(zero["estimate"] - plain["estimate"]) < 1e-12 * np.sum(np.abs(c)) * m.nrows
    own = O.band(c, mu[:m_net + m_1], -1, l1)
    exact_net = O.learned_estimate(c, mu, own, m_net, m_1, m_2, l1)
    assert np.all(np.abs(np.asarray(exact_net["level_mean"][1])) < 1e-12 * np.sum(np.abs(c)) * m.nrows)
    assert exact_net["level_var"][1] < 1e-20 * max(1.0, exact_net["level_var"][0])
    top = O.band(c, mu[m_net + m_1:], l1, n)
    assert abs(exact_net["estimate"] - (np.mean(own[:m_net]) + np.mean(top))) < 1e-12 * np.sum(np.abs(c)) * m.nrows
