"""CPU oracle of the multilevel Chebyshev-Hutchinson trace estimator
(Hallman & Troester, arXiv 2103.10516).

TEST INFRASTRUCTURE ONLY.  The CUDA library is checked against this module; it
is never part of the product path.  Only the test suite, the package smoke check
and the benchmark's CPU-baseline / reference arm may import it.  It shares no
code with the CUDA library: the heavy loops live in ``mlt_oracle.c`` (plain C,
built by ``oracle/build.py``); the host-side method (coefficients, level bands,
pilot variances, level selection, sample allocation, combination, control
variates) is written out here in numpy / plain Python, each function following
the passage it cites.
"""
from __future__ import annotations

import ctypes
import math
import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) the C part of the oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32, u64, dbl, vp = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_void_p)
        L.orc_mix64.argtypes = [u64]
        L.orc_mix64.restype = u64
        L.orc_rademacher.argtypes = [u64, u64, u64]
        L.orc_rademacher.restype = ctypes.c_int
        L.orc_probe.argtypes = [u64, u64, i64, vp]
        L.orc_probe.restype = None
        L.orc_moments.argtypes = [i64, i64, vp, vp, vp, dbl, ctypes.c_int, dbl, dbl, u64,
                                  i64, ctypes.c_int, vp, vp, i64]
        L.orc_moments.restype = ctypes.c_int
        L.orc_moments_z.argtypes = [i64, i64, vp, vp, vp, dbl, ctypes.c_int, dbl, dbl,
                                    ctypes.c_int, vp, vp, vp, i64]
        L.orc_moments_z.restype = ctypes.c_int
        L.orc_triangle_moments.argtypes = [i64, vp, vp, u64, i64, ctypes.c_int, vp]
        L.orc_triangle_moments.restype = ctypes.c_int
        L.orc_triangle_moments_z.argtypes = [i64, vp, vp, ctypes.c_int, vp, vp]
        L.orc_triangle_moments_z.restype = ctypes.c_int
        L.orc_triangle_count.argtypes = [i64, vp, vp]
        L.orc_triangle_count.restype = i64
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# Probes (Section 2.1: Rademacher vectors, entries +-1 with equal probability)
# ---------------------------------------------------------------------------

def mix64(x: int) -> int:
    return int(lib().orc_mix64(ctypes.c_uint64(x & (2**64 - 1))))


def rademacher(seed: int, p: int, d: int) -> np.ndarray:
    """Probe vector z (int8, +-1) with global probe id p."""
    z = np.empty(d, dtype=np.int8)
    lib().orc_probe(seed, p, d, _ptr(z))
    return z


# ---------------------------------------------------------------------------
# Chebyshev moments (Section 2.2, Eq. recurrence)
# ---------------------------------------------------------------------------

def _mat_args(m):
    val = None if m.val is None else np.ascontiguousarray(m.val, dtype=np.float64)
    return val


def moments(m, a, b, seed, probe_offset, degrees, gram=False, scale=1.0):
    """mu[p, j] = z_p^T T_j(At) z_p for j <= degrees[p] (zero beyond), At = g(A).

    A is the square CSR ``m`` (gram=False) or X^T X with X = ``m`` (gram=True);
    z_p is the Rademacher probe with global id probe_offset + p.
    """
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    ld = int(deg.max()) + 1 if deg.size else 1
    mu = np.zeros((deg.size, ld))
    val = _mat_args(m)
    rc = lib().orc_moments(m.nrows, m.ncols, _ptr(m.rowptr), _ptr(m.col), _ptr(val), scale,
                           int(gram), a, b, seed, probe_offset, deg.size, _ptr(deg),
                           _ptr(mu), ld)
    if rc != 0:
        raise MemoryError("oracle moments failed (%d)" % rc)
    return mu


def moments_z(m, a, b, z, degrees, gram=False, scale=1.0):
    """Moments of explicitly given probe vectors z (nprobes x dim)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    if z.ndim == 1:
        z = z[None, :]
    deg = np.ascontiguousarray(np.broadcast_to(degrees, (z.shape[0],)), dtype=np.int32)
    ld = int(deg.max()) + 1
    mu = np.zeros((z.shape[0], ld))
    val = _mat_args(m)
    rc = lib().orc_moments_z(m.nrows, m.ncols, _ptr(m.rowptr), _ptr(m.col), _ptr(val), scale,
                             int(gram), a, b, z.shape[0], _ptr(z), _ptr(deg), _ptr(mu), ld)
    if rc != 0:
        raise MemoryError("oracle moments failed (%d)" % rc)
    return mu


# ---------------------------------------------------------------------------
# Chebyshev interpolation (Section 2.2, Eq. chebSeries and the node formula)
# ---------------------------------------------------------------------------

FUNCTIONS = {
    "log": lambda t, p: math.log(t),
    "sqrt": lambda t, p: math.sqrt(t),
    "exp": lambda t, p: math.exp(t),
    "inv": lambda t, p: 1.0 / t,
    "pow": lambda t, p: t ** p,
    "cube": lambda t, p: t * t * t,
}


def cheb_coeffs(fn, a, b, n, p=0.0):
    """c_0..c_n of the degree-n interpolant of f~ = f o g^{-1} on [-1, 1] at the
    extrema nodes x_j = cos(j pi / n), g the affine map [a, b] -> [-1, 1].

    Written as the direct cosine sum (the FFT of the paper is only a speed-up):
        c_k = (2/n) sum''_{j=0..n} f~(x_j) cos(j k pi / n),
    where sum'' halves the j = 0 and j = n terms, and c_0, c_n are halved.
    """
    if n < 1:
        raise ValueError("n >= 1")
    f = FUNCTIONS[fn] if isinstance(fn, str) else fn
    fx = []
    for j in range(n + 1):
        x = math.cos(j * math.pi / n)
        t = 0.5 * ((b - a) * x + (a + b))
        fx.append(f(t, p))
    c = np.zeros(n + 1)
    for k in range(n + 1):
        terms = []
        for j in range(n + 1):
            w = 0.5 if j in (0, n) else 1.0
            r = (j * k) % (2 * n)
            terms.append(w * fx[j] * math.cos(r * math.pi / n))
        ck = 2.0 / n * math.fsum(terms)
        if k in (0, n):
            ck *= 0.5
        c[k] = ck
    return c


def cheb_eval(c, x):
    """p_n(x) = sum_j c_j T_j(x) with T_j(x) = cos(j arccos x) for |x| <= 1."""
    x = np.asarray(x, dtype=np.float64)
    th = np.arccos(np.clip(x, -1.0, 1.0))
    return sum(c[j] * np.cos(j * th) for j in range(len(c)))


# ---------------------------------------------------------------------------
# Multilevel estimator (Section 3, Eqs. def:qlevels, decomposition;
# Section 4, Eq. multiEstimator)
# ---------------------------------------------------------------------------

def band(c, mu, lo, hi):
    """Q_{lo,hi} = sum_{j=lo+1..hi} c_j mu_j for every probe row of mu."""
    mu = np.atleast_2d(mu)
    return np.array([math.fsum(c[j] * row[j] for j in range(lo + 1, hi + 1)) for row in mu])


def cost(l, model="symmetric"):
    """Section 3.1: cost of a sample of Q_{l'l} is l matvecs, or ceil(l/2) when the
    symmetry of the quadratic form is exploited."""
    return float(l) if model == "linear" else float((l + 1) // 2)


def pilot_variances(c, mu_pilot):
    """Section 3.2.1: V[l', l] = sample variance (divisor m_pilot - 1) of Q_{l'l}
    over the pilot probes, for 0 <= l' < l <= n.  Entry [l', l] for l' >= l is 0."""
    mu_pilot = np.atleast_2d(mu_pilot)
    n = len(c) - 1
    m = mu_pilot.shape[0]
    terms = np.asarray(c)[None, :] * mu_pilot[:, : n + 1]   # c_j mu_j per pilot probe
    V = np.zeros((n + 1, n + 1))
    for lo in range(0, n):
        for hi in range(lo + 1, n + 1):
            q = terms[:, lo + 1: hi + 1].sum(axis=1)
            V[lo, hi] = float(np.var(q, ddof=1)) if m > 1 else 0.0
    return V


def _mu_factor(S, mode, target):
    """Eq. optMu (variance mode, target = eps^2) or the budget form (target = C)."""
    if S <= 0.0:
        return 0.0
    return S / target if mode == "variance" else target / S


def select_levels(V, cost_model="symmetric", m_pilot=0, mode="budget", target=1.0,
                  max_levels=0):
    """Level selection by the dynamic programme of Theorem levels:
        C_0 = 0,   C_l = min_{0 <= l' < l} C_{l'} + sqrt(V_{l'l} C_{l'l}),
    with, at l = n, only predecessors whose complete path recommends at least
    m_pilot samples for the top level (Section 3.2.1).  With max_levels > 0 the
    programme is layered by the number of levels on the path.  Ties go to the
    smaller l'.  Returns the level list [l_1, ..., l_L = n]."""
    n = V.shape[0] - 1
    Lmax = max_levels if max_levels > 0 else n
    INF = float("inf")
    # best[t][l]: minimal sum of sqrt(V C) over paths 0 -> l using exactly t levels
    best = [[INF] * (n + 1) for _ in range(Lmax + 1)]
    arg = [[-1] * (n + 1) for _ in range(Lmax + 1)]
    best[0][0] = 0.0
    if max_levels <= 0:
        # plain recurrence of Theorem levels (number of levels unconstrained)
        Cl = [INF] * (n + 1)
        Cl[0] = 0.0
        pred = [-1] * (n + 1)
        for l in range(1, n):
            for lp in range(0, l):
                v = Cl[lp] + math.sqrt(V[lp, l] * cost(l, cost_model))
                if v < Cl[l]:
                    Cl[l] = v
                    pred[l] = lp
        chosen, chosen_S = -1, INF
        for lp in range(0, n):
            w = math.sqrt(V[lp, n] * cost(n, cost_model))
            S = Cl[lp] + w
            if m_pilot > 0 and not _top_ok(S, V[lp, n], cost(n, cost_model), mode, target, m_pilot):
                continue
            if S < chosen_S:
                chosen, chosen_S = lp, S
        if chosen < 0:
            return [n]
        levels = [n]
        l = chosen
        while l > 0:
            levels.append(l)
            l = pred[l]
        return levels[::-1]
    for t in range(1, Lmax + 1):
        for l in range(1, n):
            for lp in range(0, l):
                if best[t - 1][lp] == INF:
                    continue
                v = best[t - 1][lp] + math.sqrt(V[lp, l] * cost(l, cost_model))
                if v < best[t][l]:
                    best[t][l] = v
                    arg[t][l] = lp
    chosen, chosen_t, chosen_S = -1, -1, INF
    for t in range(1, Lmax + 1):
        for lp in range(0, n):
            if best[t - 1][lp] == INF:
                continue
            S = best[t - 1][lp] + math.sqrt(V[lp, n] * cost(n, cost_model))
            if m_pilot > 0 and not _top_ok(S, V[lp, n], cost(n, cost_model), mode, target, m_pilot):
                continue
            if S < chosen_S:
                chosen, chosen_t, chosen_S = lp, t, S
    if chosen < 0:
        return [n]
    levels = [n]
    l, t = chosen, chosen_t - 1
    while l > 0:
        levels.append(l)
        l, t = arg[t][l], t - 1
    return levels[::-1]


def _top_ok(S, Vtop, Ctop, mode, target, m_pilot):
    """Does the path with total S recommend m_L = mu sqrt(V/C) >= m_pilot?"""
    mu = _mu_factor(S, mode, target)
    return mu * math.sqrt(Vtop / Ctop) >= m_pilot


def allocate(levels, V, cost_model="symmetric", mode="budget", target=1.0, m_pilot=0):
    """Eqs. optSamples / optMu: m_k = mu sqrt(V_k / C_k), rounded up, at least 1
    (at least m_pilot for the top level when the pilot is reused)."""
    prev = [0] + list(levels[:-1])
    Vk = [V[lp, l] for lp, l in zip(prev, levels)]
    Ck = [cost(l, cost_model) for l in levels]
    S = math.fsum(math.sqrt(v * cc) for v, cc in zip(Vk, Ck))
    mu = _mu_factor(S, mode, target)
    m = []
    for v, cc in zip(Vk, Ck):
        m.append(max(1, int(math.ceil(mu * math.sqrt(v / cc)))))
    if m_pilot > 0:
        m[-1] = max(m[-1], m_pilot)
    return m


def exact_low_traces(m, a, b, gram=False, scale=1.0):
    """tr T_j(At) for the low degrees whose traces are cheap to get exactly
    (the closing remark of Section 5.4), At = alpha A + beta I with
    alpha = 2/(b-a), beta = -(a+b)/(b-a) (Section 2.2):
      j = 0:  tr I = d
      j = 1:  tr At = alpha tr A + beta d
      j = 2:  tr(2 At^2 - I) = 2 (alpha^2 tr A^2 + 2 alpha beta tr A + beta^2 d) - d,
              with tr A^2 = ||A||_F^2 for symmetric A.
    For A = X^T X only j <= 1 (tr X^T X = ||X||_F^2; tr (X^T X)^2 would need the
    product).  Every entry counts `scale` times its value (a pattern entry is 1);
    X^T X scales by scale^2.  Sums are exact-rounded (math.fsum)."""
    alpha = 2.0 / (b - a)
    beta = -(a + b) / (b - a)
    v = np.ones(m.nnz) if m.val is None else np.asarray(m.val, dtype=np.float64)
    sq = math.fsum((v * v).tolist())
    if gram:
        d = float(m.ncols)
        return [d, alpha * (scale * scale * sq) + beta * d]
    d = float(m.nrows)
    rows = np.repeat(np.arange(m.nrows), np.diff(m.rowptr))
    tr_a = scale * math.fsum(v[rows == np.asarray(m.col)].tolist())
    tr_a2 = scale * scale * sq
    return [d, alpha * tr_a + beta * d, 2.0 * (alpha * alpha * tr_a2 + 2.0 * alpha * beta * tr_a + beta * beta * d) - d]


def low_cv_level(q, rows, t):
    """One level's mean and variance with the low-degree terms as control
    variates (Section 5.4, applied to the bands as its closing remark
    suggests): w_j = mu_j - tr T_j(At) for 1 <= j <= J has mean zero
    (J = 2, or 1 for X^T X, and at most the level's degree), the band samples
    q are regressed on (1, w) by least squares, and the level's estimate is the
    intercept mean(q) - a . mean(w) with the residual variance (divisor
    m - 1 - J).  Reusing the samples for the fit adds an O(1/m) bias, as in the
    triangle estimator.  The fit is skipped (plain mean and variance) when
    m <= J + 1 or when the centred covariates are degenerate:
    det(W^T W) <= 1e-12 * prod(diag(W^T W)) (J = 2), or W^T W <= 0 (J = 1)."""
    m = q.size
    J = min(len(t) - 1, rows.shape[1] - 1)
    plain = (math.fsum(q) / m, float(np.var(q, ddof=1)) if m > 1 else float("nan"))
    if J < 1 or m <= J + 1:
        return plain
    W = rows[:, 1:J + 1] - np.asarray(t[1:J + 1])
    Wc = W - W.mean(axis=0)
    qc = q - q.mean()
    G = Wc.T @ Wc
    if J == 2:
        if not (G[0, 0] * G[1, 1] - G[0, 1] ** 2 > 1e-12 * G[0, 0] * G[1, 1]):
            return plain
    elif not (G[0, 0] > 0.0):
        return plain
    coef, *_ = np.linalg.lstsq(np.column_stack([np.ones(m), W]), q, rcond=None)
    res = q - np.column_stack([np.ones(m), W]) @ coef
    return float(coef[0]), float(math.fsum((res * res).tolist()) / (m - 1 - J))


def mlmc_fixed(m, fn, a, b, n, levels, samples, seed, p=0.0, gram=False, scale=1.0,
               probe_offset=0, low_cv=False):
    """Multilevel estimate with prescribed levels and sample counts (Eq.
    multiEstimator).  Level k draws probes with ids off_k .. off_k + m_k - 1,
    off_1 = probe_offset, off_{k+1} = off_k + m_k; each is run to degree l_k.
    low_cv: every level with the low-degree control variates of low_cv_level."""
    c = cheb_coeffs(fn, a, b, n, p)
    t = exact_low_traces(m, a, b, gram, scale) if low_cv else None
    out = _run_levels(m, c, a, b, levels, samples, [None] * len(levels), seed, gram, scale,
                      probe_offset, t)
    out["coeffs"] = c
    return out


def _run_levels(m, c, a, b, levels, fresh, reuse_rows, seed, gram, scale, offset, t=None):
    est_terms = []
    var_terms = []
    means = []
    variances = []
    counts = []
    lo = -1
    for k, hi in enumerate(levels):
        deg = np.full(fresh[k], hi, dtype=np.int32)
        rows = moments(m, a, b, seed, offset, deg, gram, scale) if fresh[k] > 0 else np.zeros((0, hi + 1))
        offset += fresh[k]
        if reuse_rows[k] is not None:
            rows = np.vstack([reuse_rows[k][:, : hi + 1], rows])
        q = band(c, rows, lo, hi)
        mk = q.size
        if t is not None:
            mean, var = low_cv_level(q, rows[:, : hi + 1], t)
        else:
            mean = math.fsum(q) / mk
            var = float(np.var(q, ddof=1)) if mk > 1 else float("nan")
        means.append(mean)
        variances.append(var)
        counts.append(mk)
        est_terms.append(mean)
        var_terms.append(var / mk)
        lo = hi
    return {"estimate": math.fsum(est_terms), "stderr": math.sqrt(math.fsum(var_terms)),
            "levels": list(levels), "m": counts, "level_mean": means, "level_var": variances,
            "next_probe": offset}


def mlmc_auto(m, fn, a, b, n, seed, m_pilot, mode="budget", target=1.0, p=0.0,
              cost_model="symmetric", max_levels=0, gram=False, scale=1.0, reuse_pilot=True,
              low_cv=False):
    """Automatic multilevel estimate (Section 3.2): pilot of m_pilot probes (ids
    0 .. m_pilot-1) at degree n, variances of every band, level selection with the
    top-level constraint, allocation, then fresh probes per level (ids from
    m_pilot on, level by level).  The pilot rows are reused as the first m_pilot
    samples of the top level unless reuse_pilot is False."""
    c = cheb_coeffs(fn, a, b, n, p)
    t = exact_low_traces(m, a, b, gram, scale) if low_cv else None
    mu_p = moments(m, a, b, seed, 0, np.full(m_pilot, n, dtype=np.int32), gram, scale)
    V = pilot_variances(c, mu_p)
    levels = select_levels(V, cost_model, m_pilot if reuse_pilot else 0, mode, target,
                           max_levels)
    counts = allocate(levels, V, cost_model, mode, target, m_pilot if reuse_pilot else 0)
    fresh = list(counts)
    reuse = [None] * len(levels)
    if reuse_pilot:
        fresh[-1] = counts[-1] - m_pilot
        reuse[-1] = mu_p
    out = _run_levels(m, c, a, b, levels, fresh, reuse, seed, gram, scale, m_pilot, t)
    out["coeffs"] = c
    out["pilot_V"] = V
    out["pilot_mu"] = mu_p
    return out


def learned_estimate(c, mu, s, m_net, m_1, m_2, l1):
    """The three-level estimator with a learned coarse level (a project
    addition; Eq. multiEstimator with the network as its lowest level):
    E[P_n] = E[S] + E[P_l1 - S] + E[P_n - P_l1].  mu holds the moment rows of
    m_net, then m_1, then m_2 independent probes (the first two groups to
    degree l1 at least, the last to n = len(c) - 1); s holds the network's
    estimate of P_l1 = sum_{j <= l1} c_j mu_j for the first m_net + m_1 probes.
    Level 1 samples s_i (first group), level 2 P_l1 - s_i (second group),
    level 3 Q_{l1,n} (third group, absent when l1 = n or m_2 = 0).  Each level
    reports its sample mean and variance (divisor m - 1); the estimate is the
    sum of the means and its standard error sqrt(sum var_k / m_k)."""
    n = len(c) - 1
    mu = np.atleast_2d(mu)
    s = np.asarray(s, dtype=np.float64)
    lv = [s[:m_net], band(c, mu[m_net:m_net + m_1], -1, l1) - s[m_net:m_net + m_1]]
    if l1 < n and m_2 > 0:
        lv.append(band(c, mu[m_net + m_1:m_net + m_1 + m_2], l1, n))
    means = [math.fsum(v.tolist()) / v.size for v in lv]
    variances = [float(np.var(v, ddof=1)) if v.size > 1 else float("nan") for v in lv]
    return {"estimate": math.fsum(means), "stderr": math.sqrt(math.fsum(vv / v.size for vv, v in zip(variances, lv))),
            "level_mean": means, "level_var": variances, "m": [int(v.size) for v in lv]}


# ---------------------------------------------------------------------------
# Hutch++ on the Chebyshev interpolant: the variance reduction Section 5.3
# suggests for the Estrada index (the method of Meyer, Musco, Musco and
# Woodruff, 2021: deflate an orthonormal basis Q of the range of p(At) S, take
# tr(Q^T p(At) Q) exactly and Hutchinson's estimate on the rest)
# ---------------------------------------------------------------------------

def _operator(m, gram=False, scale=1.0):
    """v -> A v on blocks (dim x k): A = scale * m, or X^T X with X = scale * m."""
    import scipy.sparse as sp
    val = np.ones(m.nnz) if m.val is None else np.asarray(m.val, dtype=np.float64)
    X = sp.csr_matrix((val * scale, np.asarray(m.col), np.asarray(m.rowptr)), shape=(m.nrows, m.ncols))
    if gram:
        return lambda v: X.T @ (X @ v)
    return lambda v: X @ v


def poly_apply(m, a, b, c, X, gram=False, scale=1.0):
    """Y = p(At) X, p = sum_j c_j T_j (Section 2.2, Eq. chebSeries), by the
    three-term recurrence W_0 = X, W_1 = At X, W_{j+1} = 2 At W_j - W_{j-1}
    (Eq. recurrence) and Y = sum_j c_j W_j; At = alpha A + beta I with
    alpha = 2/(b-a), beta = -(a+b)/(b-a)."""
    A = _operator(m, gram, scale)
    alpha = 2.0 / (b - a)
    beta = -(a + b) / (b - a)

    def At(v):
        return alpha * A(v) + beta * v

    W0 = np.array(X, dtype=np.float64)
    Y = c[0] * W0
    if len(c) == 1:
        return Y
    W1 = At(W0)
    Y = Y + c[1] * W1
    for j in range(2, len(c)):
        W0, W1 = W1, 2.0 * At(W1) - W0
        Y = Y + c[j] * W1
    return Y


def hutchpp_parts(m, a, b, c, S, G, gram=False, scale=1.0, drop_tol=1e-10):
    """Hutch++ with explicit sketch vectors S (dim x s) and remainder probes G
    (dim x g) on tr p(At), p = sum_j c_j T_j:
      Q       orthonormal basis of p(At) S (numpy's QR); a column whose residual
              |R_jj| is at most drop_tol times its own norm is dependent and dropped,
      t1      tr(Q^T p(At) Q) = sum_i sum_j c_j q_i^T T_j(At) q_i,
      samples g_i'^T p(At) g_i' with g_i' = (I - Q Q^T) g_i.
    The estimate is t1 + mean(samples).  Returns (t1, samples, rank of Q)."""
    n = len(c) - 1
    S = np.asarray(S, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    if S.shape[1] > 0:
        Y = poly_apply(m, a, b, c, S, gram, scale)
        Q, R = np.linalg.qr(Y)
        keep = np.abs(np.diag(R)) > drop_tol * np.linalg.norm(Y, axis=0)
        Q = Q[:, keep]
    else:
        Q = np.zeros((S.shape[0], 0))

    def quad(V):
        if V.shape[1] == 0:
            return np.zeros(0)
        mu = moments_z(m, a, b, V.T, n, gram, scale)
        return mu @ np.asarray(c, dtype=np.float64)

    t1 = math.fsum(quad(Q).tolist())
    Gp = G - Q @ (Q.T @ G)
    return t1, quad(Gp), int(Q.shape[1])


def hutchpp(m, a, b, c, seed, probe_offset, s, g, gram=False, scale=1.0):
    """Hutch++ with Rademacher sketch and remainder probes: S has the probes
    with ids probe_offset .. probe_offset + s - 1, G the next g.  The standard
    error is that of the remainder mean (divisor g - 1; NaN for g < 2)."""
    d = m.ncols if gram else m.nrows
    S = np.zeros((d, s))
    G = np.zeros((d, g))
    for i in range(s):
        S[:, i] = rademacher(seed, probe_offset + i, d)
    for i in range(g):
        G[:, i] = rademacher(seed, probe_offset + s + i, d)
    t1, samples, rank = hutchpp_parts(m, a, b, c, S, G, gram, scale)
    t2 = math.fsum(samples.tolist()) / g if g > 0 else 0.0
    se = math.sqrt(float(np.var(samples, ddof=1)) / g) if g > 1 else float("nan")
    return {"estimate": t1 + t2, "stderr": se, "t_sketch": t1, "t_rest": t2, "samples": samples,
            "rank": rank}


# ---------------------------------------------------------------------------
# Triangle counting (Section 2.1 Example; Section 5.4)
# ---------------------------------------------------------------------------

def triangle_moments(m, seed, probe_offset, nprobes):
    """x[p] = (z^T A z, z^T A^2 z, z^T A^3 z) in exact int64 for probe ids
    probe_offset + p of a 0/1 symmetric pattern matrix."""
    x = np.zeros((nprobes, 3), dtype=np.int64)
    rc = lib().orc_triangle_moments(m.nrows, _ptr(m.rowptr), _ptr(m.col), seed, probe_offset,
                                    nprobes, _ptr(x))
    if rc != 0:
        raise MemoryError("oracle triangle moments failed")
    return x


def triangle_moments_z(m, z):
    z = np.ascontiguousarray(np.atleast_2d(z), dtype=np.int8)
    x = np.zeros((z.shape[0], 3), dtype=np.int64)
    rc = lib().orc_triangle_moments_z(m.nrows, _ptr(m.rowptr), _ptr(m.col), z.shape[0], _ptr(z),
                                      _ptr(x))
    if rc != 0:
        raise MemoryError("oracle triangle moments failed")
    return x


def triangle_count(m):
    """Exact triangle count by brute-force neighbour-list intersection."""
    return int(lib().orc_triangle_count(m.nrows, _ptr(m.rowptr), _ptr(m.col)))


def triangle_estimate(x, nnz, use_cv=True):
    """Section 5.4.  Without control variates: T = mean(x3) / 6.  With them:
    tr(A^3) = E[z^T (A^3 - a2 A^2 - a1 A) z] + a2 nnz(A)  (tr A = 0, tr A^2 = nnz),
    a1, a2 from ordinary least squares of x3 on (x1, x2) with intercept over the
    same samples.  Sums are exact integers; the 2x2 solve and the means are then
    done in double precision in the fixed order written below.

    Returns (estimate, stderr, a1, a2)."""
    x = np.asarray(x, dtype=np.int64)
    m = x.shape[0]
    x1 = [int(v) for v in x[:, 0]]
    x2 = [int(v) for v in x[:, 1]]
    x3 = [int(v) for v in x[:, 2]]
    S1, S2, S3 = sum(x1), sum(x2), sum(x3)
    S33 = sum(v * v for v in x3)
    C33 = m * S33 - S3 * S3                          # m^2 * population variance
    fm = float(m)
    if not use_cv:
        est = (float(S3) / fm) / 6.0
        var = float(C33) / (fm * (fm - 1.0)) if m > 1 else float("nan")
        return est, math.sqrt(var / fm) / 6.0, 0.0, 0.0
    S11 = sum(v * v for v in x1)
    S22 = sum(v * v for v in x2)
    S12 = sum(u * v for u, v in zip(x1, x2))
    S13 = sum(u * v for u, v in zip(x1, x3))
    S23 = sum(u * v for u, v in zip(x2, x3))
    C11 = float(m * S11 - S1 * S1)
    C22 = float(m * S22 - S2 * S2)
    C12 = float(m * S12 - S1 * S2)
    C13 = float(m * S13 - S1 * S3)
    C23 = float(m * S23 - S2 * S3)
    det = C11 * C22 - C12 * C12
    if det == 0.0:
        a1 = 0.0
        a2 = 0.0
    else:
        a1 = (C13 * C22 - C23 * C12) / det
        a2 = (C23 * C11 - C13 * C12) / det
    mean1 = float(S1) / fm
    mean2 = float(S2) / fm
    mean3 = float(S3) / fm
    est = (mean3 - a2 * (mean2 - float(nnz)) - a1 * mean1) / 6.0
    rss = float(C33) - a1 * C13 - a2 * C23           # m * residual sum of squares
    dof = fm - 3.0
    var = rss / (fm * dof) if m > 3 else float("nan")
    return est, math.sqrt(max(var, 0.0) / fm) / 6.0, a1, a2


def triangle_cv_cheb(a, b):
    """Section 5.4's a-priori control-variate coefficients, "chosen using the
    Chebyshev expansion of x^3".  With the spectrum of A inside [a, b] and
    A = r At + c I (c = (a+b)/2, r = (b-a)/2, so At maps [a, b] onto [-1, 1]),
    the expansion x^3 = (3 T_1(x) + T_3(x)) / 4 on [-1, 1] gives
        A^3 = (r^3/4) T_3(At) + 3c A^2 + (3r^2/4 - 3c^2) A + (c^3 - 3c r^2/4) I.
    Taking a2 = 3c and a1 = 3r^2/4 - 3c^2 removes every Chebyshev term of degree
    below 3 except the constant, which carries no variance (z^T I z = d), so
    z^T (A^3 - a2 A^2 - a1 A) z = (r^3/4) z^T T_3(At) z + const.  The
    coefficients do not depend on the samples, so the estimate has no bias from
    fitting.  Returns (a1, a2)."""
    c = 0.5 * (float(a) + float(b))
    r = 0.5 * (float(b) - float(a))
    return 0.75 * r * r - 3.0 * c * c, 3.0 * c


def triangle_estimate_fixed(x, nnz, a1, a2):
    """Section 5.4 with given (not fitted) coefficients:
    T = [mean x3 - a2 (mean x2 - nnz) - a1 mean x1] / 6, and its standard error
    from the sample variance (divisor m - 1) of the residuals x3 - a2 x2 - a1 x1,
    assembled from exact integer sums as
        m (m-1) var = C33 + a2^2 C22 + a1^2 C11 - 2 a2 C23 - 2 a1 C13 + 2 a1 a2 C12,
    C_ij = m S_ij - S_i S_j, in double precision in the order written.
    Returns (estimate, stderr)."""
    x = np.asarray(x, dtype=np.int64)
    m = x.shape[0]
    x1 = [int(v) for v in x[:, 0]]
    x2 = [int(v) for v in x[:, 1]]
    x3 = [int(v) for v in x[:, 2]]
    S1, S2, S3 = sum(x1), sum(x2), sum(x3)
    C11 = float(m * sum(v * v for v in x1) - S1 * S1)
    C22 = float(m * sum(v * v for v in x2) - S2 * S2)
    C33 = float(m * sum(v * v for v in x3) - S3 * S3)
    C12 = float(m * sum(u * v for u, v in zip(x1, x2)) - S1 * S2)
    C13 = float(m * sum(u * v for u, v in zip(x1, x3)) - S1 * S3)
    C23 = float(m * sum(u * v for u, v in zip(x2, x3)) - S2 * S3)
    a1 = float(a1)
    a2 = float(a2)
    fm = float(m)
    mean1 = float(S1) / fm
    mean2 = float(S2) / fm
    mean3 = float(S3) / fm
    est = (mean3 - a2 * (mean2 - float(nnz)) - a1 * mean1) / 6.0
    q = C33 + a2 * a2 * C22 + a1 * a1 * C11 - 2.0 * a2 * C23 - 2.0 * a1 * C13 + 2.0 * a1 * a2 * C12
    var = q / (fm * (fm - 1.0)) if m > 1 else float("nan")
    return est, math.sqrt(max(var, 0.0) / fm) / 6.0


# ---------------------------------------------------------------------------
# Spectrum interval (Section 2.2: the map needs a rough estimate of the extreme
# eigenvalues); Gershgorin discs
# ---------------------------------------------------------------------------

def gershgorin(m):
    lo, hi = float("inf"), float("-inf")
    for i in range(m.nrows):
        dg, off = 0.0, 0.0
        for k in range(m.rowptr[i], m.rowptr[i + 1]):
            v = 1.0 if m.val is None else float(m.val[k])
            if m.col[k] == i:
                dg += v
            else:
                off += abs(v)
        lo = min(lo, dg - off)
        hi = max(hi, dg + off)
    return lo, hi


def interval(m, scale=1.0, gram=False):
    """The default spectrum interval [a, b] of the operator, on the host: the
    Gershgorin discs of scale * A, or [0, s^2 ||X||_1 ||X||_inf] for A = X^T X
    with X = s * m, since ||X||_2^2 <= ||X||_1 ||X||_inf (Section 2.2 asks only
    for a rough estimate of the extreme eigenvalues)."""
    if gram:
        v = np.ones(m.nnz) if m.val is None else np.abs(np.asarray(m.val, dtype=np.float64))
        rows = np.repeat(np.arange(m.nrows), np.diff(np.asarray(m.rowptr)))
        r = np.bincount(rows, weights=v, minlength=m.nrows).max() if m.nnz else 0.0
        c = np.bincount(np.asarray(m.col), weights=v, minlength=m.ncols).max() if m.nnz else 0.0
        return 0.0, scale * scale * float(r) * float(c)
    lo, hi = gershgorin(m)
    return (scale * lo, scale * hi) if scale >= 0 else (scale * hi, scale * lo)


# ---------------------------------------------------------------------------
# Learned coarse level: a 16 -> 128 -> 128 -> 1 ReLU network trained by mean
# squared error (a project addition; its nearest relative in the paper is the
# regression control variate of Section 5.4).  Plain FP64 forward and
# hand-written backward, used to check the GPU kernels' gradients.
# ---------------------------------------------------------------------------

MLP_IN, MLP_HID = 16, 128


def mlp_init(seed=0):
    """He-style initial weights (normal, std sqrt(2 / fan_in)); biases zero."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((MLP_HID, MLP_IN)) * math.sqrt(2.0 / MLP_IN),
        "b1": np.zeros(MLP_HID),
        "W2": rng.standard_normal((MLP_HID, MLP_HID)) * math.sqrt(2.0 / MLP_HID),
        "b2": np.zeros(MLP_HID),
        "w3": rng.standard_normal(MLP_HID) * math.sqrt(1.0 / MLP_HID),
        "b3": 0.0,
    }


def mlp_forward(P, X):
    """X: B x 16.  Returns (y, cache)."""
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ P["w3"] + P["b3"]
    return y, (X, h1, h2)


def mlp_loss_grad(P, X, t):
    """Loss L = mean (y - t)^2 and its gradient with respect to every parameter."""
    y, (X, h1, h2) = mlp_forward(P, X)
    t = np.asarray(t, dtype=np.float64)
    B = X.shape[0]
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B
    g = {"w3": h2.T @ dy, "b3": float(np.sum(dy))}
    dh2 = np.outer(dy, P["w3"]) * (h2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ P["W2"]) * (h1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return L, g
