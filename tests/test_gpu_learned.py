"""GPU parity of the learned coarse level: the network's loss, gradient and
forward pass (tensor-core BF16 with FP32 accumulation) against the FP64 oracle
given the same BF16-rounded weights and inputs, element by element; the
three-level estimator against the oracle's combination of the same levels
(with a trained network's outputs as the coarse level's samples), and against
the plain multilevel estimator when the network is zero.

Element-wise bounds.  Inputs X and the weights W1, W2 are BF16 values before
either side sees them.  The kernel also rounds to BF16 (8 significant bits)
the values it stores for its tensor cores: the hidden layer H1 on the forward
path, then dH2 and dH1 on the backward path.  The reference is the oracle's
FP64 network evaluated with those same three roundings (_bf16_reference);
what separates the kernel from it is FP32 accumulation, unit u_f = 2^-24 per
sum of K terms times the sum of their magnitudes (a factor 4 for the tensor
cores' internal order), a ReLU mask that differs where a pre-activation lies
within that error of zero, and a BF16 rounding that differs where the value
lies that close to a rounding boundary.  _bounds carries these term by term
through the layers; each GPU value must lie within twice its bound of the
reference, and the reference within the plain BF16 perturbation of the
oracle's own FP64 values."""
import numpy as np
import pytest

from paper_2103_10516_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    from paper_2103_10516_gb300 import build, mlt
    build.build()
    return mlt


def bf16(a):
    """Round float64 values to the nearest BF16 (round to nearest even)."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _setup(O, seed, n):
    rng = np.random.default_rng(seed)
    P = O.mlp_init(seed)
    P["b1"] = rng.standard_normal(128) * 0.1
    P["b2"] = rng.standard_normal(128) * 0.1
    P["b3"] = 0.25
    P["W1"] = bf16(P["W1"])
    P["W2"] = bf16(P["W2"])
    X = bf16(rng.uniform(-1, 1, (n, 16)))
    T = rng.standard_normal(n)
    return P, X, T


UF = 2.0 ** -24


def _bracket(v, e):
    """Largest move of bf16(v) when v moves by at most e (bf16 is monotone)."""
    r = bf16(v)
    return np.maximum(np.abs(bf16(v + e) - r), np.abs(bf16(v - e) - r))


def _bf16_reference(P, X, T=None):
    """The oracle's network in FP64 with the kernel's three BF16 roundings
    (H1, dH2, dH1) and the pieces _bounds needs."""
    R = {}
    R["A1"] = X @ P["W1"].T + P["b1"]
    R["H1"] = bf16(np.maximum(R["A1"], 0.0))
    R["A2"] = R["H1"] @ P["W2"].T + P["b2"]
    R["H2"] = np.maximum(R["A2"], 0.0)
    R["y"] = R["H2"] @ P["w3"] + P["b3"]
    if T is None:
        return R
    n = X.shape[0]
    R["r"] = R["y"] - T
    R["dy"] = 2.0 * R["r"] / n
    R["g"] = R["dy"][:, None] * P["w3"][None, :] * (R["A2"] > 0)
    R["gb"] = bf16(R["g"])
    R["D1"] = (R["gb"] @ P["W2"]) * (R["H1"] > 0)
    R["D1b"] = bf16(R["D1"])
    R["grad"] = {"b3": float(np.sum(R["dy"])), "w3": R["dy"] @ R["H2"], "b2": np.sum(R["g"], axis=0),
                 "W2": R["gb"].T @ R["H1"], "b1": np.sum(R["D1"], axis=0), "W1": R["D1b"].T @ X}
    R["loss"] = float(np.mean(R["r"] ** 2))
    return R


def _bounds(P, X, R, ex=None):
    """Element-wise bounds of |kernel - reference| (see the module docstring);
    ex bounds how far the kernel's BF16 inputs may be from X, when they are
    computed rather than given."""
    aW1, aW2, aw3 = np.abs(P["W1"]), np.abs(P["W2"]), np.abs(P["w3"])
    acc1 = 4 * 17 * UF * (np.abs(X) @ aW1.T + np.abs(P["b1"]))
    if ex is not None:
        acc1 = acc1 + ex @ aW1.T
    # H1 = bf16(relu(A1)): relu and bf16 are monotone, so an A1 error of acc1
    # moves the stored value by at most this bracket
    e1 = np.maximum(np.abs(bf16(np.maximum(R["A1"] + acc1, 0)) - R["H1"]),
                    np.abs(bf16(np.maximum(R["A1"] - acc1, 0)) - R["H1"]))
    H1p = np.abs(R["H1"]) + e1
    e2 = e1 @ aW2.T + 4 * 129 * UF * (H1p @ aW2.T + np.abs(P["b2"]))
    H2p = np.abs(R["H2"]) + e2
    ey = e2 @ aw3 + 4 * 129 * UF * (H2p @ aw3 + abs(P["b3"]))
    B = {"y": ey}
    if "g" not in R:
        return B
    n = X.shape[0]
    dy = R["dy"]
    edy = 2.0 * ey / n + UF * np.abs(dy)
    gmax = np.abs(dy)[:, None] * aw3[None, :]
    flip2 = np.abs(R["A2"]) <= e2
    eg32 = edy[:, None] * aw3[None, :] + UF * gmax + flip2 * gmax
    egb = _bracket(R["g"], eg32)
    flip1 = (e1 > 0) & (np.abs(R["H1"]) <= e1)
    gbp = np.abs(R["gb"]) + egb
    eD1 = egb @ aW2 + 4 * 129 * UF * (gbp @ aW2) + flip1 * (gbp @ aW2)
    eD1b = _bracket(R["D1"], eD1)
    aX = np.abs(X)
    B["grad"] = {
        "b3": float(np.sum(edy) + 4 * n * UF * np.sum(np.abs(dy))),
        "w3": edy @ H2p + np.abs(dy) @ e2 + 4 * n * UF * (np.abs(dy) @ H2p),
        "b2": np.sum(eg32, axis=0) + 4 * n * UF * np.sum(np.abs(R["g"]), axis=0),
        "W2": egb.T @ H1p + np.abs(R["gb"]).T @ e1 + 4 * n * UF * (gbp.T @ H1p),
        "b1": np.sum(eD1, axis=0) + 4 * n * UF * np.sum(np.abs(R["D1"]) + eD1, axis=0),
        "W1": eD1b.T @ aX + 4 * n * UF * ((np.abs(R["D1b"]) + eD1b).T @ aX),
    }
    B["loss"] = float(np.mean(2.0 * np.abs(R["r"]) * ey + ey ** 2) + 4 * n * UF * np.mean(R["r"] ** 2))
    return B


@pytest.mark.parametrize("n", [128, 300, 1000])
def test_forward_matches_oracle(L, O, n):
    P, X, _ = _setup(O, 1, n)
    with L.Surrogate(0) as S:
        S.set_params(P)
        y = S.predict(X)
    ref, _ = O.mlp_forward(P, X)
    R = _bf16_reference(P, X)
    B = _bounds(P, X, R)
    err = np.abs(y - R["y"])
    assert np.all(err <= 2.0 * B["y"] + 1e-12), float(np.max(err / (B["y"] + 1e-12)))
    # the rounded reference differs from the FP64 oracle only by the H1
    # rounding, carried through the last two layers
    dH = np.abs(R["H1"] - np.maximum(R["A1"], 0))
    assert np.all(np.abs(R["y"] - ref) <= (dH @ np.abs(P["W2"]).T) @ np.abs(P["w3"]) * 1.000001 + 1e-12)


@pytest.mark.parametrize("n", [128, 300, 1000])
def test_gradient_matches_oracle(L, O, n):
    P, X, T = _setup(O, 2, n)
    with L.Surrogate(0) as S:
        S.set_params(P)
        loss, g = S.loss_grad(X, T)
    R = _bf16_reference(P, X, T)
    B = _bounds(P, X, R)
    assert abs(loss - R["loss"]) <= 2.0 * B["loss"] + 1e-12
    G = L.unpack_params(g)
    for k in ("W1", "b1", "W2", "b2", "w3"):
        err = np.abs(np.asarray(G[k], dtype=np.float64) - R["grad"][k])
        assert np.all(err <= 2.0 * B["grad"][k] + 1e-12), (k, float(np.max(err / (B["grad"][k] + 1e-12))))
    assert abs(G["b3"] - R["grad"]["b3"]) <= 2.0 * B["grad"]["b3"] + 1e-12
    # and the rounded reference against the FP64 oracle: the three BF16
    # roundings (unit 2^-8) move each gradient, a sum over the batch, by at
    # most a few per cent of its largest entry (5.4% for dW2 at 128 samples)
    rl, rg = O.mlp_loss_grad(P, X, T)
    for k in ("W1", "b1", "W2", "b2", "w3"):
        scale = np.max(np.abs(rg[k]))
        assert np.max(np.abs(R["grad"][k] - rg[k])) <= 0.1 * scale, k
    assert abs(R["loss"] - rl) <= 0.02 * rl


def test_params_roundtrip_and_training_lowers_loss(L, O):
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (4096, 16)).astype(np.float32)
    w = rng.standard_normal(16)
    T = (np.tanh(X @ w) + 0.5 * X[:, 0] ** 2).astype(np.float32)
    with L.Surrogate(3) as S:
        v = S.get_params()
        S.set_params(v)
        assert np.array_equal(S.get_params(), v)
        l0, _ = S.loss_grad(X, T)
        l1 = S.train(X, T, epochs=30, batch=512, lr=3e-3)
        l2, _ = S.loss_grad(X, T)
    assert l2 < 0.2 * l0 and l1 < l0


def test_zero_network_is_plain_multilevel(L, O):
    # with S = 0 the levels are 0, P_l1 and P_n - P_l1 on the same probes as
    # the plain multilevel estimator with levels (l1, n) and ids after the net level
    m = synth.grid_laplacian_2d(24, shift=0.1)
    zero = np.zeros(L.MLT_NET_NPARAMS, dtype=np.float32)
    with L.Matrix(m) as M, L.Surrogate(0) as S:
        S.set_params(zero)
        P = L.learned_params("log", 0.1, 8.1, 64, 32, m_net=40, m_1=30, m_2=12, seed=4, probe_offset=7)
        got = L.mlt_learned_estimate(M.handle, S.handle, P)
    ref = O.mlmc_fixed(m, "log", 0.1, 8.1, 64, [32, 64], [30, 12], seed=4, probe_offset=7 + 40)
    tol = 1e-10 * np.sum(np.abs(ref["coeffs"])) * m.nrows
    assert got["levels"] == [15, 32, 64] and got["m"] == [40, 30, 12]
    assert got["level_mean"][0] == 0.0
    assert abs(got["estimate"] - ref["estimate"]) <= tol


def test_trained_level_reduces_variance(L, O):
    # Estrada-type workload (exp on a scaled adjacency): a network trained on
    # (mu_0..mu_15)/d -> P_64/d must leave P_64 - d S with far less variance
    # than P_64 itself, i.e. the learned level pays for itself
    g = synth.rmat_adjacency(12, 8, seed=7)
    with L.Matrix(g) as M0:
        _, rho = M0.bounds()
    scale = 4.0 / rho
    with L.Matrix(g, scale=scale) as M, L.Surrogate(1) as S:
        P = L.learned_params("exp", -4.0, 4.0, 96, 64, m_net=256, m_1=128, m_2=32, seed=9,
                             probe_offset=1 << 20)
        loss = L.mlt_learned_train(M.handle, S.handle, P, 8192, 0, 60, 1024, 2e-3)
        got = L.mlt_learned_estimate(M.handle, S.handle, P)
        plain = M.mlmc("exp", -4.0, 4.0, 96, seed=9, levels=[64, 96], m=[128, 32])
    assert np.isfinite(loss)
    var_corr = got["level_var"][1]
    var_plain = plain["level_var"][0]
    assert var_corr < 0.25 * var_plain, (var_corr, var_plain)
    # unbiased: the two estimates agree within their standard errors
    assert abs(got["estimate"] - plain["estimate"]) < 5 * np.hypot(got["stderr"], plain["stderr"])


def test_trained_learned_estimate_matches_oracle(L, O):
    """A trained network's three-level estimate (levels S, P_64 - S, P_96 - P_64)
    against the oracle's combination of the same levels on the same probes.
    The oracle side takes the trained parameters and standardisation from the
    library and evaluates the network in FP64 at the kernel's BF16 rounding
    points (features and weights rounded as the kernel rounds them); the
    features come from the oracle's own moments, which differ from the GPU's by
    at most 1e-10 d, so each feature may sit on the other side of a BF16
    rounding boundary within that distance (the bracket term).  Each level mean
    must agree within the mean of its samples' bounds plus the moment
    tolerance 1e-10 sum|c_j| d."""
    g = synth.rmat_adjacency(12, 8, seed=7)
    d = g.nrows
    sc = 4.0 / float(np.max(np.diff(g.rowptr)))          # Gershgorin: spectrum inside [-4, 4]
    n, l1, m_net, m_1, m_2, off = 96, 64, 200, 60, 20, 1 << 20
    with L.Matrix(g, scale=sc) as M, L.Surrogate(1) as S:
        P = L.learned_params("exp", -4.0, 4.0, n, l1, m_net=m_net, m_1=m_1, m_2=m_2, seed=9, probe_offset=off)
        L.mlt_learned_train(M.handle, S.handle, P, 4096, 0, 40, 1024, 2e-3)
        got = L.mlt_learned_estimate(M.handle, S.handle, P)
        prm = L.unpack_params(S.get_params())
        fm, fs, tm, ts = S.get_norm()
    c = O.cheb_coeffs("exp", -4.0, 4.0, n)
    mu = O.moments(g, -4.0, 4.0, 9, off, [15] * m_net + [l1] * m_1 + [n] * m_2, scale=sc)
    x = (mu[:m_net + m_1, :16] / d - fm) / fs
    xb = bf16(x)
    Pref = {"W1": bf16(prm["W1"]), "W2": bf16(prm["W2"]), "b1": np.asarray(prm["b1"], dtype=np.float64),
            "b2": np.asarray(prm["b2"], dtype=np.float64), "w3": np.asarray(prm["w3"], dtype=np.float64),
            "b3": float(prm["b3"])}
    R = _bf16_reference(Pref, xb)
    dx = 1e-10 / np.asarray(fs)[None, :] + 2.0 ** -24 * np.abs(x)
    B = _bounds(Pref, xb, R, ex=_bracket(x, dx))
    s_ref = d * (tm + ts * R["y"])
    tol_s = d * ts * 2.0 * B["y"]
    ref = O.learned_estimate(c, mu, s_ref, m_net, m_1, m_2, l1)
    tol_mu = 1e-10 * np.sum(np.abs(c)) * d
    tols = [float(np.mean(tol_s[:m_net])) + 1e-9 * abs(ref["level_mean"][0]),
            float(np.mean(tol_s[m_net:])) + tol_mu + 1e-9 * abs(ref["level_mean"][1]),
            tol_mu]
    assert got["levels"] == [15, l1, n] and got["m"] == [m_net, m_1, m_2]
    for k in range(3):
        assert abs(got["level_mean"][k] - ref["level_mean"][k]) <= tols[k], (k, got["level_mean"][k],
                                                                            ref["level_mean"][k], tols[k])
    assert abs(got["estimate"] - ref["estimate"]) <= sum(tols)
    # the bound is informative: far below the network level's own spread
    assert tols[0] < 0.1 * np.sqrt(ref["level_var"][0])
