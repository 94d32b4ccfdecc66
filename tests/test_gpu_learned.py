"""GPU parity of the learned coarse level: the network's loss, gradient and
forward pass (tensor-core BF16 with FP32 accumulation) against the FP64 oracle
given the same BF16-rounded weights and inputs, and the three-level estimator
against the oracle's plain multilevel estimator when the network is zero.

BF16 tolerance: inputs and weights are rounded before both sides see them, so
what remains is the BF16 rounding (unit 2^-9) of the values fed to the tensor
cores: H1 on the forward path (one rounding before the output), and dH2 then
dH1 on the backward path (two roundings before dW1).  Gradients are sums over
the batch of terms of both signs, so their relative error exceeds the
per-element 2^-9 by the cancellation; the bound used is 2e-2 for the forward
pass and 5e-2 in relative Frobenius norm per gradient tensor."""
import numpy as np
import pytest

from paper_2103_10516_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_BF16 = 2e-2
TOL_GRAD = 5e-2


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


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30)


@pytest.mark.parametrize("n", [128, 300, 1000])
def test_forward_matches_oracle(L, O, n):
    P, X, _ = _setup(O, 1, n)
    with L.Surrogate(0) as S:
        S.set_params(P)
        y = S.predict(X)
    ref, _ = O.mlp_forward(P, X)
    assert _rel(y, ref) < TOL_BF16


@pytest.mark.parametrize("n", [128, 300, 1000])
def test_gradient_matches_oracle(L, O, n):
    P, X, T = _setup(O, 2, n)
    with L.Surrogate(0) as S:
        S.set_params(P)
        loss, g = S.loss_grad(X, T)
    rl, rg = O.mlp_loss_grad(P, X, T)
    assert abs(loss - rl) <= TOL_BF16 * rl
    G = L.unpack_params(g)
    for k in ("W1", "b1", "W2", "b2", "w3"):
        assert _rel(G[k], rg[k]) < TOL_GRAD, k
    assert abs(G["b3"] - rg["b3"]) <= TOL_GRAD * (abs(rg["b3"]) + 1e-3)


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
