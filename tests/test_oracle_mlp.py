"""Pins of the oracle's learned-level network: hand-written backward against
central finite differences in FP64."""
import numpy as np
import pytest


@pytest.mark.parametrize("seed", [0, 1])
def test_mlp_gradient_matches_finite_differences(O, seed):
    rng = np.random.default_rng(seed)
    P = O.mlp_init(seed)
    P["b1"] = rng.standard_normal(128) * 0.1
    P["b2"] = rng.standard_normal(128) * 0.1
    P["b3"] = 0.3
    X = rng.standard_normal((37, 16))
    t = rng.standard_normal(37)
    L, g = O.mlp_loss_grad(P, X, t)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        arr = np.atleast_1d(P[name]) if name != "b3" else None
        idxs = [None] if name == "b3" else [tuple(rng.integers(0, s) for s in P[name].shape)
                                            for _ in range(6)]
        for ix in idxs:
            Q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in P.items()}
            if ix is None:
                Q["b3"] = P["b3"] + h
                lp, _ = O.mlp_loss_grad(Q, X, t)
                Q["b3"] = P["b3"] - h
                lm, _ = O.mlp_loss_grad(Q, X, t)
                fd, an = (lp - lm) / (2 * h), g["b3"]
            else:
                Q[name][ix] = P[name][ix] + h
                lp, _ = O.mlp_loss_grad(Q, X, t)
                Q[name][ix] = P[name][ix] - h
                lm, _ = O.mlp_loss_grad(Q, X, t)
                fd, an = (lp - lm) / (2 * h), g[name][ix]
            assert abs(fd - an) <= 1e-6 * (1.0 + abs(fd)), (name, ix, fd, an)


def test_mlp_linear_regime_closed_form(O):
    # with all pre-activations positive the network is affine in x; with
    # W2 = I and w3 = e_0 the output is the first hidden unit
    P = O.mlp_init(0)
    P["W1"] = np.zeros((128, 16))
    P["W1"][0, 3] = 2.0
    P["b1"] = np.full(128, 5.0)
    P["W2"] = np.eye(128)
    P["w3"] = np.zeros(128)
    P["w3"][0] = 1.0
    X = np.random.default_rng(2).uniform(-1, 1, (10, 16))
    y, _ = O.mlp_forward(P, X)
    assert np.allclose(y, 2.0 * X[:, 3] + 5.0, atol=1e-14)
