"""Pins of the FP64 picker-network oracle.

- central finite differences of the loss agree with the analytic gradients;
- a closed-form special case: with W2 and W3 the identity (square layers)
  and zero biases, y = relu(relu(W1 x)) = relu(W1 x), and the W1 gradient of
  the loss has the closed form (mask * (y - t) * [W1 x > 0]) x^T / sum(mask);
- masked outputs contribute nothing.
"""
import numpy as np

from oracle import mlp


def _params(rng, n_in=8, n_hidden=16, n_out=10, scale=0.5):
    return {k: rng.standard_normal(s) * scale for k, s in mlp.shapes(n_in, n_hidden, n_out).items()}


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    x = rng.standard_normal((12, 8))
    t = rng.standard_normal((12, 10))
    mask = (rng.random((12, 10)) < 0.6).astype(float)
    _, g = mlp.loss_and_grads(p, x, t, mask)
    h = 1e-6
    for name in mlp.PARAM_ORDER:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[name].shape)
            keep = p[name][idx]
            p[name][idx] = keep + h
            lp, _ = mlp.loss_and_grads(p, x, t, mask)
            p[name][idx] = keep - h
            lm, _ = mlp.loss_and_grads(p, x, t, mask)
            p[name][idx] = keep
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[name][idx])


def test_identity_layers_closed_form():
    rng = np.random.default_rng(1)
    n = 6
    p = {"W1": rng.standard_normal((n, n)), "b1": np.zeros(n), "W2": np.eye(n), "b2": np.zeros(n),
         "W3": np.eye(n), "b3": np.zeros(n)}
    x = rng.standard_normal((5, n))
    t = rng.standard_normal((5, n))
    mask = np.ones((5, n))
    y, _ = mlp.forward(p, x)
    z = x @ p["W1"].T
    assert np.allclose(y, np.maximum(z, 0.0))
    _, g = mlp.loss_and_grads(p, x, t, mask)
    expect = ((np.maximum(z, 0.0) - t) * (z > 0)).T @ x / mask.sum()
    assert np.allclose(g["W1"], expect)


def test_masked_outputs_do_not_contribute():
    rng = np.random.default_rng(2)
    p = _params(rng)
    x = rng.standard_normal((4, 8))
    t = rng.standard_normal((4, 10))
    mask = np.zeros((4, 10))
    mask[:, :3] = 1
    l1, g1 = mlp.loss_and_grads(p, x, t, mask)
    t2 = t.copy()
    t2[:, 3:] += 100.0
    l2, g2 = mlp.loss_and_grads(p, x, t2, mask)
    assert l1 == l2
    for k in mlp.PARAM_ORDER:
        assert np.array_equal(g1[k], g2[k])
