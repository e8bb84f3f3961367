"""FP64 forward/backward of the parameter-picker network (test infrastructure).

TEST INFRASTRUCTURE ONLY.  The GPU library trains and evaluates the same
network with its own kernels (FP16 weights, FP32 accumulation); this module is
the plain FP64 restatement its gradients are checked against.

Network:  x (n_in) -> z1 = W1 x + b1 -> h1 = relu(z1) -> z2 = W2 h1 + b2
          -> h2 = relu(z2) -> y = W3 h2 + b3 (n_out)
Loss:     L = sum_{b,k} mask[b,k] (y[b,k] - t[b,k])^2 / (2 sum mask)
Weights are row-major: W1 (n_hidden x n_in), W2 (n_hidden x n_hidden),
W3 (n_out x n_hidden).
"""
import numpy as np

PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(n_in, n_hidden, n_out):
    return {"W1": (n_hidden, n_in), "b1": (n_hidden,), "W2": (n_hidden, n_hidden), "b2": (n_hidden,),
            "W3": (n_out, n_hidden), "b3": (n_out,)}


def unflatten(flat, n_in, n_hidden, n_out):
    out, off = {}, 0
    for k in PARAM_ORDER:
        shp = shapes(n_in, n_hidden, n_out)[k]
        size = int(np.prod(shp))
        out[k] = np.asarray(flat[off:off + size], dtype=np.float64).reshape(shp)
        off += size
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k in PARAM_ORDER])


def forward(p, x):
    """Returns y and the intermediates (z1, h1, z2, h2)."""
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, z1, h1, z2, h2)


def loss_and_grads(p, x, t, mask):
    y, (x, z1, h1, z2, h2) = forward(p, x)
    mask = np.asarray(mask, dtype=np.float64)
    denom = max(float(mask.sum()), 1.0)
    r = (y - np.asarray(t, dtype=np.float64)) * mask
    loss = float(np.sum(r * r) / (2.0 * denom))
    gy = r / denom                              # dL/dy
    g = {"W3": gy.T @ h2, "b3": gy.sum(0)}
    gh2 = gy @ p["W3"]
    gz2 = gh2 * (z2 > 0)
    g["W2"] = gz2.T @ h1
    g["b2"] = gz2.sum(0)
    gh1 = gz2 @ p["W2"]
    gz1 = gh1 * (z1 > 0)
    g["W1"] = gz1.T @ x
    g["b1"] = gz1.sum(0)
    return loss, g
