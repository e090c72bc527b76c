"""Double-precision reference of the learned cost model's network - TEST INFRASTRUCTURE ONLY
(used by the tests to check the GPU forward pass and gradients; shares no code with the
library).

Network: standardised 4 features -> 32 tanh -> 32 tanh -> 1 (linear), loss = mean squared
error against (target - target_mean).  Parameter layout: W1[32][4], b1[32], W2[32][32], b2[32],
W3[32], b3 (1249 floats).  The GPU runs the forward pass with FP16 weights, so the tests
round the parameters to float16 before calling this reference.
"""
import numpy as np

IN, H = 4, 32
SIZES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))]
NUM_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SIZES])


def forward(p, X, mean, std, tmean):
    w = unpack(p)
    x = (np.asarray(X, np.float64) - mean) / std
    h1 = np.tanh(x @ w["W1"].T + w["b1"])
    h2 = np.tanh(h1 @ w["W2"].T + w["b2"])
    return h2 @ w["W3"] + w["b3"][0], (x, h1, h2)


def loss(p, X, T, mean, std, tmean):
    y, _ = forward(p, X, mean, std, tmean)
    e = y - (np.asarray(T, np.float64) - tmean)
    return float(np.mean(e * e))


def loss_and_grad(p, X, T, mean, std, tmean):
    """Mean squared error and its analytic gradient (back-propagation, float64)."""
    w = unpack(p)
    y, (x, h1, h2) = forward(p, X, mean, std, tmean)
    n = len(y)
    e = y - (np.asarray(T, np.float64) - tmean)
    dy = 2.0 * e / n
    g = {"W3": dy @ h2, "b3": np.array([dy.sum()])}
    d2 = np.outer(dy, w["W3"]) * (1.0 - h2 * h2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ w["W2"]) * (1.0 - h1 * h1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return float(np.mean(e * e)), pack(g)
