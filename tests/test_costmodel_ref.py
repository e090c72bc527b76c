"""Pins of the CPU reference network (no GPU): its analytic gradient must match central finite
differences of its own loss, and a planted sign error in the back-propagation must not."""
import numpy as np

from oracle import costmodel_ref as ref


def _data(seed=0, n=64):
    rng = np.random.default_rng(seed)
    X = rng.normal(2.0, 1.5, size=(n, 4))
    T = rng.normal(10.0, 2.0, size=n)
    p = rng.normal(0, 0.4, size=ref.NUM_PARAMS)
    return p, X, T, X.mean(0), X.std(0), T.mean()


def test_parameter_count():
    assert ref.NUM_PARAMS == 1249


def test_gradient_matches_finite_differences():
    p, X, T, m, s, tm = _data()
    _, g = ref.loss_and_grad(p, X, T, m, s, tm)
    rng = np.random.default_rng(1)
    for i in rng.choice(ref.NUM_PARAMS, 80, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (ref.loss(pp, X, T, m, s, tm) - ref.loss(pm, X, T, m, s, tm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_finite_differences_catch_a_wrong_sign():
    p, X, T, m, s, tm = _data(3)
    _, g = ref.loss_and_grad(p, X, T, m, s, tm)
    i = 4 * 32 + 32 + 5            # a W2 entry
    g_bad = g.copy()
    g_bad[i] = -g_bad[i]
    h = 1e-6
    pp, pm = p.copy(), p.copy()
    pp[i] += h
    pm[i] -= h
    fd = (ref.loss(pp, X, T, m, s, tm) - ref.loss(pm, X, T, m, s, tm)) / (2 * h)
    assert abs(fd - g[i]) < 1e-6 + 1e-5 * abs(fd)
    assert abs(fd - g_bad[i]) > 1e-4 * abs(fd) or abs(fd) < 1e-9
