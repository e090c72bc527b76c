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


def _one_path(a, b, c, d, wi=0, hi=0, hj=0):
    """Parameters with a single path: feature wi -> hidden1 hi -> hidden2 hj -> output."""
    p = np.zeros(ref.NUM_PARAMS)
    p[hi * 4 + wi] = a                                 # W1[hi][wi]
    p[4 * 32 + 32 + hj * 32 + hi] = b                  # W2[hj][hi]
    p[4 * 32 + 32 + 32 * 32 + 32 + hj] = c             # W3[hj]
    p[-1] = d                                          # b3
    return p


def test_forward_of_the_zero_network_is_its_output_bias():
    p = np.zeros(ref.NUM_PARAMS)
    p[-1] = 0.75
    X = np.random.default_rng(4).normal(size=(10, 4))
    y, _ = ref.forward(p, X, np.zeros(4), np.ones(4), 3.0)
    assert np.allclose(y, 0.75)


def test_forward_of_a_single_path_by_hand():
    # y = c tanh(b tanh(a (x_2 - m_2) / s_2)) + d, the composition the network's definition
    # gives for one feature -> one hidden unit -> one hidden unit -> output
    a, b, c, d = 0.7, -1.3, 2.0, 0.25
    p = _one_path(a, b, c, d, wi=2, hi=5, hj=9)
    X = np.array([[0.0, 0.0, 1.0, 0.0], [9.0, 9.0, -2.0, 9.0], [1.0, 2.0, 4.0, 3.0]])
    mean, std = np.array([0.0, 0.0, 1.0, 0.0]), np.array([1.0, 1.0, 2.0, 1.0])
    y, _ = ref.forward(p, X, mean, std, 0.0)
    for k, x2 in enumerate([1.0, -2.0, 4.0]):
        z = (x2 - 1.0) / 2.0
        want = c * np.tanh(b * np.tanh(a * z)) + d
        assert abs(y[k] - want) < 1e-12
    # the loss is the mean squared error against the centred target
    T = np.array([5.0, 6.0, 7.0])
    assert abs(ref.loss(p, X, T, mean, std, 4.0) - np.mean((y - (T - 4.0)) ** 2)) < 1e-12


def test_forward_ignores_unconnected_features():
    p = _one_path(1.1, 0.9, -0.5, 0.0, wi=1)
    X = np.random.default_rng(5).normal(size=(6, 4))
    X2 = X.copy()
    X2[:, [0, 2, 3]] += 10.0
    y1, _ = ref.forward(p, X, np.zeros(4), np.ones(4), 0.0)
    y2, _ = ref.forward(p, X2, np.zeros(4), np.ones(4), 0.0)
    assert np.allclose(y1, y2)
