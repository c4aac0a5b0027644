"""Pins of the surrogate network oracle (oracle/surrogate.py) against facts that do not
depend on it: an independent library correlation, shifts, the adjoint identity, central
finite differences of the loss, and the closed form of Adam under a constant gradient."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import surrogate as S


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("periodic", [(True, True, True), (True, True, False), (False, False, True)])
def test_conv_matches_scipy_correlate(periodic):
    x = _rand((2, 5, 6, 7), 1)
    W = _rand((3, 2, 3, 3, 3), 2)
    b = _rand(3, 3)
    y = S.conv(x, W, b, periodic)
    xp = S.pad(x, periodic)    # padding is checked on its own below
    for o in range(3):
        ref = np.full(x.shape[1:], b[o])
        for i in range(2):
            full = ndimage.correlate(xp[i], W[o, i], mode="constant", cval=0.0)
            ref += full[1:-1, 1:-1, 1:-1]
        assert np.allclose(y[o], ref, atol=1e-12)


def test_pad_is_wrap_or_zero_per_axis():
    x = _rand((1, 4, 5, 6), 4)
    p = S.pad(x, (True, False, True))         # x periodic, y zero, z periodic
    assert np.array_equal(p[0, 1:-1, 1:-1, 0], x[0, :, :, -1])   # x wraps
    assert np.array_equal(p[0, 1:-1, 0, 1:-1], np.zeros((4, 6)))   # y zero
    assert np.array_equal(p[0, 0, 1:-1, 1:-1], x[0, -1])           # z wraps


def test_single_tap_kernel_is_a_shift():
    x = _rand((1, 4, 5, 6), 5)
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 1, 1, 2] = 1.0                    # reads x at offset +1 along the x axis
    y = S.conv(x, W, np.zeros(1), (True, True, True))
    assert np.allclose(y[0], np.roll(x[0], -1, axis=2))
    y0 = S.conv(x, W, np.zeros(1), (False, True, True))
    assert np.allclose(y0[0, :, :, :-1], x[0, :, :, 1:]) and np.allclose(y0[0, :, :, -1], 0.0)


@pytest.mark.parametrize("periodic", [(True, True, True), (True, False, True), (False, False, False)])
def test_conv_adjoint_identity(periodic):
    x = _rand((2, 4, 5, 3), 6)
    gy = _rand((3, 4, 5, 3), 7)
    W = _rand((3, 2, 3, 3, 3), 8)
    lhs = np.sum(S.conv(x, W, np.zeros(3), periodic) * gy)
    rhs = np.sum(x * S.conv_adjoint(gy, W, periodic))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_gradients_match_central_differences():
    periodic = (True, True, False)
    params = S.init_params(C=2, seed=3)
    for k in range(1, 8, 2):
        params[k] = _rand(params[k].shape, 10 + k) * 0.1      # non-zero biases
    Q = _rand((4, 4, 4), 11)
    U = _rand((4, 4, 4), 12)
    sq, su = 1.7, 0.6
    loss, grads = S.loss_and_grad(params, Q, U, sq, su, periodic)
    rng = np.random.default_rng(13)
    h = 1e-6
    for k in range(8):
        for _ in range(3):
            idx = tuple(rng.integers(0, n) for n in params[k].shape)
            pp = [p.copy() for p in params]
            pm = [p.copy() for p in params]
            pp[k][idx] += h
            pm[k][idx] -= h
            fd = (S.loss_and_grad(pp, Q, U, sq, su, periodic)[0] - S.loss_and_grad(pm, Q, U, sq, su, periodic)[0]) / (2 * h)
            assert abs(fd - grads[k][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, grads[k][idx])


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g, m_hat = g and v_hat = g^2 at every step, so each step
    # moves the parameter by lr * g / (|g| + eps)
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 1e-3])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        S.adam_step(p, g, m, v, t, lr=lr, eps=eps)
    expect = np.array([1.0, -2.0, 0.5]) - 5 * lr * g[0] / (np.abs(g[0]) + eps)
    assert np.allclose(p[0], expect, rtol=0, atol=1e-12)


def test_leaky_activation_and_its_derivative():
    z = np.array([-2.0, -0.5, 0.0, 0.25, 3.0])
    h = S.act(z)
    assert np.array_equal(h, [-0.2, -0.05, 0.0, 0.25, 3.0])
    assert np.array_equal(S.act_grad(h), [0.1, 0.1, 0.1, 1.0, 1.0])
