"""Pins of the FP64 closure oracle: convolution, GELU, gradients and Adam (no GPU)."""
import math

import numpy as np
import pytest

import synthetic
from oracle import closure as cl


def _rand(seed, shape, scale=1.0):
    return (synthetic.uniform_field(seed, shape).astype(np.float64) - 0.5) * 2 * scale


def _conv_per_tap(x, w, b):
    """Brute force: accumulate one shifted, zero-padded copy of x per tap."""
    cin, nz, ny, nx = x.shape
    cout = w.shape[0]
    xp = np.zeros((cin, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((cout, nz, ny, nx)) + (b.reshape(-1, 1, 1, 1) if b is not None else 0.0)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                shifted = xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                y += np.einsum("oc,czyx->ozyx", w[:, :, dz, dy, dx], shifted)
    return y


@pytest.mark.parametrize("cin,cout,shape", [(3, 16, (5, 6, 7)), (16, 16, (4, 5, 3)), (16, 1, (6, 4, 5))])
def test_conv_matches_per_tap_brute_force(cin, cout, shape):
    x = _rand(1, (cin,) + shape)
    w = _rand(2, (cout, cin, 3, 3, 3))
    b = _rand(3, (cout,))
    np.testing.assert_allclose(cl.conv3d(x, w, b), _conv_per_tap(x, w, b), rtol=0, atol=1e-12)


def test_conv_delta_kernel_is_a_shift():
    x = _rand(4, (1, 5, 6, 7))
    w = np.zeros((1, 1, 3, 3, 3))
    w[0, 0, 2, 1, 0] = 1.0  # tap (dz, dy, dx) = (+1, 0, -1): y[z,y,x] = x[z+1, y, x-1]
    y = cl.conv3d(x, w, None)
    ref = np.zeros_like(x)
    ref[0, :-1, :, 1:] = x[0, 1:, :, :-1]
    np.testing.assert_array_equal(y, ref)


def test_gelu_values():
    assert cl.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)
    xs = np.linspace(-5, 5, 41)
    np.testing.assert_allclose(cl.gelu(xs) - cl.gelu(-xs), xs, rtol=0, atol=1e-15)
    eps = 1e-6
    fd = (cl.gelu(xs + eps) - cl.gelu(xs - eps)) / (2 * eps)
    np.testing.assert_allclose(cl.gelu_grad(xs), fd, rtol=0, atol=1e-9)


def test_conv_backward_is_adjoint():
    """<conv(x), dy> = <x, bwd_data(dy)> and = <w, bwd_weight(x, dy)> (bias-free)."""
    x = _rand(5, (3, 4, 5, 6))
    w = _rand(6, (4, 3, 3, 3, 3))
    dy = _rand(7, (4, 4, 5, 6))
    y = cl.conv3d(x, w, None)
    lhs = float(np.sum(y * dy))
    assert float(np.sum(x * cl.conv3d_bwd_data(dy, w))) == pytest.approx(lhs, rel=1e-12)
    dw, db = cl.conv3d_bwd_weight(x, dy)
    assert float(np.sum(w * dw)) == pytest.approx(lhs, rel=1e-12)
    np.testing.assert_allclose(db, dy.sum(axis=(1, 2, 3)), rtol=1e-13)


def test_closure_gradients_match_finite_differences():
    cin, hidden, shape = 3, 4, (4, 5, 4)
    p = cl.init_params(cin, hidden, seed=9)
    p["w3"] = p["w3"] * 10
    x = _rand(10, (cin,) + shape)
    t = _rand(11, (1,) + shape, 0.3)
    L, g = cl.loss_and_grads(x, t, p)
    rng_idx = synthetic.uniform_ints(12, 0, 10 ** 6, 60)
    eps = 1e-5
    checked = 0
    for k_i, name in enumerate(cl.PARAM_ORDER):
        flat = p[name].reshape(-1)
        for j in range(6):
            idx = int(rng_idx[k_i * 10 + j] % flat.size)
            q = {k: v.copy() for k, v in p.items()}
            q[name].reshape(-1)[idx] += eps
            Lp, _ = cl.mse_loss(cl.forward(x, q)[0], t)
            q[name].reshape(-1)[idx] -= 2 * eps
            Lm, _ = cl.mse_loss(cl.forward(x, q)[0], t)
            fd = (Lp - Lm) / (2 * eps)
            an = g[name].reshape(-1)[idx]
            assert an == pytest.approx(fd, rel=2e-6, abs=1e-11), (name, idx)
            checked += 1
    assert checked == 36


def test_adam_first_steps_are_sign_steps():
    p = {k: np.zeros(3) for k in cl.PARAM_ORDER}
    g = {k: np.array([2.0, -0.5, 1e-3]) for k in cl.PARAM_ORDER}
    st = {}
    lr = 1e-3
    cl.adam_step(p, g, st, lr, 1)
    # m_hat = g, v_hat = g^2 on the first step: update = lr g / (|g| + eps)
    np.testing.assert_allclose(p["w1"], -lr * g["w1"] / (np.abs(g["w1"]) + 1e-8), rtol=1e-12)
    cl.adam_step(p, g, st, lr, 2)  # constant gradient: bias correction keeps the same step
    np.testing.assert_allclose(p["w1"], -2 * lr * g["w1"] / (np.abs(g["w1"]) + 1e-8), rtol=1e-12)
    assert math.isfinite(float(p["b3"][0]))
