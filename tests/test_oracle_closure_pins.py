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


# ---------------------------------------------------------------------------
# Feature inputs (FP32 stencil features in the library, FP64 here) and the
# rollout gradient (backpropagation through corrected coarse steps)
# ---------------------------------------------------------------------------

def _poly_field(shape, f):
    """f evaluated along x (the fastest axis), broadcast over y, z."""
    x = np.arange(shape[2], dtype=np.float64)
    return np.broadcast_to(f(x)[None, None, :], shape).copy()


def test_feature_channels_on_polynomials():
    """delta^6 x^6 = 720; L x^4 = 12 x^2 and L x^2 = 2 for the order-4 star (exact to degree 5);
    D x = 1, D x^2 = 2x (central difference); away from the zero halo."""
    from oracle import closure as oc
    import oracle
    shape = (11, 12, 20)
    w = oracle.central_weights_f64(4)
    one = np.ones(8)
    inner = (slice(5, 6), slice(5, 7), slice(6, 14))
    c = 0.37
    cn2 = np.full(shape, c)
    # f4 = cn2 sum_a delta^6 u: only the x axis varies
    f = oc.feature_channels(np.zeros(shape), _poly_field(shape, lambda x: x ** 6), cn2, w, one)
    assert np.allclose(f[4][inner], 720.0 * c, rtol=1e-12)
    # f5 = cn2 L(cn2 L u) with u = x^4 and constant cn2: c L(c 12 x^2) = 24 c^2
    f = oc.feature_channels(np.zeros(shape), _poly_field(shape, lambda x: x ** 4), cn2, w, one)
    assert np.allclose(f[5][inner], 24.0 * c * c, rtol=1e-10)
    # f6 = sum_a D_a cn2 D_a u and f7 = |D cn2| L u with cn2 = 3x, u = x^2: 2x * 3, 3 * 2
    cn2x = _poly_field(shape, lambda x: 3.0 * x)
    u2 = _poly_field(shape, lambda x: x ** 2)
    f = oc.feature_channels(np.zeros(shape), u2, cn2x, w, one)
    assert np.allclose(f[6][inner], 6.0 * _poly_field(shape, lambda x: x)[inner], rtol=1e-12)
    assert np.allclose(f[7][inner], 6.0, rtol=1e-12)
    # the pointwise channels and the scales
    up = _poly_field(shape, lambda x: x + 1)
    sc = np.arange(1.0, 9.0)
    f = oc.feature_channels(up, u2, cn2x, w, sc)
    assert np.allclose(f[0], up) and np.allclose(f[1], 2.0 * u2)
    assert np.allclose(f[2], 3.0 * cn2x * up) and np.allclose(f[3], 4.0 * cn2x * u2)


def test_feature_adjoint_is_the_jacobian_transpose():
    """feature_channels is linear in (u+, u^n): its Jacobian, built column by column from unit
    inputs, transposed, must equal feature_channels_adjoint."""
    from oracle import closure as oc
    import oracle
    rng = np.random.default_rng(4)
    shape = (3, 4, 5)
    n = int(np.prod(shape))
    w = oracle.central_weights_f64(4)
    cn2 = rng.uniform(0.2, 1.0, shape)
    sc = rng.uniform(0.5, 2.0, 8)
    J = np.zeros((8 * n, 2 * n))
    for i in range(2 * n):
        e = np.zeros(2 * n)
        e[i] = 1.0
        J[:, i] = oc.feature_channels(e[:n].reshape(shape), e[n:].reshape(shape), cn2, w, sc).reshape(-1)
    dx = rng.standard_normal((8,) + shape)
    g_up, g_un = oc.feature_channels_adjoint(dx, cn2, w, sc)
    want = J.T @ dx.reshape(-1)
    assert np.allclose(g_up.reshape(-1), want[:n], rtol=1e-12, atol=1e-12)
    assert np.allclose(g_un.reshape(-1), want[n:], rtol=1e-12, atol=1e-12)


def test_rollout_gradient_matches_finite_differences():
    from oracle import closure as oc
    import oracle
    rng = np.random.default_rng(3)
    shape = (6, 7, 8)
    w = oracle.central_weights_f64(4)
    p = oc.init_params(8, 16, 7)
    kap = rng.uniform(0.01, 0.06, shape)
    cn2 = rng.uniform(0.2, 1.0, shape)
    u, up = rng.standard_normal(shape), rng.standard_normal(shape)
    refs = [rng.standard_normal(shape) for _ in range(3)]
    sc = rng.uniform(0.5, 2.0, 8)
    _, g = oc.rollout_loss_and_grads(p, u, up, kap, cn2, refs, w, sc, 2.0)
    for key in ("w1", "w2", "w3"):
        v = rng.standard_normal(p[key].shape)
        eps = 1e-5
        pp = {k: x.copy() for k, x in p.items()}
        pm = {k: x.copy() for k, x in p.items()}
        pp[key] = p[key] + eps * v
        pm[key] = p[key] - eps * v
        lp, _ = oc.rollout_loss_and_grads(pp, u, up, kap, cn2, refs, w, sc, 2.0)
        lm, _ = oc.rollout_loss_and_grads(pm, u, up, kap, cn2, refs, w, sc, 2.0)
        fd, an = (lp - lm) / (2 * eps), float(np.sum(g[key] * v))
        assert abs(fd - an) <= 1e-5 * abs(an)


def test_modified_equation_initialisation_is_exact():
    """The library's initial parameters make the FP64 network compute exactly
    a kref f4 / 90 + b kref^2 f5 / 12 (GELU(x) - GELU(-x) = x), whatever the free channels hold."""
    from oracle import closure as oc
    import oracle
    from paper_2404_02218_gb300.closure import modified_equation_params, unflatten_params
    rng = np.random.default_rng(5)
    shape = (9, 10, 11)
    w = oracle.central_weights_f64(4)
    sc = rng.uniform(0.5, 3.0, 8)
    kref, t, a, b = 0.0625, 37.0, 0.9, 0.6
    p = unflatten_params(modified_equation_params(sc, t, kref, a, b).astype(np.float64), cin=8)
    up, un = rng.standard_normal(shape), rng.standard_normal(shape)
    cn2 = rng.uniform(0.2, 1.0, shape)
    x = oc.feature_channels(up, un, cn2, w, sc)
    out, _ = oc.forward(x, p)
    f = oc.feature_channels(up, un, cn2, w, np.ones(8))
    want = a * kref * f[4] / 90.0 + b * kref * kref * f[5] / 12.0
    # the parameters pass through FP32 (flatten_params), so agreement is to FP32 rounding
    assert np.allclose(out[0] / t, want, rtol=1e-5, atol=1e-6 * np.max(np.abs(want)))
