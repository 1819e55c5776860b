"""Oracle: the learned 3D-convolution closure in FP64 (test infrastructure).

The paper has no learned component; this is the plain definition of the
network the library trains on the GPU, used to check its forward pass, its
gradients and its optimiser step:

    z1 = conv1(x) + b1,  y1 = GELU(z1)       (C_in -> H channels, 3x3x3, zero padding)
    z2 = conv2(y1) + b2, y2 = GELU(z2)       (H -> H)
    out = conv3(y2) + b3                      (H -> 1)

GELU is the exact form x * Phi(x) = x/2 (1 + erf(x / sqrt 2)) (Hendrycks and
Gimpel, 2016).  The loss is the mean squared error over all points.  Adam
follows Kingma and Ba (2015), Algorithm 1, with bias correction.

Arrays are channel-major: x[c][z][y][x]; weights w[co][ci][dz][dy][dx].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import lib, _dims, _dp


def gelu(x: np.ndarray) -> np.ndarray:
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * phi


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def conv3d(x: np.ndarray, w: np.ndarray, b: np.ndarray | None) -> np.ndarray:
    """y[co] = b[co] + sum_ci sum_taps w[co][ci][t] x[ci][p + t], zero outside."""
    x, w = _c(x), _c(w)
    cin, nz, ny, nx = x.shape
    cout = w.shape[0]
    assert w.shape == (cout, cin, 3, 3, 3)
    y = np.zeros((cout, nz, ny, nx), dtype=np.float64)
    bb = _c(b) if b is not None else None
    lib().orc_conv3d_fwd(cin, cout, _dims((nx, ny, nz)), _dp(x), _dp(w),
                         _dp(bb) if bb is not None else None, _dp(y))
    return y


def conv3d_bwd_data(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    dy, w = _c(dy), _c(w)
    cout, nz, ny, nx = dy.shape
    cin = w.shape[1]
    dx = np.zeros((cin, nz, ny, nx), dtype=np.float64)
    lib().orc_conv3d_bwd_data(cin, cout, _dims((nx, ny, nz)), _dp(dy), _dp(w), _dp(dx))
    return dx


def conv3d_bwd_weight(x: np.ndarray, dy: np.ndarray):
    x, dy = _c(x), _c(dy)
    cin, nz, ny, nx = x.shape
    cout = dy.shape[0]
    dw = np.zeros((cout, cin, 3, 3, 3), dtype=np.float64)
    db = np.zeros((cout,), dtype=np.float64)
    lib().orc_conv3d_bwd_weight(cin, cout, _dims((nx, ny, nz)), _dp(x), _dp(dy), _dp(dw), _dp(db))
    return dw, db


def init_params(cin: int, hidden: int, seed: int) -> dict:
    """Seeded uniform init with bound 1/sqrt(fan_in) (the usual conv default), last layer small."""
    import synthetic
    p = {}
    shapes = [("w1", (hidden, cin, 3, 3, 3)), ("b1", (hidden,)),
              ("w2", (hidden, hidden, 3, 3, 3)), ("b2", (hidden,)),
              ("w3", (1, hidden, 3, 3, 3)), ("b3", (1,))]
    off = 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        fan_in = (cin if name in ("w1", "b1") else hidden) * 27
        bound = 1.0 / math.sqrt(fan_in)
        if name in ("w3", "b3"):
            bound *= 0.1
        u = synthetic.uniform01(seed, n, start=off).astype(np.float64)
        p[name] = np.float32((2.0 * u - 1.0) * bound).astype(np.float64).reshape(shp)
        off += n
    return p


PARAM_ORDER = ("w1", "b1", "w2", "b2", "w3", "b3")


def forward(x: np.ndarray, p: dict):
    z1 = conv3d(x, p["w1"], p["b1"])
    y1 = gelu(z1)
    z2 = conv3d(y1, p["w2"], p["b2"])
    y2 = gelu(z2)
    out = conv3d(y2, p["w3"], p["b3"])
    return out, dict(x=_c(x), z1=z1, y1=y1, z2=z2, y2=y2)


def backward(cache: dict, dout: np.ndarray, p: dict) -> dict:
    g = {}
    g["w3"], g["b3"] = conv3d_bwd_weight(cache["y2"], dout)
    dy2 = conv3d_bwd_data(dout, p["w3"])
    dz2 = dy2 * gelu_grad(cache["z2"])
    g["w2"], g["b2"] = conv3d_bwd_weight(cache["y1"], dz2)
    dy1 = conv3d_bwd_data(dz2, p["w2"])
    dz1 = dy1 * gelu_grad(cache["z1"])
    g["w1"], g["b1"] = conv3d_bwd_weight(cache["x"], dz1)
    return g


def mse_loss(out: np.ndarray, target: np.ndarray):
    """L = mean (out - target)^2; returns (L, dL/dout)."""
    d = _c(out) - _c(target)
    n = d.size
    return float(np.sum(d * d) / n), 2.0 * d / n


def loss_and_grads(x: np.ndarray, target: np.ndarray, p: dict):
    out, cache = forward(x, p)
    L, dout = mse_loss(out, target)
    return L, backward(cache, dout, p)


def adam_step(p: dict, g: dict, state: dict, lr: float, t: int, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place (t is the 1-based step count)."""
    for k in PARAM_ORDER:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1.0 - beta1) * g[k]
        v[...] = beta2 * v + (1.0 - beta2) * g[k] * g[k]
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


# ---------------------------------------------------------------------------
# Input features of the closure, computed from the fields in FP64 (the library
# computes them in FP32 before rounding to the network's BF16 inputs).  The
# paper has no learned part; these follow the modified-equation view of the
# leapfrog scheme: for u_tt = c^2 Lap(u) the scheme's one-step defect is, to
# leading order, kappa/90 sum_a d^6u/dx_a^6 (the order-4 star's truncation) plus
# kappa L(kappa L u)/12 (the leapfrog's dt^4 u_tttt / 12 term); where the
# velocity jumps, grad(kappa).grad(u) and |grad kappa| L u carry the local
# coupling.  All vanish with the field.  cn2 = (c / c_ref)^2 stands in for kappa
# (kappa = kappa_ref cn2; the constant goes into the channel scale).
# ---------------------------------------------------------------------------

SIXTH_DIFFERENCE = (-20.0, 15.0, -6.0, 1.0)  # per-axis weights of delta^6, w_0 .. w_3


def shifted(u: np.ndarray, ax: int, m: int) -> np.ndarray:
    """v[p] = u[p + m e_ax], zero outside the array (the zero halo)."""
    u = _c(u)
    out = np.zeros_like(u)
    n = u.shape[ax]
    if abs(m) >= n:
        return out
    src = [slice(None)] * u.ndim
    dst = [slice(None)] * u.ndim
    if m >= 0:
        src[ax], dst[ax] = slice(m, n), slice(0, n - m)
    else:
        src[ax], dst[ax] = slice(0, n + m), slice(-m, n)
    out[tuple(dst)] = u[tuple(src)]
    return out


def star(u: np.ndarray, w) -> np.ndarray:
    """sum over axes, sum over m = -r..r of w_|m| u[p + m e_axis]  (w = w_0 .. w_r)."""
    u = _c(u)
    out = u.ndim * w[0] * u
    for ax in range(u.ndim):
        for m in range(1, len(w)):
            out = out + w[m] * (shifted(u, ax, m) + shifted(u, ax, -m))
    return out


def central_difference(u: np.ndarray, ax: int) -> np.ndarray:
    """(u[p + e_ax] - u[p - e_ax]) / 2."""
    return 0.5 * (shifted(u, ax, 1) - shifted(u, ax, -1))


def feature_channels(up: np.ndarray, un: np.ndarray, cn2: np.ndarray, weights, scales) -> np.ndarray:
    """The 8 input channels x[k] = scales[k] f_k of the closure:
    f0 = u+, f1 = u^n, f2 = cn2 u+, f3 = cn2 u^n, f4 = cn2 sum_a delta_a^6 u^n,
    f5 = cn2 L(cn2 L u^n), f6 = sum_a D_a(cn2) D_a(u^n), f7 = (sum_a |D_a cn2|) L u^n
    (L the grid's star with the given weights, D_a the central difference)."""
    up, un, cn2 = _c(up), _c(un), _c(cn2)
    Lu = star(un, weights)
    grads = [central_difference(cn2, a) for a in range(un.ndim)]
    f = [up, un, cn2 * up, cn2 * un, cn2 * star(un, SIXTH_DIFFERENCE), cn2 * star(cn2 * Lu, weights),
         sum(g * central_difference(un, a) for a, g in enumerate(grads)), sum(np.abs(g) for g in grads) * Lu]
    return np.stack([s * v for s, v in zip(scales, f)])


def feature_channels_adjoint(dx: np.ndarray, cn2: np.ndarray, weights, scales):
    """Transpose of feature_channels: the cotangents dx[k] of x[k] to those of (u+, u^n).
    Uses that star() is symmetric and D_a antisymmetric under the zero halo."""
    dx, cn2 = _c(dx), _c(cn2)
    grads = [central_difference(cn2, a) for a in range(cn2.ndim)]
    gabs = sum(np.abs(g) for g in grads)
    d = [scales[k] * dx[k] for k in range(8)]
    g_up = d[0] + cn2 * d[2]
    g_un = d[1] + cn2 * d[3] + star(cn2 * d[4], SIXTH_DIFFERENCE)
    g_un = g_un + star(cn2 * star(cn2 * d[5], weights), weights)
    g_un = g_un - sum(central_difference(g * d[6], a) for a, g in enumerate(grads))
    g_un = g_un + star(gabs * d[7], weights)
    return g_up, g_un


def backward_with_input(cache: dict, dout: np.ndarray, p: dict):
    """backward() plus the cotangent of the network input x."""
    g = {}
    g["w3"], g["b3"] = conv3d_bwd_weight(cache["y2"], dout)
    dy2 = conv3d_bwd_data(dout, p["w3"])
    dz2 = dy2 * gelu_grad(cache["z2"])
    g["w2"], g["b2"] = conv3d_bwd_weight(cache["y1"], dz2)
    dy1 = conv3d_bwd_data(dz2, p["w2"])
    dz1 = dy1 * gelu_grad(cache["z1"])
    g["w1"], g["b1"] = conv3d_bwd_weight(cache["x"], dz1)
    return g, conv3d_bwd_data(dz1, p["w1"])


def corrected_step(u: np.ndarray, uprev: np.ndarray, kappa: np.ndarray, cn2: np.ndarray, p: dict, weights,
                   scales, out_scale: float):
    """One source-free coarse step with the closure: u+ = 2u - uprev + kappa L u (Section 6.1's
    scheme), u^{n+1} = u+ + net(x(u+, u)) / out_scale.  Returns (u^{n+1}, u+, cache)."""
    up = 2.0 * _c(u) - _c(uprev) + _c(kappa) * star(u, weights)
    x = feature_channels(up, u, cn2, weights, scales)
    out, cache = forward(x, p)
    return up + out[0] / out_scale, up, cache


def rollout_loss_and_grads(p: dict, u_cur, u_prev, kappa, cn2, refs, weights, scales, out_scale: float):
    """FP64 reference of the rollout training gradient: len(refs) corrected steps from
    (u^{n0}, u^{n0-1}) = (u_cur, u_prev), loss = mean_j |u^{n0+j+1} - refs[j]|^2 / |refs[j]|^2,
    gradient w.r.t. every parameter by backpropagation through the steps (chain rule written
    out: network backward, feature transpose, leapfrog transpose)."""
    K = len(refs)
    us, ups, caches = [_c(u_prev), _c(u_cur)], [], []
    for j in range(K):
        un, up, cache = corrected_step(us[-1], us[-2], kappa, cn2, p, weights, scales, out_scale)
        us.append(un)
        ups.append(up)
        caches.append(cache)
    loss = 0.0
    glev = []  # dLoss/du^{n0+j+1} from its own loss term
    for j in range(K):
        d = us[j + 2] - refs[j]
        nr = float(np.sum(_c(refs[j]) ** 2))
        loss += float(np.sum(d * d)) / nr / K
        glev.append(2.0 * d / nr / K)
    grads = {k: np.zeros_like(p[k]) for k in PARAM_ORDER}
    lam = {K + 1: glev[K - 1].copy()}  # cotangent of level index (j + 1) -> us[j + 1]
    if K >= 2:
        lam[K] = glev[K - 2].copy()
    w = list(weights)
    for j in range(K - 1, -1, -1):
        a = lam[j + 2]                         # cotangent of u^{n0+j+1} = us[j + 2]
        g, dx = backward_with_input(caches[j], (a / out_scale)[None], p)
        for k in PARAM_ORDER:
            grads[k] += g[k]
        g_up, g_un = feature_channels_adjoint(dx, cn2, w, scales)
        A = a + g_up                           # cotangent of u+
        if j == 0:
            break
        # u+ = 2 u^n - u^{n-1} + kappa L u^n
        lam[j + 1] = lam[j + 1] + 2.0 * A + star(_c(kappa) * A, w) + g_un
        lam[j] = -A + (glev[j - 2] if j >= 2 else 0.0)
    return loss, grads
