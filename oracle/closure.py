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
