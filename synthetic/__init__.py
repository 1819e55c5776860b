"""Seeded synthetic inputs for the stencil workloads.

This module is shared by the oracle side and the CUDA side of every test and of
the benchmark.  It holds input *recipes* only -- random fields, initial bumps,
velocity models, source positions and batch sizes -- and none of the method's
arithmetic (no stencil weights, no time stepping).  Every array it returns is
float32-exact, so the FP32 device input and the FP64 oracle input are the same
numbers bit for bit.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
i-th draw of stream ``seed`` is ``mix64(key(seed) + (i + 1) * GOLDEN)``, with
``key(seed) = mix64(seed * GOLDEN)``.  The uniform value is the top 24 bits of
the draw divided by 2**24, which is exact in float32.

The workload recipes follow the evaluation of the paper (Section 6.1: heat
diffusion and the isotropic acoustic wave equation in 2D and 3D at space orders
2, 4 and 8, single precision) at the sizes of the five configurations the
library is measured on.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) on a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return mix64(np.array([np.uint64(seed) * GOLDEN], dtype=np.uint64))[0]


def draws_u64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of stream ``seed`` (uint64)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(stream_key(seed) + idx * GOLDEN)


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` float32 values k / 2**24 in [0, 1) from stream ``seed``."""
    top = (draws_u64(seed, start, count) >> np.uint64(40)).astype(np.float64)
    return (top * (1.0 / (1 << 24))).astype(np.float32)


def uniform_field(seed: int, shape: Sequence[int], chunk: int = 1 << 24) -> np.ndarray:
    """Dense field of U[0,1) float32 values; element i (C order) is draw i."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = uniform01(seed, e - s, start=s)
    return out.reshape(tuple(shape))


def uniform_box(seed: int, shape: Sequence[int], lo: Sequence[int], hi: Sequence[int]) -> np.ndarray:
    """The sub-box [lo, hi) (per axis, in the order of ``shape``) of ``uniform_field(seed, shape)``,
    without generating the rest of the field."""
    shape = tuple(int(v) for v in shape)
    lo = [int(v) for v in lo]
    hi = [int(v) for v in hi]
    strides = [int(np.prod(shape[a + 1:])) for a in range(len(shape))]
    sub = tuple(h - l for l, h in zip(lo, hi))
    out = np.empty(sub, dtype=np.float32)
    # linear indices of one leading-axis slice of the box, then shifted per slice
    inner = np.zeros((1,), dtype=np.int64)
    for a in range(1, len(shape)):
        inner = (inner[:, None] + (np.arange(lo[a], hi[a], dtype=np.int64) * strides[a])[None, :]).reshape(-1)
    gold, key = GOLDEN, stream_key(seed)
    for k, i0 in enumerate(range(lo[0], hi[0])):
        idx = (inner + i0 * strides[0] + 1).astype(np.uint64)
        with np.errstate(over="ignore"):
            d = mix64(key + idx * gold)
        out[k] = ((d >> np.uint64(40)).astype(np.float64) * (1.0 / (1 << 24))).astype(np.float32).reshape(sub[1:])
    return out


def uniform_ints(seed: int, lo: int, hi: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` integers uniform in [lo, hi] (inclusive), by floor of U[0,1)."""
    u = uniform01(seed, count, start).astype(np.float64)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def f32(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float32)


# --------------------------------------------------------------------------
# Initial fields
# --------------------------------------------------------------------------

def gaussian_bump_2d(nx: int, ny: int, sigma: float, seed: int) -> np.ndarray:
    """exp(-((x-x0)^2 + (y-y0)^2) / (2 sigma^2)), centre uniform in [3s, N-1-3s].

    Returned as float32 with shape (ny, nx) (x fastest).
    """
    u = uniform01(seed, 2).astype(np.float64)
    x0 = 3 * sigma + u[0] * (nx - 1 - 6 * sigma)
    y0 = 3 * sigma + u[1] * (ny - 1 - 6 * sigma)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    g = np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (2.0 * sigma * sigma))
    return g.astype(np.float32)


def layered_velocity(shape_zyx: Sequence[int], speeds: Sequence[float]) -> np.ndarray:
    """Velocity model of len(speeds) equal layers along z (the slow axis).

    Layer k covers z in [floor(k*Nz/L), floor((k+1)*Nz/L)).  float32, shape as given.
    """
    nz = shape_zyx[0]
    nl = len(speeds)
    c = np.empty(tuple(shape_zyx), dtype=np.float32)
    for k in range(nl):
        z0 = (k * nz) // nl
        z1 = ((k + 1) * nz) // nl
        c[z0:z1] = np.float32(speeds[k])
    return c


def five_layer_speeds() -> list[float]:
    """1500, 2250, 3000, 3750, 4500 m/s (five equal steps, 1500..4500)."""
    return [1500.0 + 750.0 * k for k in range(5)]


def seeded_layer_speeds(seed: int, nlayers: int = 5, cmin: float = 1500.0,
                        cmax: float = 4500.0) -> list[float]:
    """Per-grid layer speeds U[cmin, cmax], sorted with depth, max forced to cmax.

    Forcing the deepest layer to cmax gives every grid of a batch the same
    largest speed, hence the same stable time step.
    """
    u = uniform01(seed, nlayers).astype(np.float64)
    s = sorted(float(np.float32(cmin + (cmax - cmin) * v)) for v in u)
    s[-1] = cmax
    return s


def source_position(seed: int, dims_xyz: Sequence[int], margin: int) -> tuple[int, ...]:
    """Seeded integer grid index at least ``margin`` cells from every boundary."""
    nd = len(dims_xyz)
    u = uniform01(seed, nd, start=1000).astype(np.float64)
    pos = []
    for a in range(nd):
        lo, hi = margin, dims_xyz[a] - 1 - margin
        pos.append(int(lo + math.floor(u[a] * (hi - lo + 1))))
    return tuple(pos)


# --------------------------------------------------------------------------
# Workload recipes (sizes of the measured configurations)
# --------------------------------------------------------------------------

# Von Neumann amplification bound of the standard central second-derivative
# weights, S = max over theta of |sum_m w_m e^{i m theta}| = |sum_m w_m (-1)^m|:
# 4 (order 2), 16/3 (order 4), 2048/315 (order 8).  The configurations are
# specified as fractions of the stability limit, so the recipe needs these
# three numbers; they are checked against the oracle's own weights in tests.
SYMBOL_MAX = {2: 4.0, 4: 16.0 / 3.0, 8: 2048.0 / 315.0}


def heat_a_max(ndim: int, so: int) -> float:
    """Largest stable a = alpha*dt/h^2 of forward Euler: a * ndim * S <= 2."""
    return 2.0 / (ndim * SYMBOL_MAX[so])


def wave_courant_max(ndim: int, so: int) -> float:
    """Largest stable c*dt/h of the leapfrog scheme: (c dt/h)^2 * ndim * S <= 4."""
    return 2.0 / math.sqrt(ndim * SYMBOL_MAX[so])


@dataclasses.dataclass(frozen=True)
class HeatCase:
    ndim: int
    dims: tuple  # (nx, ny[, nz]) interior points, x fastest
    so: int
    a: float  # alpha*dt/h^2
    nsteps: int
    seed: int
    init: str  # "uniform" or "gaussian"

    def initial(self) -> np.ndarray:
        shape = tuple(reversed(self.dims))  # (nz, ny, nx)
        if self.init == "gaussian":
            assert self.ndim == 2
            return gaussian_bump_2d(self.dims[0], self.dims[1], 20.0, self.seed)
        return uniform_field(self.seed, shape)


def heat2d_256() -> HeatCase:
    """2D heat, 256^2, order 2, a = 0.2, Gaussian bump sigma = 20, 100 steps."""
    return HeatCase(2, (256, 256), 2, 0.2, 100, 1, "gaussian")


def heat3d(n: int = 1024, so: int = 8, nsteps: int = 50, seed: int = 2) -> HeatCase:
    """3D heat, n^3, U[0,1) seed 2, a = 0.8 of the stability limit (FP32-rounded)."""
    a = float(np.float32(0.8 * heat_a_max(3, so)))
    return HeatCase(3, (n, n, n), so, a, nsteps, seed, "uniform")


@dataclasses.dataclass(frozen=True)
class WaveCase:
    dims: tuple  # (nx, ny, nz)
    so: int
    h: float
    dt: float
    nsteps: int
    speeds: tuple
    src: tuple  # (sx, sy, sz)
    f0: float
    t0: float
    amp: float

    def velocity(self) -> np.ndarray:
        return layered_velocity(tuple(reversed(self.dims)), self.speeds)


def wave3d(n: int = 768, so: int = 8, nsteps: int = 500, seed: int = 3, f0: float = 10.0,
           speeds: Sequence[float] | None = None, h: float = 10.0, cfl_frac: float = 0.5,
           dims: Sequence[int] | None = None) -> WaveCase:
    """3D acoustic wave: layered velocity, Ricker at a seeded point, dt at cfl_frac of the limit."""
    speeds = tuple(speeds) if speeds is not None else tuple(five_layer_speeds())
    dims = tuple(dims) if dims is not None else (n, n, n)
    cmax = max(speeds)
    dt = cfl_frac * wave_courant_max(3, so) * h / cmax
    src = source_position(seed, dims, margin=so)
    return WaveCase(dims, so, h, dt, nsteps, speeds, src, f0, 1.0 / f0, 1.0)


def batch_wave_cases(count: int = 64, seed: int = 4, lo: int = 96, hi: int = 256, so: int = 4,
                     nsteps: int = 300, h: float = 10.0) -> list[WaveCase]:
    """Batched wave: per-axis sizes U[lo, hi], seeded layers, Ricker f0 U[5, 15] Hz."""
    sizes = uniform_ints(seed, lo, hi, 3 * count).reshape(count, 3)
    f0s = 5.0 + 10.0 * uniform01(seed, count, start=10_000).astype(np.float64)
    cases = []
    for i in range(count):
        sp = seeded_layer_speeds(seed * 1000 + i)
        dims = tuple(int(v) for v in sizes[i])
        cases.append(wave3d(so=so, nsteps=nsteps, seed=seed * 1000 + i, f0=float(np.float32(f0s[i])),
                            speeds=sp, h=h, dims=dims))
    return cases


# --------------------------------------------------------------------------
# The same counter-based generator in torch (for full-size device inputs)
# --------------------------------------------------------------------------

def _signed(u: int) -> int:
    u &= (1 << 64) - 1
    return u - (1 << 64) if u >= (1 << 63) else u


def uniform_field_torch(seed: int, shape: Sequence[int], device, chunk: int = 1 << 26):
    """Bit-identical to :func:`uniform_field`, computed with int64 torch ops on ``device``.

    uint64 arithmetic is emulated on int64: multiplication and addition wrap
    modulo 2**64 identically, and logical right shifts are arithmetic shifts
    masked to the remaining bits.
    """
    import torch
    n = int(np.prod(shape))
    out = torch.empty(n, dtype=torch.float32, device=device)
    key = _signed(int(stream_key(seed)))
    g = _signed(int(GOLDEN))
    m1 = _signed(int(_M1))
    m2 = _signed(int(_M2))

    def lsr(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        z = torch.arange(s + 1, e + 1, dtype=torch.int64, device=device)
        z = z * g + key
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        out[s:e] = lsr(z, 40).to(torch.float32) * (1.0 / (1 << 24))
    return out.reshape(tuple(shape))
