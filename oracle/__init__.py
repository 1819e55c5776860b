"""FP64 CPU oracle for the stencil sweeps -- test infrastructure, not the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` import this package.  It shares no
code with the CUDA library: its arithmetic lives in ``stencil_oracle.c``
(plain loops, compiled with gcc) and in the numpy helpers below.

What each function follows is cited in its docstring; the paper's section
numbers refer to Bisbas et al., "A shared compilation stack for
distributed-memory parallelism in stencil DSLs" (ASPLOS 2024).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Sequence

import numpy as np

from .weights import central_weights, central_weights_f64, symbol, symbol_max  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.POINTER(ctypes.c_double)
            c_int, c_d, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
            L.orc_padded_size.argtypes = [c_int, i64p, c_int]
            L.orc_padded_size.restype = c_i64
            L.orc_fill_ghosts.argtypes = [c_int, i64p, c_int, c_int, dp]
            L.orc_sweep_heat.argtypes = [c_int, i64p, c_int, dp, c_d, dp, dp]
            L.orc_sweep_wave.argtypes = [c_int, i64p, c_int, dp, dp, dp, dp, dp]
            L.orc_ricker.argtypes = [c_d, c_d, c_d]
            L.orc_ricker.restype = c_d
            L.orc_heat_run.argtypes = [c_int, i64p, c_int, dp, c_d, c_int, dp, c_i64]
            L.orc_heat_run.restype = c_int
            L.orc_system_run.argtypes = [c_int, i64p, c_int, dp, c_int, dp, c_int, dp, c_i64]
            L.orc_system_run.restype = c_int
            L.orc_wave_run.argtypes = [c_int, i64p, c_int, dp, c_int, dp, dp, dp, c_i64, c_i64,
                                       i64p, c_d, c_d, c_d, c_d, c_d]
            L.orc_wave_run.restype = c_int
            L.orc_energy.argtypes = [c_int, i64p, c_int, dp, c_int, dp, dp, dp, dp]
            L.orc_energy.restype = c_int
            L.orc_wave_adjoint.argtypes = [c_int, i64p, c_int, dp, dp, dp, dp, dp]
            L.orc_wave_adjoint.restype = c_int
            L.orc_conv3d_fwd.argtypes = [c_int, c_int, i64p, dp, dp, dp, dp]
            L.orc_conv3d_bwd_data.argtypes = [c_int, c_int, i64p, dp, dp, dp]
            L.orc_conv3d_bwd_weight.argtypes = [c_int, c_int, i64p, dp, dp, dp, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(dims_xyz: Sequence[int]):
    d = list(dims_xyz) + [1] * (3 - len(dims_xyz))
    return (ctypes.c_int64 * 3)(*d)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


BC_ZERO, BC_PERIODIC = 0, 1


def weights_array(so: int, coeffs=None) -> np.ndarray:
    return _f64(coeffs if coeffs is not None else central_weights_f64(so))


# ---------------------------------------------------------------------------
# Time stepping (paper Section 5.1 listing: forward Euler heat; Section 6.1:
# acoustic wave, second order in time)
# ---------------------------------------------------------------------------

def heat_run(u0: np.ndarray, so: int, a: float, nsteps: int, bc: int = BC_ZERO,
             coeffs=None) -> np.ndarray:
    """u^{n+1} = u^n + a L(u^n), nsteps times.  u0 has shape (ny, nx) or (nz, ny, nx)."""
    u = _f64(u0).copy()
    ndim = u.ndim
    dims = tuple(reversed(u.shape))
    w = weights_array(so, coeffs)
    rc = lib().orc_heat_run(ndim, _dims(dims), so // 2, _dp(w), float(a), int(bc), _dp(u), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle heat_run out of memory")
    return u


def system_run(fields: Sequence[np.ndarray], so: int, A, nsteps: int, bc: int = BC_ZERO,
               coeffs=None) -> list:
    """Coupled system (a synthetic multi-stencil sweep): u_k <- u_k + sum_j A[k][j] L(u_j),
    nsteps times, for nf = len(fields) fields of one shape."""
    nf = len(fields)
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(nf, nf))
    u = np.ascontiguousarray(np.stack([_f64(f) for f in fields]))
    ndim = u.ndim - 1
    dims = tuple(reversed(u.shape[1:]))
    w = weights_array(so, coeffs)
    rc = lib().orc_system_run(ndim, _dims(dims), so // 2, _dp(w), nf, _dp(A), int(bc), _dp(u), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle system_run out of memory")
    return [u[k] for k in range(nf)]


def wave_run(uprev: np.ndarray, u: np.ndarray, kappa: np.ndarray, so: int, nsteps: int,
             step0: int = 0, src=None, f0: float = 10.0, t0: float = 0.1, amp: float = 1.0,
             dt: float = 1.0, h: float = 1.0, bc: int = BC_ZERO, coeffs=None):
    """Leapfrog u^{n+1} = 2u^n - u^{n-1} + kappa L(u^n) (+ Ricker source), nsteps times.

    Returns (u^{n-1+nsteps}, u^{n+nsteps}).  kappa = c^2 dt^2 / h^2 per point.
    """
    P = _f64(uprev).copy()
    C = _f64(u).copy()
    K = _f64(kappa)
    ndim = C.ndim
    dims = tuple(reversed(C.shape))
    w = weights_array(so, coeffs)
    srcp = None
    if src is not None:
        s = list(src) + [0] * (3 - len(src))
        srcp = (ctypes.c_int64 * 3)(*s)
    rc = lib().orc_wave_run(ndim, _dims(dims), so // 2, _dp(w), int(bc), _dp(K), _dp(P), _dp(C),
                            int(nsteps), int(step0), srcp, float(f0), float(t0), float(amp),
                            float(dt), float(h))
    if rc != 0:
        raise MemoryError("oracle wave_run out of memory")
    return P, C


def kappa_from_velocity(c: np.ndarray, dt: float, h: float) -> np.ndarray:
    """kappa = c^2 dt^2 / h^2 in FP64."""
    c = _f64(c)
    return c * c * (dt * dt) / (h * h)


def ricker(t, f0: float, t0: float):
    """R(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)."""
    return lib().orc_ricker(float(t), float(f0), float(t0))


def sweep_heat_padded(u_pad: np.ndarray, ndim: int, dims, so: int, a: float, coeffs=None) -> np.ndarray:
    """One heat step on a padded array (ghost width r); returns a new padded array, ghosts 0."""
    w = weights_array(so, coeffs)
    out = np.zeros_like(u_pad)
    lib().orc_sweep_heat(ndim, _dims(dims), so // 2, _dp(w), float(a), _dp(u_pad), _dp(out))
    return out


def wave_step(u: np.ndarray, uprev: np.ndarray, kappa: np.ndarray, so: int, coeffs=None):
    """One source-free leapfrog step (zero ghosts): returns (u^{n+1}, u^n)."""
    P, C = wave_run(uprev, u, kappa, so, 1, coeffs=coeffs)
    return C, P


def wave_step_adjoint(lam_next: np.ndarray, lam_cur: np.ndarray, kappa: np.ndarray, so: int, coeffs=None):
    """Transpose of :func:`wave_step`: cotangents (lam^{n+1}, lam^n) of (u^{n+1}, u^n) to those of
    (u^n, u^{n-1}): (lam^n + 2 lam^{n+1} + L(kappa lam^{n+1}), -lam^{n+1})."""
    A = _f64(lam_next)
    cur = _f64(lam_cur).copy()
    prev = np.empty_like(cur)
    K = _f64(kappa)
    w = weights_array(so, coeffs)
    rc = lib().orc_wave_adjoint(A.ndim, _dims(tuple(reversed(A.shape))), so // 2, _dp(w), _dp(K), _dp(A),
                                _dp(cur), _dp(prev))
    if rc != 0:
        raise MemoryError("oracle wave_step_adjoint out of memory")
    return cur, prev


def energy(u: np.ndarray, uprev: np.ndarray, kappa: np.ndarray, so: int, bc: int = BC_ZERO,
           coeffs=None) -> float:
    """E = sum (u - uprev)^2 / kappa + sum u (A uprev), A = -L (leapfrog discrete energy)."""
    U, P, K = _f64(u), _f64(uprev), _f64(kappa)
    dims = tuple(reversed(U.shape))
    w = weights_array(so, coeffs)
    out = ctypes.c_double(0.0)
    rc = lib().orc_energy(U.ndim, _dims(dims), so // 2, _dp(w), int(bc), _dp(K), _dp(U), _dp(P),
                          ctypes.byref(out))
    if rc != 0:
        raise MemoryError("oracle energy out of memory")
    return out.value


def reduce(u: np.ndarray, kind: str) -> float:
    """FP64 reductions over the interior: 'sum', 'l2sq' (sum of squares), 'maxabs'."""
    x = _f64(u)
    if kind == "sum":
        return float(np.sum(x))
    if kind == "l2sq":
        return float(np.sum(x * x))
    if kind == "maxabs":
        return float(np.max(np.abs(x))) if x.size else 0.0
    raise ValueError(kind)


def max_rel_error(got: np.ndarray, ref: np.ndarray) -> float:
    """max_p |got - ref| / max_p |ref| over interior points."""
    g = np.asarray(got, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(r)))
    return float(np.max(np.abs(g - r))) / (den if den > 0 else 1.0)


def rel_l2_error(got: np.ndarray, ref: np.ndarray) -> float:
    g = np.asarray(got, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    den = float(np.linalg.norm(r))
    return float(np.linalg.norm(g - r)) / (den if den > 0 else 1.0)


from .decomp import (Exchange, decompose_extents, exchanges_for,  # noqa: E402,F401
                     decomposed_heat_run, decomposed_heat_run_two_step, decomposed_wave_run)
from . import closure  # noqa: E402,F401
