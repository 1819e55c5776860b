"""Oracle: brute-force dense-matrix reference for tiny grids (test infrastructure).

Builds the star-stencil operator L of the paper's finite-difference update
(Section 2: a point depends on its neighbours at the previous time step; the
halo is read-only) as an explicit dense matrix over the interior points, with
zero ghosts (Dirichlet) or wrap-around (periodic), and advances the state by
matrix products:

    heat:  u^n = (I + a L)^n u^0
    wave:  [u^{n+1}; u^n] = [[2I + K L, -I], [I, 0]] [u^n; u^{n-1}] + source

This shares nothing with the loop code in ``stencil_oracle.c``: it is an
independent construction used to pin the oracle on grids of <= ~1000 points.
"""
from __future__ import annotations

import itertools

import numpy as np


def laplacian_matrix(shape_zyx, weights, periodic: bool = False) -> np.ndarray:
    """Dense L over interior points (C order of ``shape_zyx``), weights = [w_0..w_r]."""
    shape = tuple(shape_zyx)
    nd = len(shape)
    npts = int(np.prod(shape))
    r = len(weights) - 1
    L = np.zeros((npts, npts), dtype=np.float64)
    strides = [int(np.prod(shape[d + 1:])) for d in range(nd)]
    for idx in itertools.product(*[range(n) for n in shape]):
        row = sum(i * s for i, s in zip(idx, strides))
        for d in range(nd):
            for m in range(-r, r + 1):
                q = list(idx)
                q[d] += m
                if periodic:
                    q[d] %= shape[d]
                elif q[d] < 0 or q[d] >= shape[d]:
                    continue  # zero ghost
                col = sum(i * s for i, s in zip(q, strides))
                L[row, col] += float(weights[abs(m)])
    return L


def heat_brute(u0: np.ndarray, weights, a: float, nsteps: int, periodic: bool = False) -> np.ndarray:
    L = laplacian_matrix(u0.shape, weights, periodic)
    M = np.eye(L.shape[0]) + a * L
    v = np.asarray(u0, dtype=np.float64).reshape(-1)
    for _ in range(nsteps):
        v = M @ v
    return v.reshape(u0.shape)


def wave_brute(uprev: np.ndarray, u: np.ndarray, kappa: np.ndarray, weights, nsteps: int,
               periodic: bool = False, src_flat: int | None = None, src_values=None):
    """Block recurrence; src_values[s] is added at flat index src_flat to u^{n+1} of step s."""
    L = laplacian_matrix(u.shape, weights, periodic)
    K = np.diag(np.asarray(kappa, dtype=np.float64).reshape(-1))
    n = L.shape[0]
    T = np.block([[2.0 * np.eye(n) + K @ L, -np.eye(n)], [np.eye(n), np.zeros((n, n))]])
    state = np.concatenate([np.asarray(u, dtype=np.float64).reshape(-1),
                            np.asarray(uprev, dtype=np.float64).reshape(-1)])
    for s in range(nsteps):
        state = T @ state
        if src_flat is not None:
            state[src_flat] += src_values[s]
    return state[n:].reshape(u.shape), state[:n].reshape(u.shape)
