"""Oracle: domain decomposition with dmp.swap halo exchanges (test infrastructure).

Follows the paper's Section 4.2 (the ``dmp`` dialect):

* the global domain is decomposed equally over a Cartesian grid of ranks
  (``#dmp.grid<AxB>``); the split used here gives each rank floor(N/D) points
  and the first N mod D ranks one more;
* every local domain gets a halo as wide as the stencil radius;
* before each stencil load a ``dmp.swap`` exchanges rectangular subsections:
  an ``#dmp.exchange<at A size S source offset O to T>`` receives into the
  region [A, A+S) from the rank at relative position T and, in exchange, sends
  the region [A+O, A+O+S) to that rank (Section 4.2, the exchange-declaration
  figure and its 108x108, halo-4 listing).

Only faces are exchanged: the star stencils read no edge or corner ghosts.
Two steps per exchange (temporal blocking; an extension, the paper swaps before
every step) need halos 2r deep and the edge regions two steps reach: see
:func:`decomposed_heat_run_two_step`.
Coordinates are in memref order (slowest dimension first), matching numpy's
C order for arrays shaped (nz, ny, nx).
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Sequence

import numpy as np


@dataclasses.dataclass(frozen=True)
class Exchange:
    at: tuple
    size: tuple
    source_offset: tuple
    to: tuple


def decompose_extents(n: int, parts: int) -> list[int]:
    """Equal slicing: floor(n/parts) each, plus one for the first n mod parts."""
    base, rem = divmod(n, parts)
    return [base + (1 if i < rem else 0) for i in range(parts)]


def exchanges_for(local_interior: Sequence[int], halo: Sequence[int], grid: Sequence[int],
                  coord: Sequence[int]) -> list[Exchange]:
    """dmp.exchange list of the rank at ``coord`` of ``grid`` (no wrap-around).

    ``local_interior`` and ``halo`` are per dimension (memref order).  The
    memref of the rank is interior + 2*halo in every dimension.
    """
    nd = len(local_interior)
    out = []
    for d in range(nd):
        for direction in (-1, 1):
            nb = coord[d] + direction
            if nb < 0 or nb >= grid[d]:
                continue
            at, size, off, to = [], [], [], []
            for e in range(nd):
                if e == d:
                    at.append(0 if direction < 0 else halo[e] + local_interior[e])
                    size.append(halo[e])
                    off.append(halo[e] if direction < 0 else -halo[e])
                    to.append(direction)
                else:
                    at.append(halo[e])
                    size.append(local_interior[e])
                    off.append(0)
                    to.append(0)
            out.append(Exchange(tuple(at), tuple(size), tuple(off), tuple(to)))
    return out


class _Decomposition:
    """Local padded buffers of every rank plus their exchange lists."""

    def __init__(self, shape: Sequence[int], grid: Sequence[int], r: int):
        self.shape = tuple(shape)
        self.nd = len(shape)
        self.grid = tuple(grid)
        self.r = r
        self.extents = [decompose_extents(shape[d], grid[d]) for d in range(self.nd)]
        self.starts = [np.concatenate([[0], np.cumsum(e)[:-1]]).astype(int) for e in self.extents]
        self.coords = list(itertools.product(*[range(g) for g in grid]))
        self.halo = tuple([r] * self.nd)

    def local_shape(self, c):
        return tuple(self.extents[d][c[d]] for d in range(self.nd))

    def interior_slices(self, c):
        return tuple(slice(self.starts[d][c[d]], self.starts[d][c[d]] + self.extents[d][c[d]])
                     for d in range(self.nd))

    def scatter(self, field: np.ndarray) -> dict:
        bufs = {}
        for c in self.coords:
            ls = self.local_shape(c)
            b = np.zeros(tuple(n + 2 * self.r for n in ls), dtype=np.float64)
            b[tuple(slice(self.r, self.r + n) for n in ls)] = field[self.interior_slices(c)]
            bufs[c] = b
        return bufs

    def gather(self, bufs: dict) -> np.ndarray:
        out = np.zeros(self.shape, dtype=np.float64)
        for c in self.coords:
            ls = self.local_shape(c)
            out[self.interior_slices(c)] = bufs[c][tuple(slice(self.r, self.r + n) for n in ls)]
        return out

    def swap(self, bufs: dict) -> None:
        """Perform every rank's exchanges (receive region <- neighbour's send region)."""
        sends = {}
        for c in self.coords:
            for e in exchanges_for(self.local_shape(c), self.halo, self.grid, c):
                src = tuple(a + o for a, o in zip(e.at, e.source_offset))
                sends[(c, e.to)] = bufs[c][tuple(slice(s, s + n) for s, n in zip(src, e.size))].copy()
        for c in self.coords:
            for e in exchanges_for(self.local_shape(c), self.halo, self.grid, c):
                nb = tuple(ci + ti for ci, ti in zip(c, e.to))
                data = sends[(nb, tuple(-t for t in e.to))]
                bufs[c][tuple(slice(a, a + n) for a, n in zip(e.at, e.size))] = data


def _grid_memref_order(decomp_xyz: Sequence[int], nd: int):
    return tuple(reversed(list(decomp_xyz)[:nd]))


def decomposed_heat_run(u0: np.ndarray, so: int, a: float, nsteps: int,
                        decomp_xyz: Sequence[int], coeffs=None) -> np.ndarray:
    """Heat run on a Cartesian decomposition, swapping halos before every sweep."""
    from . import sweep_heat_padded
    r = so // 2
    u0 = np.asarray(u0, dtype=np.float64)
    nd = u0.ndim
    D = _Decomposition(u0.shape, _grid_memref_order(decomp_xyz, nd), r)
    bufs = D.scatter(u0)
    for _ in range(nsteps):
        D.swap(bufs)
        for c in D.coords:
            dims = tuple(reversed(D.local_shape(c)))
            bufs[c] = sweep_heat_padded(bufs[c], nd, dims, so, a, coeffs)
    return D.gather(bufs)


def decomposed_wave_run(uprev: np.ndarray, u: np.ndarray, kappa: np.ndarray, so: int,
                        nsteps: int, decomp_xyz: Sequence[int], coeffs=None):
    """Source-free leapfrog run on a decomposition; returns (u^{n-1}, u^n) at the end."""
    from . import lib, weights_array, _dims, _dp
    r = so // 2
    u = np.asarray(u, dtype=np.float64)
    nd = u.ndim
    D = _Decomposition(u.shape, _grid_memref_order(decomp_xyz, nd), r)
    P = D.scatter(np.asarray(uprev, dtype=np.float64))
    C = D.scatter(u)
    K = {c: np.ascontiguousarray(np.asarray(kappa, dtype=np.float64)[D.interior_slices(c)])
         for c in D.coords}
    w = weights_array(so, coeffs)
    for _ in range(nsteps):
        D.swap(C)
        N = {}
        for c in D.coords:
            dims = tuple(reversed(D.local_shape(c)))
            out = np.zeros_like(C[c])
            lib().orc_sweep_wave(nd, _dims(dims), r, _dp(w), _dp(K[c]), _dp(C[c]), _dp(P[c]), _dp(out))
            N[c] = out
        P, C = C, N
    return D.gather(P), D.gather(C)


def deep_swap(D: _Decomposition, bufs: dict) -> None:
    """Halo exchange for two steps (halo 2r): one phase per dimension, fastest first;
    a phase exchanges faces 2r deep over the full padded extent of the dimensions of
    earlier phases (their halos are already filled) and the interior of the others,
    so the edge and corner regions arrive from the diagonal neighbours by way of the
    face neighbours."""
    h = D.r
    nd = D.nd
    done = set()
    for d in reversed(range(nd)):  # memref order: the last dimension is x
        sends = {}
        for c in D.coords:
            ls = D.local_shape(c)
            for direction in (-1, 1):
                nb = c[d] + direction
                if nb < 0 or nb >= D.grid[d]:
                    continue
                src = []
                for e in range(nd):
                    if e == d:
                        lo = h if direction < 0 else ls[e]  # first / last h interior layers
                        src.append(slice(lo, lo + h))
                    elif e in done:
                        src.append(slice(0, ls[e] + 2 * h))
                    else:
                        src.append(slice(h, h + ls[e]))
                sends[(c, direction)] = bufs[c][tuple(src)].copy()
        for c in D.coords:
            ls = D.local_shape(c)
            for direction in (-1, 1):
                nb = c[d] + direction
                if nb < 0 or nb >= D.grid[d]:
                    continue
                dst = []
                for e in range(nd):
                    if e == d:
                        lo = 0 if direction < 0 else h + ls[e]
                        dst.append(slice(lo, lo + h))
                    elif e in done:
                        dst.append(slice(0, ls[e] + 2 * h))
                    else:
                        dst.append(slice(h, h + ls[e]))
                ncoord = tuple(ci + (direction if e == d else 0) for e, ci in enumerate(c))
                bufs[c][tuple(dst)] = sends[(ncoord, -direction)]
        done.add(d)


def decomposed_heat_run_two_step(u0: np.ndarray, so: int, a: float, nsteps: int,
                                 decomp_xyz: Sequence[int], coeffs=None) -> np.ndarray:
    """Heat run on a decomposition with two steps per exchange: halos 2r deep, a
    :func:`deep_swap` before every pair of steps, the first step evaluated on the
    interior grown by r (zero outside the global domain), the second on the interior.
    An odd last step runs after a plain swap.  Every step-1 value in a halo is the one
    the neighbour computes for the same point, so the result equals the global run."""
    from . import sweep_heat_padded
    r = so // 2
    u0 = np.asarray(u0, dtype=np.float64)
    nd = u0.ndim
    D = _Decomposition(u0.shape, _grid_memref_order(decomp_xyz, nd), 2 * r)
    bufs = D.scatter(u0)
    left = nsteps
    while left > 0:
        deep_swap(D, bufs)  # (a lone last step reads only the inner r layers of it)
        for c in D.coords:
            ls = D.local_shape(c)
            grown = tuple(n + 2 * r for n in ls)
            # step 1 on interior + r: the padded buffer seen as a grown interior with halo r
            u1 = sweep_heat_padded(bufs[c], nd, tuple(reversed(grown)), so, a, coeffs)
            # zero outside the global domain (sides without a neighbour)
            for d in range(nd):
                if c[d] == 0:
                    sl = [slice(None)] * nd
                    sl[d] = slice(0, 2 * r)
                    u1[tuple(sl)] = 0.0
                if c[d] == D.grid[d] - 1:
                    sl = [slice(None)] * nd
                    sl[d] = slice(2 * r + ls[d], None)
                    u1[tuple(sl)] = 0.0
            if left == 1:
                bufs[c] = u1
                continue
            # step 2 on the interior, from the step-1 field with an r-wide halo
            inner = tuple(slice(r, r + n + 2 * r) for n in ls)
            u2 = sweep_heat_padded(np.ascontiguousarray(u1[inner]), nd, tuple(reversed(ls)), so, a, coeffs)
            out = np.zeros_like(bufs[c])
            out[inner] = u2
            bufs[c] = out
        left -= 2 if left >= 2 else 1
    return D.gather(bufs)
