"""Exact values of a large heat run on a small output box, from the stencil's dependency cone.

Test infrastructure (part of the oracle): no product code imports it.

After k forward-Euler steps (the Section 5.1 listing's update) a point depends
only on the initial field within r*k cells of it along each axis, because each
step reads r neighbours per axis (the read-only halo of Section 2 is as wide as
the stencil radius).  So the oracle advances the input box
[lo - r k, hi + r k) (clipped at the grid's true boundary, where the zero halo
is the real one) by single steps of ``heat_run`` and, after every step, drops
the r cells next to each cut face: those are the cells whose zero halo is an
artefact of the cut.  After k steps the cut faces have reached [lo, hi), and
its values are those of the whole-grid run.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from . import heat_run


def cone_input_box(dims_zyx: Sequence[int], lo: Sequence[int], hi: Sequence[int], reach: int):
    """Input box [in_lo, in_hi) (per axis, slow axis first) for the output box [lo, hi)."""
    in_lo = [max(0, l - reach) for l in lo]
    in_hi = [min(n, h + reach) for n, h in zip(dims_zyx, hi)]
    return in_lo, in_hi


def heat_on_box(initial_box: Callable[[list, list], np.ndarray], dims_zyx: Sequence[int], lo: Sequence[int],
                hi: Sequence[int], so: int, a: float, k: int) -> np.ndarray:
    """Values on [lo, hi) after k heat steps of the whole grid (zero Dirichlet halo).

    initial_box(in_lo, in_hi) returns the initial field on a box of the grid."""
    r = so // 2
    in_lo, in_hi = cone_input_box(dims_zyx, lo, hi, r * k)
    u = np.asarray(initial_box(in_lo, in_hi), dtype=np.float64)
    cur_lo, cur_hi = list(in_lo), list(in_hi)
    for _ in range(k):
        u = heat_run(u, so, a, 1)
        sl = []
        for ax in range(len(dims_zyx)):
            # a face is cut (not the true boundary) while it lies outside the output box
            dl = min(r, lo[ax] - cur_lo[ax]) if cur_lo[ax] > 0 else 0
            dh = min(r, cur_hi[ax] - hi[ax]) if cur_hi[ax] < dims_zyx[ax] else 0
            sl.append(slice(dl, u.shape[ax] - dh))
            cur_lo[ax] += dl
            cur_hi[ax] -= dh
        u = np.ascontiguousarray(u[tuple(sl)])
    # faces on the true boundary were never cut: keep only the output box
    for ax in range(len(dims_zyx)):
        assert (cur_lo[ax] == lo[ax] or cur_lo[ax] == 0) and (cur_hi[ax] == hi[ax] or cur_hi[ax] == dims_zyx[ax])
    sl = tuple(slice(l - cl, h - cl) for l, h, cl in zip(lo, hi, cur_lo))
    return np.ascontiguousarray(u[sl])
