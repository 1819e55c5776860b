"""Oracle: exact finite-difference weights (test infrastructure, not the product).

Central second-derivative weights of accuracy order SO = 2r on the 2r+1 points
m = -r..r.  They are defined by the moment conditions

    sum_{m=-r}^{r} w_m m^k = 2 * [k == 2],   k = 0 .. 2r,

i.e. the stencil differentiates every polynomial of degree <= 2r exactly twice.
This is the standard scheme behind the space orders 2, 4 and 8 the paper
benchmarks (Section 6.1); the paper itself prints no coefficients, so the
oracle solves the moment system exactly over the rationals.  By symmetry
w_{-m} = w_m and the odd moments vanish, leaving r+1 unknowns w_0..w_r and the
r+1 even equations k = 0, 2, .., 2r, solved here by Gaussian elimination with
``fractions.Fraction``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU baseline of ``bench.py``
use this package.
"""
from __future__ import annotations

from fractions import Fraction


def central_weights(so: int) -> list[Fraction]:
    """One-sided list [w_0, w_1, .., w_r] of exact rational weights, r = so/2."""
    if so % 2 or so < 2:
        raise ValueError("space order must be a positive even integer")
    r = so // 2
    n = r + 1
    # Row for moment k = 2e:  [k==0]*w_0 + sum_{m>=1} 2 m^k w_m = 2*[k==2]
    rows = []
    for e in range(n):
        k = 2 * e
        row = [Fraction(1 if k == 0 else 0)]
        row += [Fraction(2 * m ** k) for m in range(1, r + 1)]
        row.append(Fraction(2 if k == 2 else 0))
        rows.append(row)
    # Gauss-Jordan elimination over the rationals
    for col in range(n):
        piv = next(i for i in range(col, n) if rows[i][col] != 0)
        rows[col], rows[piv] = rows[piv], rows[col]
        p = rows[col][col]
        rows[col] = [v / p for v in rows[col]]
        for i in range(n):
            if i != col and rows[i][col] != 0:
                f = rows[i][col]
                rows[i] = [a - f * b for a, b in zip(rows[i], rows[col])]
    return [rows[i][n] for i in range(n)]


def central_weights_f64(so: int) -> list[float]:
    return [float(w) for w in central_weights(so)]


def symbol(weights, theta: float) -> float:
    """Fourier symbol lambda(theta) = w_0 + 2 sum_m w_m cos(m theta) of one axis."""
    import math
    return float(weights[0]) + 2.0 * sum(float(w) * math.cos(m * theta)
                                         for m, w in enumerate(weights) if m > 0)


def symbol_max(weights) -> Fraction:
    """max_theta |lambda(theta)| = |lambda(pi)| = |w_0 + 2 sum_m (-1)^m w_m|."""
    return abs(Fraction(weights[0]) + 2 * sum(Fraction(w) * (-1) ** m
                                               for m, w in enumerate(weights) if m > 0))
