"""Exact 1D Hermite-Birkhoff interpolation matrices for the Hermite-leapfrog oracle.

TEST INFRASTRUCTURE ONLY: the oracle package is imported by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``; the
product path never imports it.

Section 2, eq. (interp): on the cell centred at a node x_j with end points
L = x_j - h/2 and R = x_j + h/2, the interpolant q(xi) = sum_s c_s xi^s,
xi = (x - x_j)/h, of degree 2m+1 matches the scaled derivative data
(h^l/l!) d^l v/dx^l, l = 0..m, at both ends.  The paper writes the
conditions as [C^L; C^R] c = [v^L; v^R] with

    C^L[l][s] = ((L - x_j)/h)^(s-l) * (1/l!) * prod_{t=0}^{l-1} (s - t)   (s >= l)
    C^R[l][s] = ((R - x_j)/h)^(s-l) * (1/l!) * prod_{t=0}^{l-1} (s - t)   (s >= l)

and zero for s < l.  (L - x_j)/h = -1/2 and (R - x_j)/h = +1/2.  The paper
prints the condition index range as 0..2m+1; the data at each end are the
m+1 values l = 0..m (2m+2 conditions in all, matching the 2m+2 unknowns).

The inverse H = [C^L; C^R]^{-1} is computed here in exact rational
arithmetic (Gauss-Jordan on ``fractions.Fraction``) so that the oracle's
operator carries no rounding beyond the final conversion to float.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache


def _falling(s: int, l: int) -> int:
    """prod_{t=0}^{l-1} (s - t): the falling factorial in eq. (interp)."""
    out = 1
    for t in range(l):
        out *= (s - t)
    return out


def _factorial(n: int) -> int:
    out = 1
    for k in range(2, n + 1):
        out *= k
    return out


def interp_system(m: int) -> list[list[Fraction]]:
    """The 2(m+1) x 2(m+1) matrix [C^L; C^R] of Section 2, eq. (interp).

    Rows 0..m are the left-end conditions l = 0..m, rows m+1..2m+1 the
    right-end conditions; column s is the monomial xi^s, s = 0..2m+1.
    """
    if m < 0:
        raise ValueError("m must be >= 0")
    n = 2 * m + 2
    left, right = Fraction(-1, 2), Fraction(1, 2)
    A = [[Fraction(0)] * n for _ in range(n)]
    for l in range(m + 1):
        for s in range(n):
            if s < l:
                continue
            w = Fraction(_falling(s, l), _factorial(l))
            A[l][s] = left ** (s - l) * w
            A[m + 1 + l][s] = right ** (s - l) * w
    return A


@lru_cache(maxsize=None)
def hermite_inverse_exact(m: int) -> tuple[tuple[Fraction, ...], ...]:
    """H = [C^L; C^R]^{-1} in exact rationals (Gauss-Jordan with exact pivots).

    H maps the stacked end data [v^L_0..v^L_m, v^R_0..v^R_m] to the scaled
    Taylor coefficients c_0..c_{2m+1} of the interpolant at the cell centre.
    """
    A = interp_system(m)
    n = len(A)
    aug = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for col in range(n):
        piv = next((r for r in range(col, n) if aug[r][col] != 0), None)
        if piv is None:
            raise ArithmeticError("singular Hermite-Birkhoff system")
        aug[col], aug[piv] = aug[piv], aug[col]
        pv = aug[col][col]
        aug[col] = [x / pv for x in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [a - f * b for a, b in zip(aug[r], aug[col])]
    return tuple(tuple(row[n:]) for row in aug)


def hermite_inverse(m: int) -> list[list[float]]:
    """H as float64 values, rounded once from the exact rationals."""
    return [[float(x) for x in row] for row in hermite_inverse_exact(m)]
