"""Plain FP64 reference of the Hermite-leapfrog step with a spatially varying wave speed
(Section 4.2), 1D: p_t + c^2(x) u_x = z(x, t), u_t + p_x = 0 on the periodic unit interval.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU legs, never by the product path.  It shares no code with the CUDA library;
the only operator input is the exact-rational H of ``hermite.py``.

What it computes, in the paper's order (Section 2 for the leapfrog structure, Section 4.2
for the variable coefficient):
  1. gather the partner field's data at the two vertices of the node's cell and build the
     degree-2m+1 Hermite-Birkhoff interpolant (Section 2, eq. interp) as scaled Taylor
     coefficients in xi = (x - x_node)/h;
  2. take c^2 at the node as its local Taylor polynomial of degree 2m+1 with scaled
     coefficients c~_i = h^i/i! d^i c^2 (the pre-processing step of Section 4.2);
  3. run the Cauchy-Kowalevsky recurrence on polynomials of degree 2m+1: with the scaled
     time derivatives P_k = h^k d_t^k p and U_k = h^k d_t^k u (polynomials in xi, D = d/dxi),
         P_(k+1) = -c~ * D U_k + h^(k+1) Z_k,     U_(k+1) = -D P_k,
     where * is the polynomial product kept to degree 2m+1 and Z_k the scaled Taylor
     coefficients of d_t^k z at the node (zero without forcing);
  4. sum the odd-order temporal Taylor terms about the midpoint (Section 2, eq. update1):
         f~(t + dt) = f~(t) + 2 sum_{k odd <= 2m+1} lam^k / k! F_k,    lam = dt/(2h),
     with F = P for the p-half (the interpolant is U_0 = u at the midpoint) and F = U for
     the u-half (the interpolant is P_0 = p at the midpoint), keeping slots 0..m.
The time series stops at order 2m+1, the interpolant's degree: with constant c it is the
full series of the constant-coefficient scheme (the terms beyond vanish there).  Readings
of the garbled formulas: the printed c~_i = h!/i! ... is read as h^i/i!; polynomials in the
recurrence are kept to degree 2m+1.
"""
from __future__ import annotations

from math import factorial

import numpy as np

from .hermite import hermite_inverse


def _interpolant(lower: np.ndarray, upper: np.ndarray, m: int) -> np.ndarray:
    H = np.array(hermite_inverse(m), dtype=np.float64).astype(lower.dtype)  # dyadic: exact
    return np.concatenate([lower, upper], axis=1) @ H.T


def _D(f: np.ndarray) -> np.ndarray:
    """d/dxi of polynomials given by coefficient rows (degree kept)."""
    out = np.zeros_like(f)
    A = f.shape[1]
    out[:, :A - 1] = f[:, 1:] * np.arange(1, A)
    return out


def _mul(c: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Row-wise polynomial product kept to the rows' degree."""
    A = f.shape[1]
    out = np.zeros_like(f)
    for a in range(A):
        for i in range(a + 1):
            out[:, a] += c[:, i] * f[:, a - i]
    return out


def half_step(m: int, h: float, dt: float, mode: int, own: np.ndarray, partner: np.ndarray, c2: np.ndarray,
              forcing=None, t_mid: float = 0.0) -> np.ndarray:
    """One half-step of one field; returns its new (n, m+1) data.

    mode 0 = p-half (own = p on the primal grid at t, partner = u on the dual grid at
    t + dt/2, c2 = Taylor table at the primal nodes); mode 1 = u-half (own = u on the dual
    grid, partner = p on the primal grid at the midpoint, c2 at the dual nodes).
    forcing(k, t) -> (n, 2m+2) scaled Taylor coefficients of d_t^k z at the target nodes."""
    n = own.shape[0]
    A = 2 * m + 2
    lam = own.dtype.type(dt / (2.0 * h))
    if mode == 0:
        lo = (np.arange(n) - 1) % n
    else:
        lo = np.arange(n)
    hi = (lo + 1) % n
    c = _interpolant(partner[lo], partner[hi], m)
    zero = np.zeros((n, A), dtype=own.dtype)

    def Z(k):
        return zero if forcing is None else forcing(k, t_mid)

    inc = np.zeros((n, A), dtype=own.dtype)
    if mode == 0:   # U_0 known; P_k for odd k
        U, P = c, None
        for k in range(0, 2 * m + 1):
            # from order k to order k + 1
            if k % 2 == 0:
                P = -_mul(c2, _D(U)) + own.dtype.type(h) ** (k + 1) * Z(k)   # P_(k+1), k + 1 odd
                inc += 2 * lam ** (k + 1) / factorial(k + 1) * P
            else:
                U = -_D(P)                                     # U_(k+1), k + 1 even
    else:           # P_0 known; U_k for odd k
        P, U = c, None
        for k in range(0, 2 * m + 1):
            if k % 2 == 0:
                U = -_D(P)                                     # U_(k+1), k + 1 odd
                inc += 2 * lam ** (k + 1) / factorial(k + 1) * U
            else:
                P = -_mul(c2, _D(U)) + own.dtype.type(h) ** (k + 1) * Z(k)   # P_(k+1), k + 1 even
    return own + inc[:, :m + 1]


def run(m: int, n: int, dt: float, p: np.ndarray, u: np.ndarray, c2_primal: np.ndarray, c2_dual: np.ndarray,
        n_steps: int, forcing_primal=None, forcing_dual=None, t0: float = 0.0, dtype=np.float64):
    """n_steps leapfrog steps (p-half, then u-half) with the variable wave speed; p (n, m+1)
    at t0 on the primal nodes, u at t0 + dt/2 on the dual nodes; c2 tables (n, 2m+2).
    Returns float64 arrays; dtype=np.longdouble runs the steps in extended precision (the
    reference of long runs)."""
    h = 1.0 / n
    p = np.array(p, dtype=dtype)
    u = np.array(u, dtype=dtype)
    cp = np.array(c2_primal, dtype=dtype)
    cd = np.array(c2_dual, dtype=dtype)
    for st in range(n_steps):
        t = t0 + st * dt
        p = half_step(m, h, dt, 0, p, u, cp, forcing_primal, t + 0.5 * dt)
        u = half_step(m, h, dt, 1, u, p, cd, forcing_dual, t + dt)
    return np.asarray(p, dtype=np.float64), np.asarray(u, dtype=np.float64)
