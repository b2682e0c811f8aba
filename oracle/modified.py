"""Plain FP64 reference of the modified Hermite-leapfrog scheme (Section 4.3) for the 1D
pressure-velocity system p_t + u_x = 0, u_t + p_x = 0 on the periodic unit interval.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU legs, never by the product path.  It shares no code with the CUDA
library; the only operator input is the exact-rational H of ``hermite.py``.

What the scheme computes (Section 4.3, eqs. hy1, hy2, lfw1, lfw2, and the pressure-velocity
experiment that follows them):
  * both fields live on both grids: primal nodes x_j = j h hold (p, u) at t_n = n dt,
    dual nodes x_{j+1/2} hold (p, u) at t_{n+1/2} (the modified scheme needs the pressure
    on the dual grid because the Cauchy-Kowalevsky relations exchange even time
    derivatives of p for space derivatives of p, and odd ones for space derivatives of u);
  * a half-step updates every node of one grid from the other grid's data at the midpoint
    time: on the cell around the node (vertices: the two neighbouring nodes of the other
    grid) it builds the degree-2m+1 Hermite-Birkhoff interpolants of p and of u (Section 2,
    eq. interp), and expands each field in time about the midpoint, forward to t + dt and
    backward to t (eqs. option1 and option2), the time derivatives exchanged for space
    derivatives of the interpolants by the relations d_t p = -d_x u, d_t u = -d_x p;
  * even derivative slots take the difference of the two expansions (eq. hy1):
        f~_s(t + dt) =  f~_s(t) + 2 sum_{k odd}  C(s+k, k) lam^k g~_k[s+k]
    odd slots take their sum (eq. lfw2):
        f~_s(t + dt) = -f~_s(t) + 2 sum_{k even} C(s+k, k) lam^k g~_k[s+k]
    where lam = dt/(2h), g~_k is the interpolant whose k-th space derivative equals the
    k-th time derivative of f (p: k even -> p, k odd -> -u; u: k even -> u, k odd -> -p),
    and the sums run over every term with s + k <= 2m + 1 (the full series: beyond that
    degree the interpolants' derivatives vanish).

Readings of the garbled printed formulas: eq. lfw2 prints the space
derivative of order l inside the sum where order i is meant, and its limits 2+l..2m-1 are
read as the full series k = 0, 2, 4, ... with l + k <= 2m + 1 (the k = 0 term is the 2 f~_s
of the midpoint value, without which the sum of the two expansions is not consistent).
"""
from __future__ import annotations

from math import comb

import numpy as np

from .hermite import hermite_inverse


def _interpolant(lower: np.ndarray, upper: np.ndarray, m: int) -> np.ndarray:
    """Scaled Taylor coefficients (nnode, 2m+2) at the cell centre from the end data, in the
    data's precision (H's entries are dyadic rationals, exact in binary64 and wider)."""
    H = np.array(hermite_inverse(m), dtype=np.float64).astype(lower.dtype)
    return np.concatenate([lower, upper], axis=1) @ H.T


def half_step(m: int, lam: float, p_own: np.ndarray, u_own: np.ndarray, p_other: np.ndarray,
              u_other: np.ndarray, lower_offset: int) -> tuple[np.ndarray, np.ndarray]:
    """One half-step of one grid (arrays (n, m+1)): returns the new (p, u) of that grid.

    lower_offset: the other grid's node that is the lower cell vertex of node j is
    j + lower_offset (-1 for the primal update, 0 for the dual update; periodic)."""
    n = p_own.shape[0]
    lo = (np.arange(n) + lower_offset) % n
    hi = (lo + 1) % n
    cp = _interpolant(p_other[lo], p_other[hi], m)
    cu = _interpolant(u_other[lo], u_other[hi], m)
    top = 2 * m + 1

    def source(field: str, k: int) -> np.ndarray:
        # the interpolant whose k-th space derivative is the k-th time derivative of field
        if field == "p":
            return cp if k % 2 == 0 else -cu
        return cu if k % 2 == 0 else -cp

    out = []
    for field, own in (("p", p_own), ("u", u_own)):
        new = np.empty_like(own)
        for s in range(m + 1):
            if s % 2 == 0:      # eq. hy1: forward minus backward expansion, odd k
                acc = own[:, s].copy()
                ks = range(1, top - s + 1, 2)
            else:               # eq. lfw2: forward plus backward expansion, even k
                acc = -own[:, s]
                ks = range(0, top - s + 1, 2)
            for k in ks:
                acc = acc + 2 * comb(s + k, k) * lam ** k * source(field, k)[:, s + k]
            new[:, s] = acc
        out.append(new)
    return out[0], out[1]


def run(m: int, n: int, dt: float, pp: np.ndarray, up: np.ndarray, pd: np.ndarray, ud: np.ndarray,
        n_steps: int, dtype=np.float64):
    """n_steps full steps (primal update, then dual update) on the periodic unit interval
    with n nodes per grid; returns new (pp, up, pd, ud) as float64.  pp, up: primal data at
    t; pd, ud: dual data at t + dt/2; each (n, m+1) scaled derivatives h^a/a! d^a f.
    dtype=np.longdouble runs the same steps in the platform's extended precision, the
    reference of long runs (lam = dt n / 2 is formed in binary64 either way)."""
    lam = dtype(dt * n / 2.0)
    pp, up, pd, ud = (np.array(a, dtype=dtype) for a in (pp, up, pd, ud))
    for _ in range(n_steps):
        pp, up = half_step(m, lam, pp, up, pd, ud, -1)
        pd, ud = half_step(m, lam, pd, ud, pp, up, 0)
    return tuple(np.asarray(a, dtype=np.float64) for a in (pp, up, pd, ud))
