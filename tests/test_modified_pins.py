"""Pins of the modified Hermite-leapfrog oracle (Section 4.3, oracle/modified.py) against what
the paper and the mathematics fix: exact evolution of polynomial data by d'Alembert's formula,
the convergence rates of Table 4, stability of the step at the paper's Courant numbers, and the
difference from the unmodified scheme (which the slot-parity rule must produce)."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

from oracle import modified as MO
from paper_1808_10481_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table4():
    out = {}
    with open(os.path.join(GOLDEN, "table4_rates.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                m, cfl, r = line.split()
                out[(int(m), float(cfl))] = float(r)
    return out


def _scaled_poly_data(coef, x, h, m):
    """Scaled derivatives h^a/a! d^a q(x) of the polynomial with monomial coefficients coef."""
    P = np.polynomial.Polynomial(coef)
    out = np.empty((np.size(x), m + 1))
    for a in range(m + 1):
        out[:, a] = P.deriv(a)(x) * h ** a / math.factorial(a) if a else P(x)
    return out


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
def test_primal_update_is_exact_for_polynomial_data(m):
    """For p and u polynomials of degree 2m+1 the update reproduces the exact solution:
    with w = p + u moving right and z = p - u moving left (d'Alembert), p(x, t) =
    (w0(x - t) + z0(x + t))/2 and u = (w0(x - t) - z0(x + t))/2, evaluated by numpy's
    polynomial arithmetic, an independent route to the same numbers."""
    rng = np.random.default_rng(40 + m)
    n, deg = 12, 2 * m + 1
    h = 1.0 / n
    dt = 0.9 * h
    w0 = rng.uniform(-1, 1, deg + 1)
    z0 = rng.uniform(-1, 1, deg + 1)

    def fields(x, t):
        W = np.polynomial.Polynomial(w0)
        Z = np.polynomial.Polynomial(z0)
        def shift(Q, s):  # the polynomial x -> Q(x + s), by composition
            return Q(np.polynomial.Polynomial([s, 1.0]))
        Pp = (shift(W, -t) + shift(Z, t)) / 2
        Pu = (shift(W, -t) - shift(Z, t)) / 2
        return _scaled_poly_data(Pp.coef, x, h, m), _scaled_poly_data(Pu.coef, x, h, m)

    # one primal node j = 5 away from the periodic seam: only dual nodes 4 and 5 enter
    xp = np.arange(n) * h
    xd = (np.arange(n) + 0.5) * h
    pp, up = fields(xp, 0.0)
    pd, ud = fields(xd, 0.5 * dt)
    p1, u1 = MO.half_step(m, dt / (2 * h), pp, up, pd, ud, -1)
    pe, ue = fields(xp, dt)
    scale = max(np.abs(pe).max(), np.abs(ue).max())
    np.testing.assert_allclose(p1[5], pe[5], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(u1[5], ue[5], rtol=0, atol=1e-12 * scale)


def _rate(m, cfl, Ns=(16, 24, 32, 48, 64), T=4.13 / 2, wave=3):
    errs = []
    for N in Ns:
        steps = math.ceil(T / (cfl / N))
        dt = T / steps
        st = I.standing_mode_1d_both_grids(m, N, dt, wave)
        pp, _, _, _ = MO.run(m, N, dt, *st, steps)
        ex = I.standing_mode_1d_both_grids(m, N, dt, wave, t0=steps * dt)
        errs.append(math.sqrt(np.sum((pp[:, 0] - ex[0][:, 0]) ** 2) / N))
    return float(np.polyfit(np.log(1.0 / np.array(Ns)), np.log(errs), 1)[0])


@pytest.mark.parametrize("cfl", [0.9, 0.5, 0.1])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_convergence_rate_matches_table4(m, cfl):
    """The paper's experiment (p = cos(3 pi t) sin(3 pi x) on [-1, 1], T = 4.13, here mapped
    to the unit interval: wave number 3, T = 4.13/2): the observed rate is 2m + 2 at every
    Courant number, within 0.35 of Table 4."""
    paper = _table4()[(m, cfl)]
    got = _rate(m, cfl)
    assert abs(got - paper) <= 0.35, (m, cfl, got, paper)


def test_odd_slots_use_the_sum_of_the_expansions():
    """Replacing the sum rule of the odd slots by the difference rule (the unmodified scheme's
    update) must lose the uniform 2m + 2 rate at m = 1 (Table 4 against Table 1: 4 against 2)."""
    orig = MO.half_step

    def all_difference(m, lam, p_own, u_own, p_other, u_other, lower_offset):
        n = p_own.shape[0]
        lo = (np.arange(n) + lower_offset) % n
        hi = (lo + 1) % n
        cp = MO._interpolant(p_other[lo], p_other[hi], m)
        cu = MO._interpolant(u_other[lo], u_other[hi], m)
        res = []
        for own, src in ((p_own, -cu), (u_own, -cp)):
            new = own.copy()
            for s in range(m + 1):
                for k in range(1, 2 * m + 2 - s, 2):
                    new[:, s] += 2.0 * math.comb(s + k, k) * lam ** k * src[:, s + k]
            res.append(new)
        return res[0], res[1]

    try:
        MO.half_step = all_difference
        plain = _rate(1, 0.9)
    finally:
        MO.half_step = orig
    assert plain < 3.0 and _rate(1, 0.9) > 3.7


@pytest.mark.parametrize("m", [1, 2, 3])
def test_step_is_stable_at_the_papers_courant_numbers(m):
    """Spectral radius of the assembled full step (primal then dual update) on a periodic
    grid of 10 nodes: at most 1 (to rounding and the defective eigenvalue 1 of periodic slope
    data) for C_CFL = 0.9, 0.5 and 0.1."""
    n = 10
    nst = 4 * (m + 1) * n
    for cfl in (0.9, 0.5, 0.1):
        dt = cfl / n
        A = np.empty((nst, nst))
        for c in range(nst):
            e = np.zeros(nst)
            e[c] = 1.0
            parts = [e[i * n * (m + 1):(i + 1) * n * (m + 1)].reshape(n, m + 1) for i in range(4)]
            out = MO.run(m, n, dt, *parts, 1)
            A[:, c] = np.concatenate([o.ravel() for o in out])
        rho = float(np.abs(np.linalg.eigvals(A)).max())
        assert rho <= 1.0 + 1e-5, (m, cfl, rho)
