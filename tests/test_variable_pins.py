"""Pins of the variable-wave-speed oracle (Section 4.2, oracle/variable.py) against what the
paper and the mathematics fix: it reduces to the constant-speed oracle when c^2 = 1; its
Cauchy-Kowalevsky recurrence reproduces, for polynomial data and a linear c^2, the exact
local time series that sympy obtains by differentiating the PDE symbolically; and the
manufactured-solution experiment of Section 4.2 converges at the rates of Table 2."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from oracle import variable as V
from paper_1808_10481_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table2():
    out = {}
    with open(os.path.join(GOLDEN, "table2_rates.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                m, cfl, r = line.split()
                out[(int(m), float(cfl))] = float(r)
    return out


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
def test_unit_speed_is_the_constant_coefficient_oracle(m):
    n = 19
    dt = 0.9 / n
    st = I.random_state(1, m, [n], seed=300 + m)
    ones = np.zeros((n, 2 * m + 2))
    ones[:, 0] = 1.0
    p, u = V.run(m, n, dt, st.p, st.u[0], ones, ones, 7)
    po, uo = oracle.run(1, m, [n], dt, st.p, st.u, 7)
    np.testing.assert_allclose(p, po, rtol=0, atol=1e-12 * np.abs(po).max())
    np.testing.assert_allclose(u, uo[0], rtol=0, atol=1e-12 * np.abs(uo).max())


@pytest.mark.parametrize("m", [2, 3])
def test_recurrence_matches_symbolic_time_series(m):
    """Polynomial u (degree 3) about a primal node and c^2 = 1 + a x (linear): no product
    reaches degree 2m+1, so the recurrence is the exact local evolution.  sympy differentiates
    p_t = -c^2 u_x, u_t = -p_x in time (exchanging for space derivatives) and sums the odd
    temporal Taylor terms about the midpoint; the oracle's p-half increment at the node must
    agree for every slot."""
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    n, h = 16, sp.Rational(1, 16)
    dt = sp.Rational(9, 10) * h
    alpha = sp.Rational(3, 10)
    c2 = 1 + alpha * x
    u0 = sp.Rational(1, 3) - 2 * x + 5 * x ** 2 + 7 * x ** 3     # u about the primal node x = 0
    # time derivatives of p at the node from u at the midpoint: P_1 = -c2 u', U_2 = -P_1', ...
    U = u0
    total = 0
    for k in range(1, 2 * m + 2, 2):
        P = -c2 * sp.diff(U, x)
        total += 2 * (dt / 2) ** k / sp.factorial(k) * P
        U = -sp.diff(P, x)
    want = [float(sp.diff(total, x, s).subs(x, 0) * h ** s / sp.factorial(s)) for s in range(m + 1)]
    # the oracle sees the same u through its scaled nodal data at the dual nodes -1/2, +1/2 (x in units of h)
    A = 2 * m + 2
    data = np.zeros((n, m + 1))
    for j, xc in ((n - 1, -h / 2), (0, h / 2)):
        data[j] = [float(sp.diff(u0, x, a).subs(x, xc) * h ** a / sp.factorial(a)) for a in range(m + 1)]
    c2tab = np.zeros((n, A))
    c2tab[:, 0] = 1.0
    c2tab[0, 0], c2tab[0, 1] = 1.0, float(alpha * h)               # c^2 about the node x = 0
    p0 = np.zeros((n, m + 1))
    got = V.half_step(m, float(h), float(dt), 0, p0, data, c2tab)[0]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("cfl", [0.9, 0.5, 0.1])
@pytest.mark.parametrize("m", [0, 1, 2, 3])
def test_convergence_rate_matches_table2(m, cfl):
    """The paper's experiment (c^2 = 1 + sin(x)/2 on [0, 2 pi], p = sin(x - t), T = 3.2) on
    the unit interval, dt = C_CFL h / c_max: rates within 0.35 of Table 2."""
    T = 3.2 / (2 * math.pi)
    Ns = [16, 24, 32, 48, 64]
    errs = []
    for N in Ns:
        steps = math.ceil(T / (cfl / N / I.c2_max()))
        dt = T / steps
        p, u, fp, fd = I.variable_speed_wave(m, N, dt)
        p, u = V.run(m, N, dt, p, u, I.c2_taylor_table(N, m, False), I.c2_taylor_table(N, m, True), steps, fp, fd)
        ex = np.sin(2 * math.pi * (np.arange(N) / N - steps * dt))
        errs.append(math.sqrt(np.sum((p[:, 0] - ex) ** 2) / N))
    got = float(np.polyfit(np.log(1.0 / np.array(Ns)), np.log(errs), 1)[0])
    assert abs(got - _table2()[(m, cfl)]) <= 0.35, (m, cfl, got)


def test_wrong_speed_table_breaks_convergence():
    """Planting c^2 = 1 in place of the varying speed (the forcing kept) must destroy the
    agreement with the manufactured solution."""
    m, N = 2, 32
    T = 3.2 / (2 * math.pi)
    steps = math.ceil(T / (0.9 / N / I.c2_max()))
    dt = T / steps
    p, u, fp, fd = I.variable_speed_wave(m, N, dt)
    ones = np.zeros((N, 2 * m + 2))
    ones[:, 0] = 1.0
    pw, _ = V.run(m, N, dt, p, u, ones, ones, steps, fp, fd)
    pr, _ = V.run(m, N, dt, p, u, I.c2_taylor_table(N, m, False), I.c2_taylor_table(N, m, True), steps, fp, fd)
    ex = np.sin(2 * math.pi * (np.arange(N) / N - steps * dt))
    assert np.abs(pw[:, 0] - ex).max() > 1e3 * np.abs(pr[:, 0] - ex).max()
