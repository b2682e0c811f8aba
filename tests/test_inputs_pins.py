"""Pins of the seeded input generators (paper_1808_10481_gb300/inputs.py) against symbolic
derivatives.  Both the oracle and the CUDA path start from these arrays, so parity between
them cannot catch an error here; sympy differentiates the analytic fields independently.

Each slot holds the scaled derivative prod_k h_k^{a_k}/a_k! d^a f (slot index a_0 fastest,
node index x fastest), with p at t = 0 and u at t = dt/2."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from paper_1808_10481_gb300 import inputs as I

sp = pytest.importorskip("sympy")

X = sp.symbols("x0:3", real=True)
T = sp.Symbol("t", real=True)


def _scaled_slots(expr, d, m, hs, point, t):
    """All (m+1)^d scaled derivatives of expr at point and time t, in slot order."""
    subs = {X[k]: sp.Float(point[k], 30) for k in range(d)}
    subs[T] = sp.Float(t, 30)
    out = []
    for q in range((m + 1) ** d):
        a = [(q // (m + 1) ** k) % (m + 1) for k in range(d)]
        e = expr
        w = sp.Integer(1)
        for k in range(d):
            if a[k]:
                e = sp.diff(e, X[k], a[k])
            w *= sp.Float(hs[k], 30) ** a[k] / sp.factorial(a[k])
        out.append(float((w * e).subs(subs).evalf(25)))
    return np.array(out)


def _node_point(ncell, node, dual):
    idx, rest = [], node
    for n in ncell:
        idx.append(rest % n)
        rest //= n
    return [(idx[k] + (0.5 if dual else 0.0)) / ncell[k] for k in range(len(ncell))]


def _check(field, expr, d, m, ncell, nodes, dual, t):
    hs = [1.0 / n for n in ncell]
    scale = float(np.abs(field).max())
    for node in nodes:
        ref = _scaled_slots(expr, d, m, hs, _node_point(ncell, node, dual), t)
        np.testing.assert_allclose(field[node], ref, rtol=0, atol=1e-12 * scale,
                                   err_msg=f"node {node} dual={dual}")


def test_gaussian_pulse_slots_are_the_scaled_derivatives():
    d, m, ncell, dt, width = 2, 3, [16, 12], 0.02, 0.2
    st = I.gaussian_pulse(d, m, ncell, dt, seed=7, width=width)
    x0 = st.desc["x0"]
    expr = sum(sp.exp(-((X[0] - x0[0] - i) ** 2 + (X[1] - x0[1] - j) ** 2) / sp.Float(width) ** 2)
               for i, j in itertools.product((-1, 0, 1), repeat=2))
    nodes = [0, 5, 37, 100, ncell[0] * ncell[1] - 1]
    _check(st.p, expr, d, m, ncell, nodes, False, 0.0)
    assert not st.u.any()


def test_plane_wave_slots_are_the_scaled_derivatives():
    m, ncell, dt = 2, [4, 5, 6], 0.01
    st = I.plane_wave(m, ncell, dt, seed=11)
    n, phi = st.desc["n"], st.desc["phi"]
    k = [2 * sp.pi * sp.Integer(int(c)) for c in n]
    kn = sp.sqrt(sum(c * c for c in k))
    p = sp.cos(sum(k[j] * X[j] for j in range(3)) - kn * T + sp.Float(phi, 30))
    nodes = [0, 7, 33, 119]
    _check(st.p, p, 3, m, ncell, nodes, False, 0.0)
    for j in range(3):
        _check(st.u[j], k[j] / kn * p, 3, m, ncell, nodes, True, 0.5 * dt)


def test_standing_mode_slots_are_the_scaled_derivatives():
    d, m, ncell, dt, wave = 2, 3, [10, 8], 0.03, [2, 1]
    st = I.standing_mode(d, m, ncell, dt, wave=wave, t0=0.1)
    nrm = sp.sqrt(sum(sp.Integer(w) ** 2 for w in wave))
    om = 2 * sp.pi * nrm
    p = sp.sin(2 * sp.pi * wave[0] * X[0]) * sp.sin(2 * sp.pi * wave[1] * X[1]) * sp.cos(om * T)
    u = [-(sp.Integer(wave[0]) / nrm) * sp.cos(2 * sp.pi * wave[0] * X[0]) * sp.sin(2 * sp.pi * wave[1] * X[1])
         * sp.sin(om * T),
         -(sp.Integer(wave[1]) / nrm) * sp.sin(2 * sp.pi * wave[0] * X[0]) * sp.cos(2 * sp.pi * wave[1] * X[1])
         * sp.sin(om * T)]
    nodes = [0, 9, 41, 79]
    _check(st.p, p, d, m, ncell, nodes, False, 0.1)
    for j in range(d):
        _check(st.u[j], u[j], d, m, ncell, nodes, True, 0.1 + 0.5 * dt)


def test_analytic_fields_solve_the_acoustic_system():
    """The plane wave and the standing mode of the generators solve p_t + div u = 0,
    u_t + grad p = 0 exactly (the sign convention the solver and the oracle share)."""
    n = [sp.Integer(1), sp.Integer(-2), sp.Integer(3)]
    k = [2 * sp.pi * c for c in n]
    kn = sp.sqrt(sum(c * c for c in k))
    phi = sp.Symbol("phi", real=True)
    p = sp.cos(sum(k[j] * X[j] for j in range(3)) - kn * T + phi)
    u = [k[j] / kn * p for j in range(3)]
    assert sp.simplify(sp.diff(p, T) + sum(sp.diff(u[j], X[j]) for j in range(3))) == 0
    for j in range(3):
        assert sp.simplify(sp.diff(u[j], T) + sp.diff(p, X[j])) == 0
    nrm = sp.sqrt(5)                        # wave numbers (2, 1)
    om = 2 * sp.pi * nrm
    s0, s1 = sp.sin(2 * sp.pi * 2 * X[0]), sp.sin(2 * sp.pi * X[1])
    c0, c1 = sp.cos(2 * sp.pi * 2 * X[0]), sp.cos(2 * sp.pi * X[1])
    p = s0 * s1 * sp.cos(om * T)
    u = [-(2 / nrm) * c0 * s1 * sp.sin(om * T), -(1 / nrm) * s0 * c1 * sp.sin(om * T)]
    assert sp.simplify(sp.diff(p, T) + sp.diff(u[0], X[0]) + sp.diff(u[1], X[1])) == 0
    for j in range(2):
        assert sp.simplify(sp.diff(u[j], T) + sp.diff(p, X[j])) == 0


def test_a_planted_generator_error_fails_the_pin(monkeypatch):
    """A dropped factorial in the scaled derivatives (a plausible slip) must fail the
    Gaussian pin above."""
    good = I._fact
    monkeypatch.setattr(I, "_fact", lambda a: 1.0 if a == 2 else good(a))
    with pytest.raises(AssertionError):
        test_gaussian_pulse_slots_are_the_scaled_derivatives()


def test_modified_scheme_standing_mode_on_both_grids():
    """Both fields on both grids (the modified scheme's state): p = sin(2 pi w x) cos(2 pi w t),
    u = -cos(2 pi w x) sin(2 pi w t), primal at t0 and dual at t0 + dt/2."""
    m, n, dt, w, t0 = 3, 12, 0.04, 2, 0.3
    pp, up, pd, ud = I.standing_mode_1d_both_grids(m, n, dt, w, t0=t0)
    kap = 2 * sp.pi * w
    p = sp.sin(kap * X[0]) * sp.cos(kap * T)
    u = -sp.cos(kap * X[0]) * sp.sin(kap * T)
    assert sp.simplify(sp.diff(p, T) + sp.diff(u, X[0])) == 0
    assert sp.simplify(sp.diff(u, T) + sp.diff(p, X[0])) == 0
    for arr, expr, dual, t in ((pp, p, False, t0), (up, u, False, t0), (pd, p, True, t0 + 0.5 * dt),
                               (ud, u, True, t0 + 0.5 * dt)):
        _check(arr, expr, 1, m, [n], [0, 5, n - 1], dual, t)


def test_variable_speed_inputs():
    """The variable-speed workload: the Taylor table of c^2 = 1 + sin(2 pi x)/2 (degree 2m+1),
    the initial data of p = u = sin(2 pi (x - t)), and the scaled Taylor coefficients of the
    time derivatives of the forcing z = pi sin(2 pi x) cos(2 pi (x - t)), which makes that pair
    an exact solution of p_t + c^2 u_x = z, u_t + p_x = 0."""
    m, n, dt, t = 2, 10, 0.03, 0.17
    x = X[0]
    c2 = 1 + sp.sin(2 * sp.pi * x) / 2
    sol = sp.sin(2 * sp.pi * (x - T))
    z = sp.pi * sp.sin(2 * sp.pi * x) * sp.cos(2 * sp.pi * (x - T))
    assert sp.simplify(sp.diff(sol, T) + c2 * sp.diff(sol, x) - z) == 0
    assert sp.simplify(sp.diff(sol, T) + sp.diff(sol, x)) == 0
    A = 2 * m + 2
    for dual in (False, True):
        _check(I.c2_taylor_table(n, m, dual), c2, 1, A - 1, [n], [0, 3, n - 1], dual, 0.0)
    p, u, fp, fd = I.variable_speed_wave(m, n, dt)
    _check(p, sol, 1, m, [n], [0, 4, n - 1], False, 0.0)
    _check(u, sol, 1, m, [n], [0, 4, n - 1], True, 0.5 * dt)
    for forcing, dual in ((fp, False), (fd, True)):
        for k in range(3):
            _check(forcing(k, t), sp.diff(z, T, k), 1, A - 1, [n], [0, 7], dual, t)
