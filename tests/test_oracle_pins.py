"""Pins for the CPU oracle: facts the paper and the mathematics fix, checked by routes
that share nothing with the oracle's own arithmetic.

* Section 2, eq. (interp): the matrices C^L, C^R reproduce the end data of any
  polynomial of degree 2m+1 (numpy's polynomial derivatives as the reference),
  and H inverts them.
* Sections 2 and 3.1.2, eqs. (final1), (pdup), (vdup): for polynomial partner data
  of per-axis degree <= 2m+1 the interpolant is exact, so one node update must equal
  the exact local evolution, computed here as exp(tau L) - exp(-tau L) of the PDE
  generator L on the polynomial space (scipy's matrix exponential).
* Section 1 (a high-order Yee scheme): m = 0 in 1D is exactly the staggered
  second-order FDTD update.
* Section 3.1.1, eq. (fullcons1d): Q^h(n dt) = R^h((n+1/2) dt) = Q^h(0) in 1D, with
  the H^{m+1} seminorms evaluated by Gauss quadrature of an independently built
  piecewise interpolant.
* Section 3 (the CFL remark after eq. (vh1evolve)): stable for c dt/dx < 1, unstable
  well above it.
* Tables 1 and 5: observed L2 convergence rates at C_CFL = 0.9, 0.5 and 0.1.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest
from numpy.polynomial import polynomial as P
from scipy.linalg import expm

import oracle
from oracle.hermite import hermite_inverse, hermite_inverse_exact, interp_system
from paper_1808_10481_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rates(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                m, r = line.split()
                out[int(m)] = float(r)
    return out


# ----------------------------------------------------------------------------- helpers
def _taylor_at(xi0: float, m: int, A: int) -> np.ndarray:
    """(m+1) x A matrix: monomial coefficients -> scaled data (1/l!) q^(l)(xi0), via numpy."""
    T = np.zeros((m + 1, A))
    for a in range(A):
        e = np.zeros(A)
        e[a] = 1.0
        for l in range(m + 1):
            T[l, a] = P.polyval(xi0, P.polyder(e, l)) / math.factorial(l) if l <= a else 0.0
    return T


def _kron_axes(mats):
    """Kronecker product acting on a tensor index with axis 0 fastest."""
    out = np.ones((1, 1))
    for M in mats:
        out = np.kron(M, out)
    return out


def _diff_matrix(A: int) -> np.ndarray:
    D = np.zeros((A, A))
    for a in range(A):
        e = np.zeros(A)
        e[a] = 1.0
        der = P.polyder(e, 1)
        D[: der.size, a] = der
    return D


def _exact_increment(d, m, lam, mode, rng):
    """Random polynomial partner data on one cell and the exact increment of the target.

    Returns (vertex data in the oracle's node_update layout, exact increment (ncd, nq)).
    """
    A = 2 * m + 2
    n = m + 1
    NA = A ** d
    nq = n ** d
    ncs, ncd = (d, 1) if mode == 0 else (1, d)
    D1 = _diff_matrix(A)
    Dk = []
    for k in range(d):
        mats = [np.eye(A)] * d
        mats = list(mats)
        mats[k] = D1
        Dk.append(_kron_axes(mats))
    # state = [p, u_0, ..., u_{d-1}], each a coefficient tensor in xi = (x - x_node)/h
    G = np.zeros(((d + 1) * NA, (d + 1) * NA))
    for k in range(d):
        G[0:NA, (k + 1) * NA:(k + 2) * NA] = -lam[k] * Dk[k]      # p_t = -div u
        G[(k + 1) * NA:(k + 2) * NA, 0:NA] = -lam[k] * Dk[k]      # u_t = -grad p
    E = expm(G) - expm(-G)
    coefs = rng.uniform(-1.0, 1.0, size=(ncs, NA))
    state = np.zeros((d + 1) * NA)
    if mode == 0:
        for k in range(d):
            state[(k + 1) * NA:(k + 2) * NA] = coefs[k]
    else:
        state[0:NA] = coefs[0]
    inc = E @ state
    # slot s of a node = Taylor coefficient of xi^s at xi = 0
    sel = []
    for q in range(nq):
        s = [(q // n ** k) % n for k in range(d)]
        sel.append(sum(s[k] * A ** k for k in range(d)))
    if mode == 0:
        exact = inc[0:NA][sel][None, :]
    else:
        exact = np.stack([inc[(k + 1) * NA:(k + 2) * NA][sel] for k in range(d)])
    # vertex data: bit k of v selects xi_k = -1/2 (0) or +1/2 (1)
    Tm, Tp = _taylor_at(-0.5, m, A), _taylor_at(0.5, m, A)
    vtx = np.zeros((ncs, 1 << d, nq))
    for v in range(1 << d):
        T = _kron_axes([Tp if (v >> k) & 1 else Tm for k in range(d)])
        for c in range(ncs):
            vtx[c, v] = T @ coefs[c]
    return vtx, exact


# ----------------------------------------------------------------------------- eq. (interp)
@pytest.mark.parametrize("m", range(0, 7))
def test_interp_system_reproduces_polynomial_end_data(m):
    rng = np.random.default_rng(100 + m)
    A = 2 * m + 2
    Amat = np.array([[float(x) for x in row] for row in interp_system(m)])
    H = np.array(hermite_inverse(m))
    for _ in range(5):
        c = rng.uniform(-1, 1, A)
        data = np.concatenate([_taylor_at(-0.5, m, A) @ c, _taylor_at(0.5, m, A) @ c])
        np.testing.assert_allclose(Amat @ c, data, rtol=0, atol=1e-13)
        np.testing.assert_allclose(H @ data, c, rtol=0, atol=1e-10 * max(1.0, np.abs(H).max()))


@pytest.mark.parametrize("m", range(0, 7))
def test_hermite_inverse_is_exact(m):
    A = interp_system(m)
    H = hermite_inverse_exact(m)
    n = len(A)
    for i in range(n):
        for j in range(n):
            assert sum(H[i][k] * A[k][j] for k in range(n)) == (1 if i == j else 0)


# ----------------------------------------------------------------------------- exact local evolution
CASES = [(1, m) for m in range(7)] + [(2, m) for m in range(5)] + [(3, m) for m in range(4)]


@pytest.mark.parametrize("d,m", CASES)
@pytest.mark.parametrize("mode", [0, 1])
def test_node_update_equals_exact_local_evolution(d, m, mode):
    rng = np.random.default_rng(1000 * d + 10 * m + mode)
    lam = [0.45, 0.31, 0.23][:d]   # distinct per axis: catches a transposed axis
    vtx, exact = _exact_increment(d, m, lam, mode, rng)
    got = oracle.node_update(d, m, lam, mode, vtx)
    scale = np.abs(exact).max()
    assert np.abs(got - exact).max() <= 1e-12 * scale, (np.abs(got - exact).max(), scale)


def test_node_update_truncated_data_is_not_exact():
    """Data of degree 2m+3 lie outside the interpolation space: the update must then
    differ from the exact shift (guards against a pin that passes vacuously)."""
    m = 2
    A = 2 * m + 4
    c = np.zeros(A)
    c[-1] = 1.0                       # xi^(2m+3): odd, so the exact increment is non-zero
    lam = 0.45
    vtx = np.stack([_taylor_at(-0.5, m, A) @ c, _taylor_at(0.5, m, A) @ c])[None]
    got = oracle.node_update(1, m, [lam], 0, vtx)[0, 0]
    exact = -(P.polyval(lam, c) - P.polyval(-lam, c))
    assert abs(got - exact) > 1e-6 * abs(exact)


def test_1d_update_is_dalembert_shift():
    """In 1D the exact evolution is a shift: p(t+dt) - p(t) = -[u(x+dt/2) - u(x-dt/2)]
    (Section 3.1.1, eq. (p1evolve) with v = -u).  Checked for every slot."""
    rng = np.random.default_rng(7)
    for m in range(0, 7):
        A = 2 * m + 2
        c = rng.uniform(-1, 1, A)
        lam = 0.41
        vtx = np.stack([_taylor_at(-0.5, m, A) @ c, _taylor_at(0.5, m, A) @ c])[None]
        got = oracle.node_update(1, m, [lam], 0, vtx)[0]
        exact = -(_taylor_at(lam, m, A) @ c - _taylor_at(-lam, m, A) @ c)
        np.testing.assert_allclose(got, exact, rtol=0, atol=1e-12 * np.abs(exact).max())


# ----------------------------------------------------------------------------- Yee special case
def test_m0_1d_is_yee_fdtd():
    rng = np.random.default_rng(3)
    N = 11
    h = 1.0 / N
    dt = 0.8 * h
    p = rng.uniform(-1, 1, (N, 1))
    u = rng.uniform(-1, 1, (1, N, 1))
    p2, u2 = oracle.run(1, 0, [N], dt, p, u, 1)
    pe = p[:, 0] - dt / h * (u[0, :, 0] - np.roll(u[0, :, 0], 1))
    ue = u[0, :, 0] - dt / h * (np.roll(pe, -1) - pe)
    np.testing.assert_allclose(p2[:, 0], pe, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u2[0, :, 0], ue, rtol=0, atol=1e-14)


# ----------------------------------------------------------------------------- stability
def _step_matrix(d, m, ncell, dt):
    nnode = int(np.prod(ncell))
    nq = (m + 1) ** d
    npd = nnode * nq
    tot = npd * (1 + d)
    S = np.zeros((tot, tot))
    for j in range(tot):
        e = np.zeros(tot)
        e[j] = 1.0
        p, u = oracle.run(d, m, ncell, dt, e[:npd].reshape(nnode, nq), e[npd:].reshape(d, nnode, nq), 1)
        S[:, j] = np.concatenate([p.ravel(), u.ravel()])
    return S


@pytest.mark.parametrize("m", range(0, 4))
def test_1d_stable_at_cfl_unstable_beyond(m):
    N = 8
    h = 1.0 / N
    rho = np.abs(np.linalg.eigvals(_step_matrix(1, m, [N], 0.9 * h))).max()
    assert rho <= 1.0 + 1e-6
    rho_bad = np.abs(np.linalg.eigvals(_step_matrix(1, m, [N], 1.8 * h))).max()
    assert rho_bad > 1.5


@pytest.mark.parametrize("m", [1, 2])
def test_2d_stable_at_cfl(m):
    ncell = [4, 5]                   # h_x != h_y
    dt = 0.9 * min(1.0 / n for n in ncell)
    rho = np.abs(np.linalg.eigvals(_step_matrix(2, m, ncell, dt))).max()
    assert rho <= 1.0 + 1e-6
    rho_bad = np.abs(np.linalg.eigvals(_step_matrix(2, m, ncell, 2.0 * dt))).max()
    assert rho_bad > 1.5


@pytest.mark.parametrize("m", [0, 1])
def test_3d_stable_at_cfl(m):
    """Section 5 builds the multi-dimensional scheme as a tensor product and states that
    three dimensions follow the same construction; the 3D step at dt = 0.9 min(h) keeps its
    spectrum in the unit disc and loses it at twice that step.  The eigenvalue 1 of the
    periodic step is defective: derivative data can be periodic while the field they
    describe is not (a constant slope of p drives a velocity that grows linearly in time),
    and such modes grow polynomially.  Rounding moves a defective eigenvalue by about
    eps^(1/3), so the bound carries that margin."""
    ncell = [2, 3, 2]                # three different h
    dt = 0.9 * min(1.0 / n for n in ncell)
    rho = np.abs(np.linalg.eigvals(_step_matrix(3, m, ncell, dt))).max()
    assert rho <= 1.0 + 1e-5
    rho_bad = np.abs(np.linalg.eigvals(_step_matrix(3, m, ncell, 2.0 * dt))).max()
    assert rho_bad > 1.5


# ----------------------------------------------------------------------------- conservation
def _piecewise(data, m, h, offset):
    """Independent piecewise interpolant of node data (N, m+1) on the periodic unit line.

    Nodes at offset + j*h; cell j spans nodes j and j+1, centred at offset + (j+1/2)h.
    Built by solving the Hermite conditions with numpy (not the oracle's H).
    """
    A = 2 * m + 2
    M = np.vstack([_taylor_at(-0.5, m, A), _taylor_at(0.5, m, A)])
    rhs = np.concatenate([data, np.roll(data, -1, axis=0)], axis=1)  # (N, 2m+2)
    coef = np.linalg.solve(M, rhs.T).T                               # (N, 2m+2)
    return coef, offset + 0.5 * h


def _deriv_eval(coef, centre0, h, m, x):
    """(m+1)-th x-derivative of the piecewise polynomial at points x (periodic)."""
    N = coef.shape[0]
    y = (x - centre0 + 0.5 * h) % 1.0            # distance from the first cell's start
    j = np.minimum((y / h).astype(int), N - 1)
    xi = (y - (j + 0.5) * h) / h
    out = np.zeros_like(x)
    for a in range(m + 1, coef.shape[1]):
        fall = math.factorial(a) / math.factorial(a - m - 1)
        out += coef[j, a] * fall * xi ** (a - m - 1)
    return out / h ** (m + 1)


def _seminorm_pair(fa, fb, sign, shift, m, h):
    """| f_a(x) + sign * f_b(x + shift) |^2_{m+1} on [0,1), piecewise Gauss quadrature."""
    (ca, oa), (cb, ob) = fa, fb
    N = ca.shape[0]
    bps = np.concatenate([(oa - 0.5 * h + np.arange(N) * h) % 1.0,
                          (ob - 0.5 * h + np.arange(N) * h - shift) % 1.0, [0.0, 1.0]])
    bps = np.unique(np.round(bps, 15))
    gx, gw = np.polynomial.legendre.leggauss(2 * m + 4)
    total = 0.0
    for a, b in zip(bps[:-1], bps[1:]):
        if b - a < 1e-15:
            continue
        x = 0.5 * (a + b) + 0.5 * (b - a) * gx
        f = _deriv_eval(ca, oa, h, m, x) + sign * _deriv_eval(cb, ob, h, m, (x + shift) % 1.0)
        total += 0.5 * (b - a) * float(np.sum(gw * f * f))
    return total


@pytest.mark.parametrize("m", [1, 2, 3])
def test_1d_discrete_conservation(m):
    """Q^h(n dt) = R^h((n+1/2) dt) = Q^h(0), with P_pm = p^h pm S_pm u^h and
    V_pm = u^h pm S_pm p^h (the paper's definitions with v = -u)."""
    N = 12
    h = 1.0 / N
    dt = 0.9 * h
    tau = 0.5 * dt
    rng = np.random.default_rng(50 + m)
    p = rng.uniform(-1, 1, (N, m + 1))
    u = rng.uniform(-1, 1, (1, N, m + 1))

    def R(p, u):    # u at t + dt/2, p at t
        ph = _piecewise(p, m, h, 0.0)          # p on primal nodes j*h
        uh = _piecewise(u[0], m, h, 0.5 * h)   # u on dual nodes (j+1/2)h
        return _seminorm_pair(uh, ph, +1.0, tau, m, h) + _seminorm_pair(uh, ph, -1.0, -tau, m, h)

    def Q(p, u):    # p at t, u at t - dt/2
        ph = _piecewise(p, m, h, 0.0)
        uh = _piecewise(u[0], m, h, 0.5 * h)
        return _seminorm_pair(ph, uh, +1.0, tau, m, h) + _seminorm_pair(ph, uh, -1.0, -tau, m, h)

    vals = [R(p, u)]
    for _ in range(6):
        oracle.half_step(1, m, [N], dt, 0, u, p)
        vals.append(Q(p, u))
        oracle.half_step(1, m, [N], dt, 1, p, u)
        vals.append(R(p, u))
    vals = np.array(vals)
    assert np.abs(vals - vals[0]).max() <= 1e-10 * vals[0], vals


def test_1d_conservation_detects_wrong_step():
    """The seminorm machinery above is sensitive: a p-half at the wrong dt breaks it."""
    m, N = 2, 12
    h = 1.0 / N
    dt = 0.9 * h
    rng = np.random.default_rng(9)
    p = rng.uniform(-1, 1, (N, m + 1))
    u = rng.uniform(-1, 1, (1, N, m + 1))
    ph, uh = _piecewise(p, m, h, 0.0), _piecewise(u[0], m, h, 0.5 * h)
    r0 = _seminorm_pair(uh, ph, 1.0, dt / 2, m, h) + _seminorm_pair(uh, ph, -1.0, -dt / 2, m, h)
    oracle.half_step(1, m, [N], 1.1 * dt, 0, u, p)
    ph, uh = _piecewise(p, m, h, 0.0), _piecewise(u[0], m, h, 0.5 * h)
    q1 = _seminorm_pair(ph, uh, 1.0, dt / 2, m, h) + _seminorm_pair(ph, uh, -1.0, -dt / 2, m, h)
    assert abs(q1 - r0) > 1e-6 * r0


# ----------------------------------------------------------------------------- convergence rates
def _rate(d, m, Ns, T, wave, cfl=0.9):
    errs = []
    for N in Ns:
        ncell = [N] * d
        h = 1.0 / N
        n = math.ceil(T / (cfl * h))
        dt = T / n
        st = I.standing_mode(d, m, ncell, dt, wave=wave)
        p, u = oracle.run(d, m, ncell, dt, st.p, st.u, n)
        ex = I.standing_mode_exact(d, m, ncell, wave, n * dt, (n + 0.5) * dt)
        errs.append(I.l2_error(d, ncell, p, ex.p))
    return float(np.polyfit(np.log(1.0 / np.array(Ns)), np.log(errs), 1)[0])


def _check_rate(m, got, paper):
    if m % 2 == 0:
        # even orders: the paper observes (and the dispersion analysis explains) 2m+2
        assert abs(got - paper) <= 0.35, (m, got, paper)
    else:
        # odd orders: the proven 2m (Section 3.2) up to the pre-asymptotic excess the
        # paper's tables show; the local rates between successive grids oscillate
        # (2D m = 3 at T = 0.5: 4.5 to 6.8 on 8..32 nodes, 5.9 to 6.0 beyond), so the
        # fitted rate depends on the grid range, which the paper does not state for 2D
        assert 2 * m - 0.5 <= got <= 2 * m + 1.5, (m, got, paper)


@pytest.mark.parametrize("cfl,table", [(0.9, "table1_rates_cfl09.txt"), (0.5, "table1_rates_cfl05.txt"),
                                       (0.1, "table1_rates_cfl01.txt")])
@pytest.mark.parametrize("m", range(0, 4))
def test_1d_convergence_rate_matches_table1(m, cfl, table):
    paper = _read_rates(table)[m]
    # the paper's [-1,1] standing wave sin(2 pi x) cos(2 pi t), T = 4.13, mapped to [0,1]
    got = _rate(1, m, [16, 24, 32, 48, 64, 96], T=4.13 / 2, wave=[2], cfl=cfl)
    _check_rate(m, got, paper)
    if m in (0, 2):
        assert abs(got - paper) <= 0.35


@pytest.mark.parametrize("cfl,table", [(0.9, "table5_rates_cfl09.txt"), (0.5, "table5_rates_cfl05.txt"),
                                       (0.1, "table5_rates_cfl01.txt")])
@pytest.mark.parametrize("m", range(0, 4))
def test_2d_convergence_rate_matches_table5(m, cfl, table):
    paper = _read_rates(table)[m]
    # the paper's [-1,1]^2 mode sin(pi x) sin(pi y) cos(sqrt(2) pi t) mapped to [0,1]^2
    got = _rate(2, m, [8, 12, 16, 24, 32], T=0.5, wave=[1, 1], cfl=cfl)
    if m % 2 == 0:
        # The paper states neither its 2D grids nor its final time, and its own even-order
        # entries for one scheme spread over the three C_CFL columns (m = 2: 5.68, 5.71,
        # 6.01, around the expected 2m + 2 = 6): the fitted rate must lie within 0.35 of
        # that spread.
        cols = [_read_rates(t)[m] for t in ("table5_rates_cfl01.txt", "table5_rates_cfl05.txt",
                                            "table5_rates_cfl09.txt")]
        assert min(cols) - 0.35 <= got <= max(cols) + 0.35, (m, got, cols)
    else:
        _check_rate(m, got, paper)


def test_half_step_nodes_matches_full_half_step():
    """The sampled-node entry point is the full half-step restricted to those nodes."""
    rng = np.random.default_rng(11)
    for d, m, ncell in [(1, 3, [9]), (2, 2, [5, 7]), (3, 1, [3, 4, 5])]:
        st = I.random_state(d, m, ncell, seed=5)
        nodes = rng.choice(int(np.prod(ncell)), size=6, replace=False)
        for mode in (0, 1):
            src, dst = (st.u, st.p) if mode == 0 else (st.p, st.u)
            full = np.array(dst, copy=True)
            oracle.half_step(d, m, ncell, 0.3 / max(ncell), mode, np.ascontiguousarray(src), full)
            got = oracle.half_step_nodes(d, m, ncell, 0.3 / max(ncell), mode, src, dst, nodes)
            full = full.reshape(-1 if mode == 0 else d, int(np.prod(ncell)), (m + 1) ** d)
            if mode == 0:
                full = full.reshape(1, int(np.prod(ncell)), (m + 1) ** d)
            np.testing.assert_array_equal(got, full[:, nodes, :])


# ----------------------------------------------------------------------------- point source
def test_source_spatial_factor_matches_symbolic_derivatives():
    """g~_a = prod_k h^{a_k}/a_k! d^{a_k} exp(-(x_k - x0_k)^2 / (2 sigma^2)), checked against
    sympy's symbolic derivatives; R(t0) = 1 isolates the spatial factor."""
    sp = pytest.importorskip("sympy")
    d, m, ncell = 2, 3, [40, 32]
    x0 = [0.512, 0.47]
    sigma, f0 = 0.03, 12.0
    p = np.zeros((int(np.prod(ncell)), (m + 1) ** d))
    oracle.add_source(d, m, ncell, x0, sigma, f0, amp=1.0, t_mid=1.2 / f0, dt=1.0, p=p)
    X = sp.Symbol("x")
    derivs = []
    for k in range(d):
        g = sp.exp(-(X - sp.Rational(str(x0[k]))) ** 2 / (2 * sp.Rational(str(sigma)) ** 2))
        derivs.append([sp.lambdify(X, sp.diff(g, X, a)) for a in range(m + 1)])
    for node in [0, 20 + 40 * 15, 21 + 40 * 14, 25 + 40 * 18]:
        j = [node % ncell[0], node // ncell[0]]
        for q in range((m + 1) ** d):
            a = [q % (m + 1), q // (m + 1)]
            want = 1.0
            for k in range(d):
                h = 1.0 / ncell[k]
                want *= h ** a[k] / math.factorial(a[k]) * float(derivs[k][a[k]](j[k] * h))
            assert abs(p[node, q] - want) <= 1e-13 * max(1.0, abs(want))


def test_ricker_wavelet_closed_form_points():
    """R(t0) = 1 and R vanishes at t0 +- 1/(sqrt(2) pi f0), read through a one-node-sized
    source: with x0 on a node, g~_0 = 1 there."""
    d, m, ncell = 1, 0, [16]
    f0 = 15.0
    t0 = 1.2 / f0
    for t, want in [(t0, 1.0), (t0 + 1.0 / (math.sqrt(2.0) * math.pi * f0), 0.0),
                    (t0 - 1.0 / (math.sqrt(2.0) * math.pi * f0), 0.0)]:
        p = np.zeros((16, 1))
        oracle.add_source(d, m, ncell, [0.25], 0.01, f0, amp=1.0, t_mid=t, dt=1.0, p=p)
        assert abs(p[4, 0] - want) <= 1e-14


def test_source_superposition():
    """The forced scheme is linear: run with source = run without + forced run from rest."""
    d, m, ncell = 2, 2, [24, 20]
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=21)
    args = dict(x0=[0.4, 0.6], sigma=0.05, f0=10.0, amp=3.0)
    pf, uf = oracle.run_source(d, m, ncell, dt, st.p, st.u, 12, **args)
    p0, u0 = oracle.run(d, m, ncell, dt, st.p, st.u, 12)
    ps, us = oracle.run_source(d, m, ncell, dt, np.zeros_like(st.p), np.zeros_like(st.u), 12, **args)
    np.testing.assert_allclose(pf, p0 + ps, rtol=0, atol=1e-12 * np.abs(pf).max())
    np.testing.assert_allclose(uf, u0 + us, rtol=0, atol=1e-12 * np.abs(uf).max())


def test_double_double_build_agrees_with_binary64():
    """The double-double build (the reference of long GPU runs) is the same algorithm: on a short
    run the two builds agree to binary64 rounding, and on the 1000-step 1D workload they
    differ by no more than the binary64 build's accumulated rounding."""
    d, m, ncell = 2, 3, [12, 10]
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=31)
    p64, u64 = oracle.run(d, m, ncell, dt, st.p, st.u, 3)
    pdd, udd = oracle.run(d, m, ncell, dt, st.p, st.u, 3, prec="dd")
    assert np.abs(p64 - pdd).max() <= 1e-13 * np.abs(pdd).max()
    assert np.abs(u64 - udd).max() <= 1e-13 * np.abs(udd).max()
    d, m, ncell = 1, 3, [64]
    dt = I.cfl_dt(ncell)
    st = I.standing_mode(d, m, ncell, dt, wave=[3])
    p64, _ = oracle.run(d, m, ncell, dt, st.p, st.u, 1000)
    pdd, _ = oracle.run(d, m, ncell, dt, st.p, st.u, 1000, prec="dd")
    assert np.abs(p64 - pdd).max() <= 1e-11 * np.abs(pdd).max()


# ----------------------------------------------------------------------------- learned correction
def test_mlp_gradients_match_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(5)
    params = mlp.init_params(rng, n_in=6, n_h=5, n_out=3)
    for k in params:
        params[k] = params[k] + 0.1 * rng.standard_normal(params[k].shape)   # non-zero biases
    X = rng.standard_normal((7, 6))
    T = rng.standard_normal((7, 3))
    _, g = mlp.loss_and_grads(params, X, T)
    h = 1e-6
    for k, v in params.items():
        it = np.nditer(v, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = v[idx]
            v[idx] = old + h
            lp, _ = mlp.loss_and_grads(params, X, T)
            v[idx] = old - h
            lm, _ = mlp.loss_and_grads(params, X, T)
            v[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, g[k][idx])


def test_restriction_of_fine_analytic_data_is_coarse_analytic_data():
    """Scaled derivatives restricted from a 4x finer grid equal the coarse grid's own
    samples of the same analytic field (h^|a| scaling with h_c = 4 h_f)."""
    from oracle import mlp
    m = 3
    nc, r = [20, 16], 4
    nf = [nc[0] * r, nc[1] * r]
    fine = I.standing_mode(2, m, nf, 0.01, wave=[2, 1])
    coarse = I.standing_mode(2, m, nc, 0.01, wave=[2, 1])
    got = mlp.restrict_p(fine.p, nf, r, m)
    np.testing.assert_allclose(got, coarse.p, rtol=0, atol=1e-12)


def test_features_follow_translation():
    """Shifting the fields by whole cells shifts the feature rows with them."""
    from oracle import mlp
    m, ncell = 3, [10, 8]
    st = I.random_state(2, m, ncell, seed=2)
    nq = (m + 1) ** 2
    P = st.p.reshape(8, 10, nq)
    U = st.u.reshape(2, 8, 10, nq)
    Ps = np.roll(P, shift=(2, 3), axis=(0, 1)).reshape(-1, nq)
    Us = np.roll(U, shift=(2, 3), axis=(1, 2)).reshape(2, -1, nq)
    nodes = [0, 13, 79]
    f0 = mlp.features(st.p, st.u, ncell, nodes, 0.5, 0.25)
    moved = [((n // 10 + 2) % 8) * 10 + (n % 10 + 3) % 10 for n in nodes]
    f1 = mlp.features(Ps, Us, ncell, moved, 0.5, 0.25)
    np.testing.assert_array_equal(f0, f1)
    assert np.all(f0[:, 272] == 0.25) and np.all(f0[:, 273:] == 0.0)


def test_features_stencil_fixed_by_coordinate_codes():
    """Every feature column carries a value that encodes (field, iy, ix, slot), so each
    column block is checked against the node and component the stencil names: p at the
    3x3 primal nodes J + {-1,0,1}^2 (y offset outer), then u and then v at the four dual
    vertices of J's cell, dual nodes J + {-1,0}^2 (y offset outer), then t, then zeros."""
    from oracle import mlp
    m, n0, n1 = 3, 11, 7
    nq = 16

    def code(field, iy, ix, q):
        return float(((field * 1000 + iy) * 1000 + ix) * 100 + q)

    P = np.array([[code(0, n // n0, n % n0, q) for q in range(nq)] for n in range(n0 * n1)])
    U = np.array([[[code(1 + c, n // n0, n % n0, q) for q in range(nq)] for n in range(n0 * n1)]
                  for c in range(2)])
    nodes = [0, 5, n0 - 1, n0 * (n1 - 1), n0 * n1 - 1, 3 * n0 + 4]
    X = mlp.features(P, U, [n0, n1], nodes, 1.0, 0.375)
    for r, node in enumerate(nodes):
        jx, jy = node % n0, node // n0
        blocks = [(0, dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        blocks += [(1 + c, vy, vx) for c in range(2) for vy in (-1, 0) for vx in (-1, 0)]
        for b, (field, oy, ox) in enumerate(blocks):
            want = [code(field, (jy + oy) % n1, (jx + ox) % n0, q) for q in range(nq)]
            np.testing.assert_array_equal(X[r, b * nq:(b + 1) * nq], want)
        assert X[r, 17 * nq] == 0.375
        assert np.all(X[r, 17 * nq + 1:] == 0.0)
        assert X.shape[1] == mlp.N_IN == 288


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2, so each
    step moves w by -lr * g / (|g| + eps): after t steps w_t = w_0 - t lr g / (|g| + eps)."""
    from oracle import mlp
    rng = np.random.default_rng(5)
    w0 = {"a": rng.standard_normal((4, 3)), "b": rng.standard_normal(5)}
    g = {"a": rng.standard_normal((4, 3)), "b": rng.standard_normal(5) * 1e-3}
    w = {k: v.copy() for k, v in w0.items()}
    m1 = {k: np.zeros_like(v) for k, v in w0.items()}
    m2 = {k: np.zeros_like(v) for k, v in w0.items()}
    lr, eps = 0.01, 1e-8
    for t in range(1, 8):
        mlp.adam_step(w, g, m1, m2, t, lr, eps=eps)
        for k in w0:
            want = w0[k] - t * lr * g[k] / (np.abs(g[k]) + eps)
            np.testing.assert_allclose(w[k], want, rtol=0, atol=1e-13)


def test_adam_two_step_weighted_means():
    """After gradients g1 then g2 the bias-corrected moments are the weighted means
    (b1 g1 + g2) / (1 + b1) and (b2 g1^2 + g2^2) / (1 + b2) (the exponential averages
    divided by their weight sums), which fixes which beta goes with which moment."""
    from oracle import mlp
    rng = np.random.default_rng(6)
    b1, b2, lr, eps = 0.9, 0.999, 0.003, 1e-8
    w0 = {"a": rng.standard_normal(6)}
    g1, g2 = {"a": rng.standard_normal(6)}, {"a": rng.standard_normal(6)}
    w = {"a": w0["a"].copy()}
    m1, m2 = {"a": np.zeros(6)}, {"a": np.zeros(6)}
    mlp.adam_step(w, g1, m1, m2, 1, lr, b1, b2, eps)
    w1 = w0["a"] - lr * g1["a"] / (np.abs(g1["a"]) + eps)
    np.testing.assert_allclose(w["a"], w1, rtol=0, atol=1e-14)
    mlp.adam_step(w, g2, m1, m2, 2, lr, b1, b2, eps)
    mh = (b1 * g1["a"] + g2["a"]) / (1 + b1)
    vh = (b2 * g1["a"] ** 2 + g2["a"] ** 2) / (1 + b2)
    np.testing.assert_allclose(w["a"], w1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-14)


def test_adam_is_invariant_to_gradient_scale_without_eps():
    """Adam's step is invariant to a positive rescaling of every gradient when eps = 0."""
    from oracle import mlp
    rng = np.random.default_rng(7)
    gs = [{"a": rng.standard_normal(9)} for _ in range(4)]
    out = []
    for scale in (1.0, 37.5):
        w = {"a": np.ones(9)}
        m1, m2 = {"a": np.zeros(9)}, {"a": np.zeros(9)}
        for t, g in enumerate(gs, 1):
            mlp.adam_step(w, {"a": scale * g["a"]}, m1, m2, t, 0.01, eps=0.0)
        out.append(w["a"])
    np.testing.assert_allclose(out[0], out[1], rtol=1e-14, atol=0)


@pytest.mark.parametrize("m", [1, 3])
def test_2d_odd_order_local_rates_settle_at_2m(m):
    """Odd orders in 2D: the local rates log(e_N / e_2N) / log 2 between successive finer grids
    settle at the proven 2m (Section 3.2's h^(2m) bound) once the grids resolve the mode; the
    paper's larger odd entries of Table 5 (6.74, 7.45, 6.84 for m = 3) lie within the spread of
    the pre-asymptotic local rates on coarse grids."""
    Ns = [24, 32, 48, 64]
    errs = []
    for N in Ns:
        ncell = [N, N]
        n = math.ceil(2.065 / (0.9 / N))
        dt = 2.065 / n
        st = I.standing_mode(2, m, ncell, dt, wave=[1, 1])
        p, _ = oracle.run(2, m, ncell, dt, st.p, st.u, n)
        ex = I.standing_mode_exact(2, m, ncell, [1, 1], n * dt, (n + 0.5) * dt)
        errs.append(I.l2_error(2, ncell, p, ex.p))
    local = [math.log(errs[i] / errs[i + 1]) / math.log(Ns[i + 1] / Ns[i]) for i in range(len(Ns) - 1)]
    assert all(abs(r - 2 * m) <= 0.3 for r in local), local
