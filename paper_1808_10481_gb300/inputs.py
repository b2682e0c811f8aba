"""Seeded synthetic initial data for the Hermite-leapfrog solver.

This module holds none of the method's arithmetic: it evaluates analytic
fields and their exact scaled derivatives at the grid nodes, in the library's
host layout, and nothing else.  Both the CUDA path's tests/benchmark and the
CPU oracle's tests draw their inputs from here.

Conventions (the ones the solver uses):
  * periodic unit box, n_k nodes per axis on each grid, h_k = 1/n_k;
  * primal node j at j*h (holds p), dual node j at (j + 1/2)*h (holds u);
  * scaled data f~_a = prod_k h_k^{a_k}/a_k! d^a f, a_k = 0..m
    (Section 2 for the 1D form, Section 5 for the tensor form);
  * host layout f[comp][node][q], node = ix + nx*(iy + ny*iz),
    q = a_0 + (m+1)*(a_1 + (m+1)*a_2);
  * p is given at t = 0 and u at t = dt/2 (the staggered start of Section 2);
  * PDE p_t + div u = 0, u_t + grad p = 0 (unit wave speed).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TWO_PI = 2.0 * math.pi


def node_coords(n: int, dual: bool) -> np.ndarray:
    """Coordinates of the n nodes of one axis: j/n (primal) or (j+1/2)/n (dual)."""
    return (np.arange(n, dtype=np.float64) + (0.5 if dual else 0.0)) / n


def _fact(a: int) -> float:
    return float(math.factorial(a))


def scaled_trig(x: np.ndarray, h: float, m: int, kappa: float, phase: float) -> np.ndarray:
    """Scaled derivatives of sin(kappa*x + phase): h^a/a! kappa^a sin(kappa x + phase + a pi/2).

    Returns shape (len(x), m+1).
    """
    out = np.empty((x.size, m + 1))
    for a in range(m + 1):
        out[:, a] = (h * kappa) ** a / _fact(a) * np.sin(kappa * x + phase + a * math.pi / 2.0)
    return out


def scaled_gauss(x: np.ndarray, h: float, m: int, centre: float, width: float,
                 images=(-1, 0, 1)) -> np.ndarray:
    """Scaled derivatives of the periodised Gaussian sum_i exp(-(x - centre - i)^2 / width^2).

    d^a/dx^a exp(-z^2) = (-1)^a He_a(z) exp(-z^2) with physicists' Hermite
    polynomials He_a and z = (x - c)/w, so the scaled value is
    (h/w)^a/a! (-1)^a He_a(z) exp(-z^2).  Returns shape (len(x), m+1).
    """
    out = np.zeros((x.size, m + 1))
    for img in images:
        z = (x - centre - img) / width
        g = np.exp(-z * z)
        hp = [np.ones_like(z), 2.0 * z]
        for a in range(1, m):
            hp.append(2.0 * z * hp[a] - 2.0 * a * hp[a - 1])
        for a in range(m + 1):
            out[:, a] += (h / width) ** a / _fact(a) * (-1.0) ** a * hp[a] * g
    return out


def tensor_field(factors: list[np.ndarray]) -> np.ndarray:
    """Tensor product of per-axis scaled-derivative tables -> (nnode, nq).

    factors[k] has shape (n_k, m+1); node index x-fastest, slot a_0-fastest.
    """
    d = len(factors)
    n1 = factors[0].shape[1]
    out = factors[0]  # (n0, m+1) -> grows as (nodes..., slots...)
    # build with einsum, then reorder to (node, q) with x-fastest / a_0-fastest
    if d == 1:
        return np.ascontiguousarray(out)
    if d == 2:
        t = np.einsum("ia,jb->jiba", factors[0], factors[1])  # [y][x][b][a]
        return np.ascontiguousarray(t.reshape(factors[0].shape[0] * factors[1].shape[0], n1 * n1))
    if d == 3:
        t = np.einsum("ia,jb,kc->kjicba", factors[0], factors[1], factors[2])
        nn = factors[0].shape[0] * factors[1].shape[0] * factors[2].shape[0]
        return np.ascontiguousarray(t.reshape(nn, n1 ** 3))
    raise ValueError("d must be 1, 2 or 3")


@dataclass
class InitialData:
    """Initial node data in host layout plus what generated it."""
    p: np.ndarray          # (nnode, nq) at t = 0
    u: np.ndarray          # (d, nnode, nq) at t = dt/2
    desc: dict


# ---------------------------------------------------------------- standing mode
def standing_mode(d: int, m: int, ncell, dt: float, wave=None, t0: float = 0.0) -> InitialData:
    """Standing mode p = prod_k sin(2 pi n_k x_k) cos(w t), w = 2 pi |n|.

    u_k = -(n_k/|n|) cos(2 pi n_k x_k) prod_{j != k} sin(2 pi n_j x_j) sin(w t),
    an exact solution of p_t + div u = 0, u_t + grad p = 0.  p is sampled at
    t0 and u at t0 + dt/2.
    """
    wave = list(wave) if wave is not None else [1] * d
    nrm = math.sqrt(sum(w * w for w in wave))
    omega = TWO_PI * nrm
    hs = [1.0 / n for n in ncell]
    prim = [scaled_trig(node_coords(ncell[k], False), hs[k], m, TWO_PI * wave[k], 0.0) for k in range(d)]
    p = tensor_field(prim) * math.cos(omega * t0)
    u = np.empty((d,) + p.shape)
    tu = t0 + 0.5 * dt
    for k in range(d):
        fac = []
        for j in range(d):
            x = node_coords(ncell[j], True)
            ph = math.pi / 2.0 if j == k else 0.0  # cos = sin(. + pi/2)
            fac.append(scaled_trig(x, hs[j], m, TWO_PI * wave[j], ph))
        u[k] = -(wave[k] / nrm) * tensor_field(fac) * math.sin(omega * tu)
    return InitialData(p, u, {"kind": "standing_mode", "wave": wave, "t0": t0})


def standing_mode_exact(d: int, m: int, ncell, wave, t_p: float, t_u: float) -> InitialData:
    """Exact node data of ``standing_mode`` at times t_p (p) and t_u (u)."""
    nrm = math.sqrt(sum(w * w for w in wave))
    omega = TWO_PI * nrm
    # reuse the generator with dt chosen so that t0 + dt/2 = t_u
    data = standing_mode(d, m, ncell, 2.0 * (t_u - t_p), wave=wave, t0=t_p)
    return data


# ---------------------------------------------------------------- Gaussian pulse
def gaussian_pulse(d: int, m: int, ncell, dt: float, seed: int, width: float = 0.05) -> InitialData:
    """Periodised Gaussian pressure pulse exp(-|x - x0|^2 / width^2), x0 ~ U[0,1)^d from the seed.

    u = 0 at t = dt/2 (the pulse starts from rest half a step later).  The
    periodisation sums the 3^d nearest images, which factorises per axis.
    """
    rng = np.random.default_rng(seed)
    x0 = rng.random(d)
    hs = [1.0 / n for n in ncell]
    fac = [scaled_gauss(node_coords(ncell[k], False), hs[k], m, float(x0[k]), width) for k in range(d)]
    p = tensor_field(fac)
    u = np.zeros((d,) + p.shape)
    return InitialData(p, u, {"kind": "gaussian", "seed": seed, "x0": x0.tolist(), "width": width})


# ---------------------------------------------------------------- plane wave
def plane_wave_vectors(kmax: float = 8.0) -> list[tuple[int, ...]]:
    out = []
    r = int(math.floor(kmax))
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            for c in range(-r, r + 1):
                if (a, b, c) != (0, 0, 0) and a * a + b * b + c * c <= kmax * kmax:
                    out.append((a, b, c))
    return out


def plane_wave(m: int, ncell, dt: float, seed: int, kmax: float = 8.0, t0: float = 0.0,
               nvec=None, phase=None) -> InitialData:
    """3D plane wave p = cos(k.x - |k| t + phi), u = (k/|k|) p, k = 2 pi n.

    n is drawn from the seed among integer vectors 0 < |n| <= kmax, phi ~ U[0, 2pi).
    Scaled derivatives: h^a/a! prod_j k_j^{a_j} cos(theta + |a| pi/2).
    """
    rng = np.random.default_rng(seed)
    vecs = plane_wave_vectors(kmax)
    n = np.array(vecs[int(rng.integers(len(vecs)))] if nvec is None else nvec, dtype=np.float64)
    phi = float(rng.random() * TWO_PI) if phase is None else float(phase)
    k = TWO_PI * n
    kn = float(np.linalg.norm(k))
    hs = np.array([1.0 / c for c in ncell])

    def field(dual: bool, t: float) -> np.ndarray:
        # theta at node (ix, iy, iz), x fastest, built by broadcasting the per-axis terms
        xs = [k[j] * node_coords(ncell[j], dual) for j in range(3)]
        theta = (xs[2][:, None, None] + xs[1][None, :, None] + xs[0][None, None, :] - kn * t + phi).reshape(-1)
        # cos(theta + s pi/2) cycles through cos, -sin, -cos, sin
        c, sn = np.cos(theta), np.sin(theta)
        quarter = (c, -sn, -c, sn)
        nq = (m + 1) ** 3
        out = np.empty((theta.size, nq))
        for q in range(nq):
            a = (q % (m + 1), (q // (m + 1)) % (m + 1), q // (m + 1) ** 2)
            w = 1.0
            for j in range(3):
                w *= (hs[j] * k[j]) ** a[j] / _fact(a[j])
            np.multiply(quarter[sum(a) % 4], w, out=out[:, q])
        return out

    p = field(False, t0)
    pu = field(True, t0 + 0.5 * dt)
    u = np.stack([(k[j] / kn) * pu for j in range(3)])
    return InitialData(p, u, {"kind": "plane_wave", "seed": seed, "n": n.tolist(), "phi": phi, "t0": t0})


# ---------------------------------------------------------------- random data
def random_state(d: int, m: int, ncell, seed: int) -> InitialData:
    """Uniform random node data in [-1, 1) for every slot: the hardest parity input."""
    rng = np.random.default_rng(seed)
    nnode = int(np.prod(ncell))
    nq = (m + 1) ** d
    p = rng.uniform(-1.0, 1.0, size=(nnode, nq))
    u = rng.uniform(-1.0, 1.0, size=(d, nnode, nq))
    return InitialData(p, u, {"kind": "random", "seed": seed})


def cfl_dt(ncell, c_cfl: float = 0.9) -> float:
    """dt = C_CFL * min_k h_k (unit wave speed); C_CFL = 0.9 gives lam = 0.45."""
    return c_cfl * min(1.0 / n for n in ncell)


def l2_error(d: int, ncell, approx: np.ndarray, exact: np.ndarray) -> float:
    """Discrete L2 norm of the value slot: sqrt(prod h_k * sum (f~_0 - f_0)^2)."""
    vol = float(np.prod([1.0 / n for n in ncell]))
    diff = approx.reshape(-1, approx.shape[-1])[:, 0] - exact.reshape(-1, exact.shape[-1])[:, 0]
    return math.sqrt(vol * float(np.sum(diff * diff)))


# ---------------------------------------------------------------- both fields on both grids (1D)
def standing_mode_1d_both_grids(m: int, n: int, dt: float, wave: int = 1, t0: float = 0.0):
    """The 1D standing mode p = sin(2 pi w x) cos(2 pi w t), u = -cos(2 pi w x) sin(2 pi w t)
    with both fields on both grids, as the modified scheme holds them: primal nodes j/n at
    t0 and dual nodes (j+1/2)/n at t0 + dt/2.  Returns (pp, up, pd, ud), each (n, m+1)."""
    h = 1.0 / n
    kap = TWO_PI * wave
    out = []
    for dual, t in ((False, t0), (True, t0 + 0.5 * dt)):
        x = node_coords(n, dual)
        p = scaled_trig(x, h, m, kap, 0.0) * math.cos(kap * t)
        u = -scaled_trig(x, h, m, kap, math.pi / 2.0) * math.sin(kap * t)
        out += [p, u]
    return tuple(out)


# ---------------------------------------------------------------- variable wave speed (1D)
def c2_taylor_table(n: int, m: int, dual: bool, amp: float = 0.5, wave: int = 1) -> np.ndarray:
    """Scaled Taylor coefficients h^i/i! d^i c^2 (i = 0..2m+1) of the squared wave speed
    c^2(x) = 1 + amp sin(2 pi wave x) at the primal (j/n) or dual ((j+1/2)/n) nodes; the
    unit-interval form of the paper's c^2 = 1 + sin(x)/2 on [0, 2 pi] (amp 1/2, wave 1)."""
    x = node_coords(n, dual)
    tab = amp * scaled_trig(x, 1.0 / n, 2 * m + 1, TWO_PI * wave, 0.0)
    tab[:, 0] += 1.0
    return tab


def c2_max(amp: float = 0.5) -> float:
    return math.sqrt(1.0 + abs(amp))


def _cauchy(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Row-wise product of two truncated Taylor series (same number of terms)."""
    A = a.shape[1]
    out = np.zeros_like(a)
    for k in range(A):
        for i in range(k + 1):
            out[:, k] += a[:, i] * b[:, k - i]
    return out


def variable_speed_wave(m: int, n: int, dt: float, t0: float = 0.0):
    """The paper's variable-speed experiment (Section 4.2) mapped from [0, 2 pi] to the unit
    interval: p = u = sin(2 pi (x - t)) solves p_t + c^2 u_x = z, u_t + p_x = 0 with
    c^2 = 1 + sin(2 pi x)/2 and the forcing z = pi sin(2 pi x) cos(2 pi (x - t)).
    Returns (p at t0 on the primal nodes, u at t0 + dt/2 on the dual nodes) and the forcing
    callbacks of the two grids: forcing(k, t) = scaled Taylor coefficients (degree 0..2m+1)
    of d_t^k z at those nodes."""
    h = 1.0 / n
    kap = TWO_PI
    p = scaled_trig(node_coords(n, False), h, m, kap, -kap * t0)
    u = scaled_trig(node_coords(n, True), h, m, kap, -kap * (t0 + 0.5 * dt))

    def make(dual):
        x = node_coords(n, dual)
        s = math.pi * scaled_trig(x, h, 2 * m + 1, kap, 0.0)

        def forcing(k, t):
            # d_t^k cos(2 pi (x - t)) = (2 pi)^k cos(2 pi (x - t) - k pi/2) = (2 pi)^k sin(. + pi/2 - k pi/2)
            c = kap ** k * scaled_trig(x, h, 2 * m + 1, kap, -kap * t + math.pi / 2.0 - k * math.pi / 2.0)
            return _cauchy(s, c)
        return forcing

    return p, u, make(False), make(True)
