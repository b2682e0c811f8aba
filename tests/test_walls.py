"""Reflecting walls by ghost mirroring, checked on the CPU.

The reference is the method of images: a box [0, 1/2] along each walled axis is the
periodic unit box with the data extended across the walls, p with parity s (-1 for a
Dirichlet wall p = 0, +1 for a Neumann wall), the normal velocity with -s and the
tangential velocities with s.  The mirror map is written here independently of the
library's ghost filling (whole-grid index maps instead of ghost planes) and pinned to
the PDE first: exact standing modes that satisfy the wall conditions are invariant under
it, and the periodic oracle keeps mirrored data mirrored.  Then the library's ghost fill
(`walls.fill_ghosts`), with the oracle as the stepper of the local periodic grid, must
reproduce the oracle's doubled box restricted to the walled domain."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_1808_10481_gb300 import inputs as I
from paper_1808_10481_gb300 import walls as W

PARITY = {"dirichlet": -1, "neumann": 1}


def _doubled(ncell, walls):
    """Node counts of the periodic unit box that holds the walled box [0, 1/2] per walled axis."""
    return [2 * n if w != "periodic" else n for n, w in zip(ncell, walls)]


def _lengths(walls):
    return [0.5 if w != "periodic" else 1.0 for w in walls]


def _mirror(f, dim, m, nd, k, parity, dual):
    """The reflection x_k -> -x_k of node data f (ncomp, nnode, nq) on the doubled grid nd,
    each component c multiplied by parity[c] and by (-1)^(a_k) per slot."""
    n = m + 1
    nq = n ** dim
    M = nd[k]
    src = np.arange(M)
    src = (M - 1 - src) if dual else (M - src) % M
    g = f.reshape((f.shape[0],) + tuple(reversed(nd)) + (nq,))
    g = np.take(g, src, axis=1 + (dim - 1 - k))
    a = (np.arange(nq) // n ** k) % n
    sign = np.array(parity, dtype=np.float64)[:, None] * (-1.0) ** a[None, :]
    g = g * sign.reshape((f.shape[0],) + (1,) * dim + (nq,))
    return g.reshape(f.shape)


def _parities(dim, kind, k):
    s = PARITY[kind]
    return [s], [(-s if c == k else s) for c in range(dim)]


def _symmetrize(p, u, dim, m, nd, walls, wrong_tangential=False):
    p = p[None].copy()
    u = u.copy()
    for k, w in enumerate(walls):
        if w == "periodic":
            continue
        pp, pu = _parities(dim, w, k)
        if wrong_tangential:
            pu = [(-x if c != k else x) for c, x in enumerate(pu)]
        p = 0.5 * (p + _mirror(p, dim, m, nd, k, pp, dual=False))
        u = 0.5 * (u + _mirror(u, dim, m, nd, k, pu, dual=True))
    return np.ascontiguousarray(p[0]), np.ascontiguousarray(u)


def _restrict_doubled(p, u, dim, m, ncell, walls):
    """The walled domain's nodes of doubled-grid data: primal 0..N and dual 0..N-1 per walled axis."""
    nq = (m + 1) ** dim
    nd = _doubled(ncell, walls)
    ps = tuple(slice(0, n + 1) if w != "periodic" else slice(None) for n, w in zip(reversed(ncell), reversed(walls)))
    us = tuple(slice(0, n) if w != "periodic" else slice(None) for n, w in zip(reversed(ncell), reversed(walls)))
    pr = p.reshape(tuple(reversed(nd)) + (nq,))[ps]
    ur = u.reshape((dim,) + tuple(reversed(nd)) + (nq,))[(slice(None),) + us]
    return np.ascontiguousarray(pr).reshape(-1, nq), np.ascontiguousarray(ur).reshape(dim, -1, nq)


def _wall_mode(dim, m, nd, walls, wave, t_p, t_u):
    """Exact standing mode on the unit box nd that meets the walls at x_k = 0 and 1/2:
    p = cos(w t) prod_k sin(2 pi n_k x_k + phi_k), phi_k = 0 (Dirichlet) or pi/2 (Neumann);
    u_k = -(n_k/|n|) sin(w t) cos(2 pi n_k x_k + phi_k) prod_{j != k} sin(2 pi n_j x_j + phi_j)."""
    nrm = math.sqrt(sum(w * w for w in wave))
    om = 2.0 * math.pi * nrm
    phi = [math.pi / 2 if w == "neumann" else 0.0 for w in walls]
    hs = [1.0 / n for n in nd]
    kap = [2.0 * math.pi * wave[k] for k in range(dim)]
    p = I.tensor_field([I.scaled_trig(I.node_coords(nd[k], False), hs[k], m, kap[k], phi[k])
                        for k in range(dim)]) * math.cos(om * t_p)
    u = np.empty((dim,) + p.shape)
    for k in range(dim):
        fac = [I.scaled_trig(I.node_coords(nd[j], True), hs[j], m, kap[j], phi[j] + (math.pi / 2 if j == k else 0.0))
               for j in range(dim)]
        u[k] = -(wave[k] / nrm) * I.tensor_field(fac) * math.sin(om * t_u)
    return p, u


def _walled_oracle_run(dim, m, ncell, dt, walls, p, u, steps, fill=True):
    """Walled box stepped as the library steps it: the local periodic grid, ghost planes
    filled by walls.fill_ghosts before every step, the oracle as the stepper."""
    loc = W.local_ncell(ncell, walls)
    inv_h = [n / L for n, L in zip(ncell, _lengths(walls))]
    p_loc, u_loc = W.embed(p, u, dim, m, ncell, walls)
    tables = W.mirror_tables(dim, m, walls, "host")
    for _ in range(steps):
        if fill:
            W.fill_ghosts(*W.field_views(p_loc, u_loc, dim, m, loc, "host"), dim, walls, "host", tables)
        p_loc, u_loc = oracle.run(dim, m, loc, dt, p_loc, u_loc, 1, inv_h=inv_h)
    return W.restrict(p_loc, u_loc, dim, m, ncell, walls)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


KIND_SETS = [
    (1, ["dirichlet"]),
    (1, ["neumann"]),
    (2, ["dirichlet", "neumann"]),
    (2, ["neumann", "dirichlet"]),
    (2, ["dirichlet", "periodic"]),
    (3, ["dirichlet", "dirichlet", "neumann"]),
]


# ----------------------------------------------------------------------------- the reading, pinned
@pytest.mark.parametrize("dim,walls", KIND_SETS)
def test_exact_wall_modes_are_mirror_symmetric(dim, walls):
    """The parities follow from the PDE: exact modes meeting the wall conditions are fixed
    points of the mirror map (any wrong sign in the parity table fails here)."""
    m = 3 if dim < 3 else 2
    ncell = [5, 4, 3][:dim]
    nd = _doubled(ncell, walls)
    p, u = _wall_mode(dim, m, nd, walls, [1, 2, 1][:dim], 0.13, 0.17)
    for k, w in enumerate(walls):
        if w == "periodic":
            continue
        pp, pu = _parities(dim, w, k)
        assert _rel(_mirror(p[None], dim, m, nd, k, pp, dual=False)[0], p) < 1e-13
        assert _rel(_mirror(u, dim, m, nd, k, pu, dual=True), u) < 1e-13
        bad = [(-x if c != k else x) for c, x in enumerate(pu)] if dim > 1 else [-pu[0]]
        assert _rel(_mirror(u, dim, m, nd, k, bad, dual=True), u) > 0.1


def test_dirichlet_wall_nodes_hold_zero_pressure():
    """p = 0 on a Dirichlet wall: the mirrored data's even slots vanish at the wall nodes."""
    dim, m, ncell, walls = 1, 3, [6], ["dirichlet"]
    nd = _doubled(ncell, walls)
    rng = np.random.default_rng(1)
    p, u = _symmetrize(rng.uniform(-1, 1, (nd[0], 4)), rng.uniform(-1, 1, (1, nd[0], 4)), dim, m, nd, walls)
    for node in (0, ncell[0]):
        assert abs(p[node, 0]) < 1e-15 and abs(p[node, 2]) < 1e-15


@pytest.mark.parametrize("dim,walls", [(1, ["dirichlet"]), (2, ["dirichlet", "neumann"]),
                                       (3, ["neumann", "dirichlet", "periodic"])])
def test_oracle_keeps_mirrored_data_mirrored(dim, walls):
    """The mirror map is a symmetry of the scheme (the oracle on the doubled box keeps it to
    rounding); the same data with the tangential parity flipped is not preserved."""
    m = 2 if dim < 3 else 1
    ncell = [5, 4, 3][:dim]
    nd = _doubled(ncell, walls)
    nq = (m + 1) ** dim
    nn = int(np.prod(nd))
    rng = np.random.default_rng(7 + dim)
    p0, u0 = rng.uniform(-1, 1, (nn, nq)), rng.uniform(-1, 1, (dim, nn, nq))
    dt = I.cfl_dt(nd)
    p, u = _symmetrize(p0, u0, dim, m, nd, walls)
    p1, u1 = oracle.run(dim, m, nd, dt, p, u, 6)
    ps, us = _symmetrize(p1, u1, dim, m, nd, walls)
    assert _rel(ps, p1) < 1e-13 and _rel(us, u1) < 1e-13
    if dim > 1:
        pb, ub = _symmetrize(p0, u0, dim, m, nd, walls, wrong_tangential=True)
        pb1, ub1 = oracle.run(dim, m, nd, dt, pb, ub, 6)
        pbs, ubs = _symmetrize(pb1, ub1, dim, m, nd, walls, wrong_tangential=True)
        assert max(_rel(pbs, pb1), _rel(ubs, ub1)) > 1e-6


# ----------------------------------------------------------------------------- the library's ghost fill
@pytest.mark.parametrize("dim,walls", KIND_SETS)
def test_ghost_fill_reproduces_exact_ghost_data(dim, walls):
    """Filled ghost planes (corners and edges included) equal the exact mode's data at the
    ghost positions -h/2 and L + h/2."""
    m = 3 if dim < 3 else 2
    ncell = [5, 4, 3][:dim]
    nd = _doubled(ncell, walls)
    nq = (m + 1) ** dim
    p, u = _wall_mode(dim, m, nd, walls, [1, 2, 1][:dim], 0.21, 0.26)
    pw, uw = _restrict_doubled(p, u, dim, m, ncell, walls)
    p_loc, u_loc = W.embed(pw, uw, dim, m, ncell, walls)
    loc = W.local_ncell(ncell, walls)
    W.fill_ghosts(*W.field_views(p_loc, u_loc, dim, m, loc, "host"), dim, walls, "host",
                  W.mirror_tables(dim, m, walls, "host"))
    # exact dual data on the local grid: local plane j <-> doubled dual node j - 1 (walled axes)
    idx = [np.arange(n) - 1 if w != "periodic" else np.arange(n) for n, w in zip(loc, walls)]
    ud = u.reshape((dim,) + tuple(reversed(nd)) + (nq,))
    for k in range(dim):
        ud = np.take(ud, idx[k] % nd[k], axis=1 + (dim - 1 - k))
    assert _rel(u_loc, ud.reshape(u_loc.shape)) < 1e-13


@pytest.mark.parametrize("dim,walls", KIND_SETS)
def test_ghost_fill_device_layout_on_torch_matches_host_layout(dim, walls):
    """The fill on torch tensors in the device layout (what the solver runs on the GPU)
    writes the same values as the numpy host-layout fill."""
    torch = pytest.importorskip("torch")
    m = 2
    ncell = [4, 3, 3][:dim]
    nq = (m + 1) ** dim
    loc = W.local_ncell(ncell, walls)
    nn = int(np.prod(loc))
    rng = np.random.default_rng(3)
    p, u = rng.uniform(-1, 1, (nn, nq)), rng.uniform(-1, 1, (dim, nn, nq))
    ph, uh = p.copy(), u.copy()
    W.fill_ghosts(*W.field_views(ph, uh, dim, m, loc, "host"), dim, walls, "host", W.mirror_tables(dim, m, walls, "host"))
    pt = torch.from_numpy(np.ascontiguousarray(p.T)).contiguous()                        # [q][node]
    ut = torch.from_numpy(np.ascontiguousarray(u.transpose(0, 2, 1))).contiguous()       # [comp][q][node]
    W.fill_ghosts(*W.field_views(pt, ut, dim, m, loc, "device"), dim, walls, "device",
                  W.mirror_tables(dim, m, walls, "device", like=pt))
    np.testing.assert_array_equal(pt.numpy().T, ph)
    np.testing.assert_array_equal(ut.numpy().transpose(0, 2, 1), uh)


def test_embed_restrict_round_trip():
    dim, m, ncell, walls = 2, 1, [4, 3], ["dirichlet", "periodic"]
    nq = (m + 1) ** dim
    rng = np.random.default_rng(0)
    np_, nu = int(np.prod(W.p_counts(ncell, walls))), int(np.prod(W.u_counts(ncell, walls)))
    p, u = rng.standard_normal((np_, nq)), rng.standard_normal((dim, nu, nq))
    p2, u2 = W.restrict(*W.embed(p, u, dim, m, ncell, walls), dim, m, ncell, walls)
    np.testing.assert_array_equal(p2, p)
    np.testing.assert_array_equal(u2, u)
    with pytest.raises(ValueError):
        W.embed(p, u, dim, m, ncell, ["dirichlet", "wall"])


@pytest.mark.parametrize("dim,walls,m,ncell", [
    (1, ["dirichlet"], 3, [10]),
    (1, ["neumann"], 2, [9]),
    (2, ["dirichlet", "neumann"], 2, [5, 6]),
    (2, ["dirichlet", "periodic"], 3, [6, 5]),
    (3, ["dirichlet", "dirichlet", "neumann"], 1, [3, 3, 4]),
])
def test_walled_steps_equal_the_doubled_periodic_box(dim, walls, m, ncell):
    nd = _doubled(ncell, walls)
    nq = (m + 1) ** dim
    nn = int(np.prod(nd))
    rng = np.random.default_rng(100 + dim + m)
    p, u = _symmetrize(rng.uniform(-1, 1, (nn, nq)), rng.uniform(-1, 1, (dim, nn, nq)), dim, m, nd, walls)
    dt = I.cfl_dt(nd)
    steps = 6
    ref_p, ref_u = _restrict_doubled(*oracle.run(dim, m, nd, dt, p, u, steps), dim, m, ncell, walls)
    pw, uw = _restrict_doubled(p, u, dim, m, ncell, walls)
    got_p, got_u = _walled_oracle_run(dim, m, ncell, dt, walls, pw, uw, steps)
    assert _rel(got_p, ref_p) < 1e-12 and _rel(got_u, ref_u) < 1e-12
    # control: without the ghost fill the walls are not closed
    bad_p, _ = _walled_oracle_run(dim, m, ncell, dt, walls, pw, uw, steps, fill=False)
    assert _rel(bad_p, ref_p) > 1e-6


@pytest.mark.parametrize("dim,walls,Ns", [
    (1, ["dirichlet"], [8, 12, 16, 24, 32]),
    (1, ["neumann"], [8, 12, 16, 24, 32]),
    (2, ["dirichlet", "neumann"], [4, 6, 8, 12, 16]),
])
def test_walled_standing_mode_converges_at_the_periodic_rate(dim, walls, Ns):
    """m = 2 on the walled box [0, 1/2]^d against the exact mode: the observed L2 rate is the
    sixth order (2m + 2) that Tables 1 and 5 report for even m on periodic grids, with the
    spread those tables show between runs (5.7 to 6.0 there, up to 6.6 here)."""
    m = 2
    T = 0.25
    errs = []
    for N in Ns:
        ncell = [N] * dim
        nd = _doubled(ncell, walls)
        n = math.ceil(T / (0.9 / nd[0]))
        dt = T / n
        p, u = _wall_mode(dim, m, nd, walls, [1] * dim, 0.0, 0.5 * dt)
        pw, uw = _restrict_doubled(p, u, dim, m, ncell, walls)
        got_p, _ = _walled_oracle_run(dim, m, ncell, dt, walls, pw, uw, n)
        ex_p, _ = _restrict_doubled(*_wall_mode(dim, m, nd, walls, [1] * dim, n * dt, (n + 0.5) * dt),
                                    dim, m, ncell, walls)
        h = 0.5 / N
        errs.append(math.sqrt(h ** dim * float(np.sum((got_p[:, 0] - ex_p[:, 0]) ** 2))))
    rate = float(np.polyfit(np.log(1.0 / np.array(Ns)), np.log(errs), 1)[0])
    assert 5.5 <= rate <= 7.0, (rate, errs)


# ----------------------------------------------------------------------------- on the GPU
@pytest.mark.gpu
@pytest.mark.parametrize("dim,walls,m,ncell", [
    (1, ["dirichlet"], 3, [40]),
    (2, ["dirichlet", "neumann"], 3, [24, 19]),
    (2, ["neumann", "periodic"], 2, [16, 20]),
    (3, ["dirichlet", "dirichlet", "neumann"], 2, [7, 6, 5]),
])
def test_walled_solver_on_the_gpu_matches_the_doubled_box(dim, walls, m, ncell):
    """The CUDA kernels on the local periodic grid with the ghost planes filled on the
    device before every step: the walled box equals the oracle's doubled periodic box,
    restricted, within the FP64 parity bar (1e-12 of the field's maximum)."""
    from paper_1808_10481_gb300 import build, hl
    build.build()
    hl.load()
    nd = _doubled(ncell, walls)
    nq = (m + 1) ** dim
    nn = int(np.prod(nd))
    rng = np.random.default_rng(200 + dim + m)
    p, u = _symmetrize(rng.uniform(-1, 1, (nn, nq)), rng.uniform(-1, 1, (dim, nn, nq)), dim, m, nd, walls)
    dt = I.cfl_dt(nd)
    steps = 10
    ref_p, ref_u = _restrict_doubled(*oracle.run(dim, m, nd, dt, p, u, steps), dim, m, ncell, walls)
    pw, uw = _restrict_doubled(p, u, dim, m, ncell, walls)
    s = W.WalledSolver(dim, m, ncell, dt, walls, length=_lengths(walls))
    try:
        s.set_initial(pw, uw)
        s.step(steps)
        got_p, got_u = s.fields()
    finally:
        s.close()
    assert _rel(got_p, ref_p) <= 1e-12
    assert _rel(got_u, ref_u) <= 1e-12


@pytest.mark.parametrize("kind,sign", [("dirichlet", -1.0), ("neumann", 1.0)])
def test_pulse_reflects_with_the_walls_sign(kind, sign):
    """A right-moving pressure pulse (p = u = g(x - t)) in the walled box [0, 1/2] returns
    from the wall at x = 1/2 inverted by a pressure-release wall and upright from a rigid
    one (the reflection the paper's walled pulse experiment shows in 2D): at t = 1/2 the
    pulse is back at its start, moving left, with p = sign * g."""
    m, N = 3, 64
    ncell, walls = [N], [kind]
    nd = _doubled(ncell, walls)
    h = 1.0 / nd[0]
    x0, w = 0.25, 0.03
    dt = 0.9 * h
    n = math.ceil(0.5 / dt)
    dt = 0.5 / n
    xp = I.node_coords(nd[0], False)[: N + 1]
    xu = I.node_coords(nd[0], True)[:N]
    p = I.scaled_gauss(xp, h, m, x0, w, images=(0,))
    u = I.scaled_gauss(xu, h, m, x0 + 0.5 * dt, w, images=(0,))[None]
    got_p, _ = _walled_oracle_run(1, m, ncell, dt, walls, p, u, n)
    want = sign * I.scaled_gauss(xp, h, m, x0, w, images=(0,))[:, 0]
    assert np.abs(got_p[:, 0] - want).max() < 1e-3
    if kind == "dirichlet":
        assert abs(got_p[0, 0]) < 1e-12 and abs(got_p[N, 0]) < 1e-12


def _tm_mode(m, N, L, t_p, t_u, a=16, b=16):
    """Maxwell TM field E_z = sin(kx x) sin(ky y) cos(w t) on [0, L]^2 with perfectly
    conducting walls (E_z = 0 on all four), as p = E_z and u = (-H_y, H_x):
    u_x = -(kx/w) cos(kx x) sin(ky y) sin(w t), u_y = -(ky/w) sin(kx x) cos(ky y) sin(w t),
    kx = 2 pi a, ky = 2 pi b, w = |k|.  Returns the walled-domain host layout (p on the
    (N+1)^2 primal nodes at t_p, u on the N^2 dual nodes at t_u)."""
    h = L / N
    kx, ky = 2 * math.pi * a, 2 * math.pi * b
    w = math.hypot(kx, ky)
    xp = np.arange(N + 1) * h
    xd = (np.arange(N) + 0.5) * h

    def tensor(fx, fy):  # x fastest, slot a_x fastest
        return np.einsum("ia,jb->jiba", fx, fy).reshape(fx.shape[0] * fy.shape[0], -1)
    sx, sy = I.scaled_trig(xp, h, m, kx, 0.0), I.scaled_trig(xp, h, m, ky, 0.0)
    p = tensor(sx, sy) * math.cos(w * t_p)
    sxd, syd = I.scaled_trig(xd, h, m, kx, 0.0), I.scaled_trig(xd, h, m, ky, 0.0)
    cxd, cyd = I.scaled_trig(xd, h, m, kx, math.pi / 2), I.scaled_trig(xd, h, m, ky, math.pi / 2)
    u = np.stack([-(kx / w) * tensor(cxd, syd), -(ky / w) * tensor(sxd, cyd)]) * math.sin(w * t_u)
    return p, u


@pytest.mark.gpu
@pytest.mark.parametrize("m", [3, 4, 5, 6])
def test_maxwell_tm_with_conducting_walls_converges(m):
    """Section 5.3's high-frequency Maxwell TM experiment on the GPU through hl_set_walls:
    omega_x = omega_y = 8 pi on [-1, 1] is 16 periods per unit on the walled square
    [0, 1/2]^2 here, perfect conductors (HL_WALL_DIRICHLET for E_z) on all four walls,
    C_CFL = 0.8, m = 3..6.  The L2 error of E_z against the exact mode falls with the grid
    at high order and ends small, as the paper's Maxwell figure shows."""
    from paper_1808_10481_gb300 import build, hl
    build.build()
    hl.load()
    L, T = 0.5, 0.125
    errs, Ns = [], [24, 32, 48]
    for N in Ns:
        h = L / N
        steps = math.ceil(T / (0.8 * h))
        dt = T / steps
        p0, u0 = _tm_mode(m, N, L, 0.0, 0.5 * dt)
        s = W.WalledSolver(2, m, [N, N], dt, ["dirichlet", "dirichlet"], length=[L, L])
        try:
            s.set_initial(p0, u0)
            s.step(steps)
            got_p, _ = s.fields()
        finally:
            s.close()
        ex, _ = _tm_mode(m, N, L, steps * dt, (steps + 0.5) * dt)
        errs.append(math.sqrt(h * h * float(np.sum((got_p[:, 0] - ex[:, 0]) ** 2))))
    rate = float(np.polyfit(np.log(1.0 / np.array(Ns)), np.log(errs), 1)[0])
    print(f"Maxwell TM m={m}: L2 errors {errs}, rate {rate:.2f}")
    assert rate >= 2 * m - 1, (m, rate, errs)
    assert errs[-1] < {3: 1e-7, 4: 1e-7, 5: 1e-10, 6: 1e-12}[m], (m, errs)


@pytest.mark.gpu
def test_walls_in_graph_mode_and_tc_split_match_fp64_steps():
    """The ghost fill is stream-ordered: the same walled run captured as one CUDA graph, and
    run with the tensor-core split contraction, matches the FP64 launches (the split mode
    within its error bound)."""
    from paper_1808_10481_gb300 import build, hl
    build.build()
    hl.load()
    m, N, L = 3, 40, 0.5
    dt = 0.8 * L / N
    p0, u0 = _tm_mode(m, N, L, 0.0, 0.5 * dt, a=2, b=3)
    out = {}
    for name, graph, prec in (("plain", 0, hl.HL_FP64), ("graph", 1, hl.HL_FP64), ("tc", 0, hl.HL_TC_SPLIT)):
        s = W.WalledSolver(2, m, [N, N], dt, ["dirichlet", "neumann"], length=[L, L])
        try:
            hl.hl_set_option(s.h, hl.HL_OPT_GRAPH, graph)
            hl.hl_set_precision(s.h, prec)
            s.set_initial(p0, u0)
            s.step(30)
            out[name] = s.fields()
        finally:
            s.close()
    np.testing.assert_array_equal(out["graph"][0], out["plain"][0])
    np.testing.assert_array_equal(out["graph"][1], out["plain"][1])
    assert _rel(out["tc"][0], out["plain"][0]) < 1e-10 and _rel(out["tc"][1], out["plain"][1]) < 1e-10


@pytest.mark.gpu
def test_3d_walls_in_tc_split_match_the_doubled_box():
    """3D walls with the tensor-core split contraction (field digit planes cut after every
    ghost fill): the walled box equals the oracle's doubled periodic box, restricted, within
    the split mode's error (its bound at this size is far above 1e-10; measured ~1e-12)."""
    from paper_1808_10481_gb300 import build, hl
    build.build()
    hl.load()
    dim, m, ncell, walls = 3, 2, [7, 6, 5], ["dirichlet", "neumann", "periodic"]
    nd = _doubled(ncell, walls)
    nq = (m + 1) ** dim
    nn = int(np.prod(nd))
    rng = np.random.default_rng(231)
    p, u = _symmetrize(rng.uniform(-1, 1, (nn, nq)), rng.uniform(-1, 1, (dim, nn, nq)), dim, m, nd, walls)
    dt = I.cfl_dt(nd)
    steps = 6
    ref_p, ref_u = _restrict_doubled(*oracle.run(dim, m, nd, dt, p, u, steps, prec="dd"), dim, m, ncell, walls)
    pw, uw = _restrict_doubled(p, u, dim, m, ncell, walls)
    s = W.WalledSolver(dim, m, ncell, dt, walls, length=_lengths(walls))
    try:
        hl.hl_set_precision(s.h, hl.HL_TC_SPLIT)
        s.set_initial(pw, uw)
        s.step(steps)
        got_p, got_u = s.fields()
    finally:
        s.close()
    print("3D walls, tensor-core split vs doubled box:", _rel(got_p, ref_p), _rel(got_u, ref_u))
    assert _rel(got_p, ref_p) <= 1e-10 and _rel(got_u, ref_u) <= 1e-10
