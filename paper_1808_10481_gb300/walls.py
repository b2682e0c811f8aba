"""Reflecting walls by ghost mirroring, on the periodic kernels.

Section 5.2 of the paper closes the box with walls by filling ghost nodes of
the velocity (dual) grid before every pressure update, with values that
mirror the velocity polynomials across the wall, even or odd as the boundary
condition demands.  Section 5.3 uses the same mirroring for Maxwell's
equations in transverse-magnetic form, which is this acoustic system with
p = E_z and u = (-H_y, H_x).

Wall kinds along an axis k (the domain is [0, L_k] with N_k cells):
  * "dirichlet": p = 0 on the walls (a pressure-release wall, or a perfect
    conductor for E_z).  p is odd across the wall, so the normal velocity u_k
    (u_k,t = -d_k p) is even and the tangential velocities u_j, j != k, are odd;
  * "neumann": d_k p = 0 on the walls (a rigid wall, u_k = 0).  p is even,
    u_k odd, u_j even;
  * "periodic": no walls along k.
Mirroring a field of parity s across a wall negates the derivative order
along k: the scaled derivative a_k of the ghost is s (-1)^{a_k} times that
of its mirror node.

Nodes.  Along a walled axis the primal grid holds N + 1 nodes, x = i h for
i = 0..N (both walls are primal nodes), and the dual grid N nodes,
x = (i + 1/2) h for i = 0..N-1; two dual ghosts sit at -h/2 and L + h/2.
The solver steps a periodic grid of N + 2 planes along that axis with the
spacing h = L/N (hl_create_spacing):

    local plane     0        1 .. N+1        N+2 = wrap to 0
    primal          unused   i = 0 .. N
    dual            ghost    i = 0 .. N-1,   plane N+1 ghost

The p-half at local primal plane j reads dual planes j-1 and j, so the wall
nodes (planes 1 and N+1) read the ghosts; the u-half at dual plane j reads
primal planes j and j+1, so dual planes 1..N read primal planes 1..N+1 only.
What the wrap feeds into the unused primal plane 0 and into the ghost planes
is never read by a domain node before the ghosts are filled again, so one
fill per step (before its p-half) closes the walls.  Axes are filled in
order 0, 1, 2, each from planes that already hold the previous axes'
ghosts, so corner and edge ghosts get the product of the mirrors.

The exact discrete counterpart is the method of images: the walled solution
is the periodic solution on the domain doubled across each walled axis, with
initial data extended by the same parities.
"""
from __future__ import annotations

import numpy as np

KINDS = ("periodic", "dirichlet", "neumann")


def _check_walls(dim: int, walls) -> list[str]:
    walls = [walls] * dim if isinstance(walls, str) else list(walls)
    if len(walls) != dim or any(w not in KINDS for w in walls):
        raise ValueError(f"walls must be one of {KINDS} per axis")
    return walls


def p_parity(kind: str) -> int:
    """Parity of p across a wall of this kind (-1 odd, +1 even)."""
    return {"dirichlet": -1, "neumann": 1}[kind]


def u_mirror_factors(dim: int, m: int, axis: int, kind: str) -> np.ndarray:
    """(dim, nq) signs: ghost slot q of u component c = sign * the mirror node's slot q."""
    s = p_parity(kind)
    n = m + 1
    nq = n ** dim
    out = np.empty((dim, nq))
    for c in range(dim):
        parity = -s if c == axis else s
        for q in range(nq):
            a = (q // n ** axis) % n
            out[c, q] = parity * (-1.0) ** a
    return out


def p_counts(ncell, walls) -> list[int]:
    """Primal nodes per axis of the walled domain."""
    return [int(n) + (0 if w == "periodic" else 1) for n, w in zip(ncell, walls)]


def u_counts(ncell, walls) -> list[int]:
    """Dual nodes per axis of the walled domain."""
    return [int(n) for n in ncell]


def local_ncell(ncell, walls) -> list[int]:
    """Planes per axis of the periodic grid the solver steps."""
    return [int(n) + (0 if w == "periodic" else 2) for n, w in zip(ncell, walls)]


def _domain_slices(counts, walls):
    # numpy axis order of a (n_{d-1}, ..., n_0) node block: x last
    return tuple(slice(0, c) if w == "periodic" else slice(1, 1 + c)
                 for c, w in zip(reversed(counts), reversed(walls)))


def embed(p, u, dim: int, m: int, ncell, walls):
    """Walled-domain host-layout data -> the local periodic grid's host layout.

    p: (prod p_counts, nq); u: (dim, prod u_counts, nq).  Returns (p_loc, u_loc)
    of shapes (prod local, nq) and (dim, prod local, nq); unused and ghost
    planes are zero."""
    walls = _check_walls(dim, walls)
    nq = (m + 1) ** dim
    loc = local_ncell(ncell, walls)
    pc, uc = p_counts(ncell, walls), u_counts(ncell, walls)
    p_loc = np.zeros(tuple(reversed(loc)) + (nq,))
    u_loc = np.zeros((dim,) + tuple(reversed(loc)) + (nq,))
    p_loc[_domain_slices(pc, walls)] = np.asarray(p).reshape(tuple(reversed(pc)) + (nq,))
    u_loc[(slice(None),) + _domain_slices(uc, walls)] = np.asarray(u).reshape((dim,) + tuple(reversed(uc)) + (nq,))
    n = int(np.prod(loc))
    return p_loc.reshape(n, nq), u_loc.reshape(dim, n, nq)


def restrict(p_loc, u_loc, dim: int, m: int, ncell, walls):
    """The inverse of embed: the walled domain's p (prod p_counts, nq) and u (dim, prod u_counts, nq)."""
    walls = _check_walls(dim, walls)
    nq = (m + 1) ** dim
    loc = local_ncell(ncell, walls)
    pc, uc = p_counts(ncell, walls), u_counts(ncell, walls)
    p = np.asarray(p_loc).reshape(tuple(reversed(loc)) + (nq,))[_domain_slices(pc, walls)]
    u = np.asarray(u_loc).reshape((dim,) + tuple(reversed(loc)) + (nq,))[(slice(None),) + _domain_slices(uc, walls)]
    return (np.ascontiguousarray(p).reshape(-1, nq),
            np.ascontiguousarray(u).reshape(dim, -1, nq))


def _select(view, ax: int, i: int):
    idx = [slice(None)] * view.ndim
    idx[ax] = i
    return tuple(idx)


def field_views(p, u, dim: int, m: int, loc, layout: str):
    """Node-indexed views of the local p and u buffers.

    layout "host"   (f[comp][node][q]): p -> (1, n_{d-1}, .., n_0, nq), u -> (dim, .., nq)
    layout "device" (f[comp][q][node]): p -> (1, nq, n_{d-1}, .., n_0), u -> (dim, nq, ..)
    Works on numpy arrays and torch tensors (contiguous buffers)."""
    nq = (m + 1) ** dim
    nodes = tuple(reversed([int(x) for x in loc]))
    if layout == "host":
        return p.reshape((1,) + nodes + (nq,)), u.reshape((dim,) + nodes + (nq,))
    if layout == "device":
        return p.reshape((1, nq) + nodes), u.reshape((dim, nq) + nodes)
    raise ValueError("layout must be 'host' or 'device'")


def mirror_tables(dim: int, m: int, walls, layout: str, like=None):
    """Per walled axis, the u sign table shaped to broadcast over one ghost plane."""
    walls = _check_walls(dim, walls)
    nq = (m + 1) ** dim
    out = {}
    for k, w in enumerate(walls):
        if w == "periodic":
            continue
        f = u_mirror_factors(dim, m, k, w)
        # one plane has the node axes minus one
        shape = (dim,) + (1,) * (dim - 1) + (nq,) if layout == "host" else (dim, nq) + (1,) * (dim - 1)
        f = f.reshape(shape)
        if like is not None and not isinstance(like, np.ndarray):
            import torch
            f = torch.as_tensor(f, dtype=like.dtype, device=like.device)
        out[k] = f
    return out


def fill_ghosts(p_view, u_view, dim: int, walls, layout: str, tables) -> None:
    """Fill the u ghost planes of every walled axis (axes in order) and clear the unused
    primal plane 0.  p_view, u_view from field_views; tables from mirror_tables."""
    walls = _check_walls(dim, walls)
    node0 = 1 if layout == "host" else 2          # first node axis in the views
    for k, w in enumerate(walls):
        if w == "periodic":
            continue
        ax = node0 + (dim - 1 - k)
        n = u_view.shape[ax]
        f = tables[k]
        u_view[_select(u_view, ax, 0)] = u_view[_select(u_view, ax, 1)] * f
        u_view[_select(u_view, ax, n - 1)] = u_view[_select(u_view, ax, n - 2)] * f
        p_view[_select(p_view, ax, 0)] = 0.0


class WalledSolver:
    """A walled box stepped by the solver library on the current CUDA device.

    ncell: cells per axis; walls: one kind per axis (or one for all); length:
    L_k per axis (default 1).  The state lives in two device buffers bound to
    the handle (device layout); the library fills the u ghost planes before
    every step inside hl_step (hl_set_walls), so a run of n steps is one call."""

    def __init__(self, dim: int, m: int, ncell, dt: float, walls, length=None, stream=None):
        import torch

        from . import hl
        self.hl = hl
        self.dim, self.m = dim, m
        self.ncell = [int(x) for x in ncell]
        self.walls = _check_walls(dim, walls)
        self.length = [1.0] * dim if length is None else [float(x) for x in length]
        self.nq = (m + 1) ** dim
        self.local = local_ncell(self.ncell, self.walls)
        nnode = int(np.prod(self.local))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        inv_h = [n / L for n, L in zip(self.ncell, self.length)]
        self.h = hl.hl_create_spacing(dim, m, self.local, inv_h, dt)
        hl.hl_set_stream(self.h, self.stream)
        self.p = torch.zeros(self.nq * nnode, dtype=torch.float64, device="cuda")
        self.u = torch.zeros(dim * self.nq * nnode, dtype=torch.float64, device="cuda")
        hl.hl_bind_device(self.h, self.p, self.u)
        hl.hl_set_walls(self.h, self.walls)

    def set_initial(self, p, u) -> None:
        """Walled-domain host-layout data: p at t = 0 on the primal nodes, u at dt/2 on the dual nodes."""
        p_loc, u_loc = embed(p, u, self.dim, self.m, self.ncell, self.walls)
        self.hl.hl_set_initial(self.h, np.ascontiguousarray(p_loc), np.ascontiguousarray(u_loc))

    def step(self, n_steps: int) -> None:
        self.hl.hl_step(self.h, int(n_steps))

    def fields(self):
        """Host copies of the walled domain's p (prod p_counts, nq) and u (dim, prod u_counts, nq)."""
        p_loc, u_loc, _, _ = self.hl.hl_get_fields(self.h)
        return restrict(p_loc, u_loc, self.dim, self.m, self.ncell, self.walls)

    def close(self) -> None:
        if self.h is not None:
            self.hl.hl_destroy(self.h)
            self.h = None
