"""Slab decomposition of one periodic grid over several ranks, with ghost-plane exchange.

The grid is cut along its slowest axis (x in 1D, y in 2D, z in 3D).  Nodes
are numbered x-fastest, so one plane of that axis is a contiguous run of
nodes in both the host layout f[comp][node][q] and the device layout
f[comp][q][node].  Rank r owns global planes [a_r, b_r), L_r = b_r - a_r of
them, and holds L_r + 2 planes:

    local plane 0          ghost copy of global plane a_r - 1
    local planes 1..L_r    the owned planes a_r .. b_r - 1
    local plane L_r + 1    ghost copy of global plane b_r

(global indices periodic).  The local grid is stepped as a periodic grid of
L_r + 2 planes with the GLOBAL spacing (`hl_create_spacing` with 1/h_k of the
whole grid), so its wrap-around joins the two ghost planes to each other.

One exchange before every full step is enough.  In the staggering of
Section 2 the p-half at primal plane i reads the dual planes i-1 and i, and
the u-half at dual plane i reads the primal planes i and i+1.  If every local
plane holds the right data when a step starts:

  * p-half: primal planes 1..L+1 read dual planes 0..L+1, all right.  Primal
    plane 0 reads dual plane -1, which the wrap turns into plane L+1, so
    primal plane 0 comes out wrong;
  * u-half: dual planes 1..L read primal planes 1..L+1, all right.  Dual
    planes 0 and L+1 read the wrong primal plane 0 and come out wrong.

So the owned planes 1..L of both grids are right after the step, and copying
the neighbours' edge planes into the four ghost planes (p and u, local planes
0 and L+1) restores the starting condition.  Every owned node goes through
exactly the arithmetic it goes through on the undivided grid: the result is
the same bit for bit.

This module holds the index logic and the exchange, for any stepper: the
solver library on a GPU (`SlabSolver`) or any other implementation of the
same update.  Transport is torch.distributed point-to-point (NCCL between
GPUs, gloo on the CPU) or plain copies between slabs held by one process.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- index logic
def slab_planes(n: int, world: int) -> list[tuple[int, int]]:
    """Owned plane ranges [a, b) of an axis of n planes over `world` ranks: contiguous,
    in rank order, sizes differing by at most one (the first n % world ranks get the
    larger share)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if n < world:
        raise ValueError("every rank needs at least one plane (n >= world)")
    base, extra = divmod(n, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def local_ncell(ncell, planes: tuple[int, int]) -> list[int]:
    """Node counts of one rank's local grid: the slowest axis holds L + 2 planes."""
    a, b = planes
    out = [int(x) for x in ncell]
    out[-1] = (b - a) + 2
    return out


def spacing(ncell) -> list[float]:
    """1/h_k of the undivided unit-box grid (what every slab is created with)."""
    return [float(x) for x in ncell]


def local_planes(n: int, planes: tuple[int, int]) -> np.ndarray:
    """Global plane index of every local plane: ghost, owned..., ghost (periodic)."""
    a, b = planes
    return np.concatenate([[(a - 1) % n], np.arange(a, b), [b % n]]).astype(np.int64)


def plane_view(t, ncomp: int, nplanes: int, plane_nodes: int, nq: int, layout: str):
    """A (rows, nplanes, plane_elems) view of a field buffer, for either layout.

    layout "host": f[comp][node][q]  -> (ncomp, nplanes, plane_nodes * nq)
    layout "device": f[comp][q][node] -> (ncomp * nq, nplanes, plane_nodes)
    Works on numpy arrays and torch tensors; the buffer must be contiguous."""
    if layout == "host":
        return t.reshape(ncomp, nplanes, plane_nodes * nq)
    if layout == "device":
        return t.reshape(ncomp * nq, nplanes, plane_nodes)
    raise ValueError("layout must be 'host' or 'device'")


def extract(field, ncell, nq: int, ncomp: int, planes: tuple[int, int]):
    """One rank's local field, ghost planes filled, from a global field in host layout
    (ncomp, nnode, nq).  Returns (ncomp, (L + 2) * plane_nodes, nq)."""
    n = int(ncell[-1])
    plane_nodes = int(np.prod(ncell[:-1])) if len(ncell) > 1 else 1
    v = plane_view(field, ncomp, n, plane_nodes, nq, "host")
    idx = local_planes(n, planes)
    loc = v[:, idx] if isinstance(v, np.ndarray) else v[:, _as_index(idx, v)]
    return loc.reshape(ncomp, len(idx) * plane_nodes, nq)


def owned(local, ncell, nq: int, ncomp: int, planes: tuple[int, int]):
    """The owned planes of a local host-layout field: (ncomp, L * plane_nodes, nq)."""
    a, b = planes
    plane_nodes = int(np.prod(ncell[:-1])) if len(ncell) > 1 else 1
    v = plane_view(local, ncomp, (b - a) + 2, plane_nodes, nq, "host")
    return v[:, 1:1 + (b - a)].reshape(ncomp, (b - a) * plane_nodes, nq)


def _as_index(idx: np.ndarray, like):
    import torch
    return torch.as_tensor(idx, device=like.device)


# ----------------------------------------------------------------------------- exchange
def exchange_local(views) -> None:
    """Refresh the ghost planes of slabs held by one process, in rank order.

    views[r]: the (rows, L_r + 2, plane_elems) view of one field of rank r (numpy
    or torch, same rows and plane size on every rank).  Ghost planes are written,
    owned planes only read, so one rank alone (periodic wrap) works too."""
    world = len(views)
    for r in range(world):
        below, above = views[(r - 1) % world], views[(r + 1) % world]
        views[r][:, 0] = below[:, below.shape[1] - 2]
        views[r][:, views[r].shape[1] - 1] = above[:, 1]


_TAG_UP, _TAG_DOWN = 0, 1


def exchange(view, rank: int, world: int, dist) -> None:
    """Refresh one rank's ghost planes from its neighbours over torch.distributed.

    view: this rank's (rows, L + 2, plane_elems) torch view of one field.  The last
    owned plane goes up (to rank + 1, its ghost plane 0), the first owned plane goes
    down (to rank - 1, its ghost plane L + 1).  Two ranks are each other's upper and
    lower neighbour; the tags (gloo) and the fixed order of the operations (NCCL
    matches in issue order) keep the two messages apart."""
    if world == 1:
        exchange_local([view])
        return
    import torch
    L2 = view.shape[1]
    up, down = (rank + 1) % world, (rank - 1) % world
    send_up = view[:, L2 - 2].contiguous()
    send_down = view[:, 1].contiguous()
    recv_below = torch.empty_like(send_up)
    recv_above = torch.empty_like(send_down)
    ops = [
        dist.P2POp(dist.isend, send_up, up, tag=_TAG_UP),
        dist.P2POp(dist.isend, send_down, down, tag=_TAG_DOWN),
        dist.P2POp(dist.irecv, recv_below, down, tag=_TAG_UP),
        dist.P2POp(dist.irecv, recv_above, up, tag=_TAG_DOWN),
    ]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    view[:, 0] = recv_below
    view[:, L2 - 1] = recv_above


# ----------------------------------------------------------------------------- the solver on one slab
class SlabSolver:
    """One rank's slab, stepped by the solver library on the current CUDA device.

    The state lives in two caller-owned device buffers bound to the handle
    (hl_bind_device, device layout); the ghost planes of both are refreshed by
    `exchange_fn(p_view, u_view)` before every step, all on one stream."""

    def __init__(self, dim: int, m: int, ncell, dt: float, planes: tuple[int, int], stream=None):
        import torch

        from . import hl
        self.hl = hl
        self.dim, self.m, self.ncell, self.dt, self.planes = dim, m, [int(x) for x in ncell], float(dt), planes
        self.nq = (m + 1) ** dim
        self.local = local_ncell(ncell, planes)
        self.plane_nodes = int(np.prod(self.local[:-1])) if dim > 1 else 1
        self.nnode = int(np.prod(self.local))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = hl.hl_create_spacing(dim, m, self.local, spacing(ncell), dt)
        hl.hl_set_stream(self.h, self.stream)
        self.p = torch.zeros(self.nq * self.nnode, dtype=torch.float64, device="cuda")
        self.u = torch.zeros(dim * self.nq * self.nnode, dtype=torch.float64, device="cuda")
        hl.hl_bind_device(self.h, self.p, self.u)

    def views(self):
        """(p, u) as (rows, L + 2, plane_nodes) views of the bound device buffers."""
        n2 = self.local[-1]
        return (plane_view(self.p, 1, n2, self.plane_nodes, self.nq, "device"),
                plane_view(self.u, self.dim, n2, self.plane_nodes, self.nq, "device"))

    def set_initial(self, p, u) -> None:
        """Global host-layout initial data (p at 0, u at dt/2); this rank takes its planes."""
        p = np.ascontiguousarray(extract(np.asarray(p).reshape(1, -1, self.nq), self.ncell, self.nq, 1, self.planes))
        u = np.ascontiguousarray(extract(np.asarray(u).reshape(self.dim, -1, self.nq), self.ncell, self.nq,
                                         self.dim, self.planes))
        self.hl.hl_set_initial(self.h, p.reshape(-1, self.nq), u)

    def step(self, n_steps: int, exchange_fn) -> None:
        import torch
        with torch.cuda.stream(self.stream):
            for _ in range(int(n_steps)):
                exchange_fn(*self.views())
                self.hl.hl_step(self.h, 1)

    def owned_fields(self):
        """Host copies of the owned planes: p (L * plane_nodes, nq), u (dim, L * plane_nodes, nq)."""
        p, u, _, _ = self.hl.hl_get_fields(self.h)
        return (owned(p.reshape(1, -1, self.nq), self.ncell, self.nq, 1, self.planes)[0],
                owned(u.reshape(self.dim, -1, self.nq), self.ncell, self.nq, self.dim, self.planes))

    def close(self) -> None:
        if self.h is not None:
            self.hl.hl_destroy(self.h)
            self.h = None


def step_slabs(slabs, n_steps: int) -> None:
    """Step slabs that one process holds on one device (their ghosts exchanged by copies).
    All slabs must share one stream, so that copies and steps stay in order."""
    import torch
    raw = [getattr(s.stream, "cuda_stream", s.stream) for s in slabs]
    if any(r != raw[0] for r in raw):
        raise ValueError("slabs stepped together must share one stream")
    with torch.cuda.stream(slabs[0].stream):
        for _ in range(int(n_steps)):
            views = [s.views() for s in slabs]
            exchange_local([v[0] for v in views])
            exchange_local([v[1] for v in views])
            for s in slabs:
                s.hl.hl_step(s.h, 1)
