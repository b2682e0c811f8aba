"""The host glue of `walls.WalledSolver` and `halo.SlabSolver` on the CPU.

The two classes bind device buffers to a solver handle, fill or exchange ghost planes in
those buffers (device layout) and call hl_step between the fills.  Here the binding is
replaced by a stand-in that keeps the bound buffers as CPU tensors and steps them with the
oracle (converting the device layout to the host layout and back), so that everything the
classes do around the kernels runs as on the GPU: buffer shapes, layout views, the order
of fills and steps, embedding and restriction.  The CUDA kernels themselves are covered by
the GPU tests."""
from __future__ import annotations

import contextlib
import sys
import types

import numpy as np
import pytest

import oracle
from paper_1808_10481_gb300 import halo
from paper_1808_10481_gb300 import inputs as I
from paper_1808_10481_gb300 import walls as W

torch = pytest.importorskip("torch")


class _Handle:
    def __init__(self, dim, m, n, inv_h, dt):
        self.dim, self.m, self.n, self.inv_h, self.dt = dim, m, list(n), list(inv_h), dt
        self.nq = (m + 1) ** dim
        self.nn = int(np.prod(n))
        self.p = self.u = None
        self.steps = 0


def _fake_binding():
    """A stand-in for paper_1808_10481_gb300.hl with the calls the two classes make."""
    hl = types.SimpleNamespace()
    hl.hl_create_spacing = lambda dim, m, n, inv_h, dt: _Handle(dim, m, n, inv_h, dt)
    hl.hl_set_stream = lambda h, s: None

    def bind(h, p, u):
        assert p.numel() == h.nq * h.nn and u.numel() == h.dim * h.nq * h.nn
        h.p, h.u = p, u
    hl.hl_bind_device = bind

    def set_initial(h, p, u):
        p = np.asarray(p).reshape(h.nn, h.nq)
        u = np.asarray(u).reshape(h.dim, h.nn, h.nq)
        h.p.view(h.nq, h.nn)[:] = torch.from_numpy(np.ascontiguousarray(p.T))
        h.u.view(h.dim, h.nq, h.nn)[:] = torch.from_numpy(np.ascontiguousarray(u.transpose(0, 2, 1)))
        h.steps = 0
    hl.hl_set_initial = set_initial

    def host(h):
        return (np.ascontiguousarray(h.p.view(h.nq, h.nn).numpy().T),
                np.ascontiguousarray(h.u.view(h.dim, h.nq, h.nn).numpy().transpose(0, 2, 1)))

    def set_walls(h, kinds):
        h.walls = None if kinds is None else list(kinds)
    hl.hl_set_walls = set_walls

    def step(h, n):
        # as the library: with walls, the ghost planes are filled (in the device layout)
        # before every step; without, the steps run at once
        walls = getattr(h, "walls", None)
        if walls is None:
            p, u = oracle.run(h.dim, h.m, h.n, h.dt, *host(h), int(n), inv_h=h.inv_h)
            set_initial(h, p, u)
            return
        tables = W.mirror_tables(h.dim, h.m, walls, "device", like=h.p)
        for _ in range(int(n)):
            W.fill_ghosts(*W.field_views(h.p, h.u, h.dim, h.m, h.n, "device"), h.dim, walls, "device", tables)
            p, u = oracle.run(h.dim, h.m, h.n, h.dt, *host(h), 1, inv_h=h.inv_h)
            set_initial(h, p, u)
    hl.hl_step = step
    hl.hl_get_fields = lambda h: host(h) + (0.0, 0.0)
    hl.hl_destroy = lambda h: None
    return hl


@pytest.fixture
def fake_gpu(monkeypatch):
    """CPU tensors where the classes ask for CUDA ones, and the stand-in binding."""
    fake = _fake_binding()
    zeros = torch.zeros
    monkeypatch.setattr(torch, "zeros", lambda *a, **k: zeros(*a, **{x: v for x, v in k.items() if x != "device"}))
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    import paper_1808_10481_gb300 as pkg
    monkeypatch.setitem(sys.modules, "paper_1808_10481_gb300.hl", fake)
    monkeypatch.setattr(pkg, "hl", fake, raising=False)
    return fake


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dim,walls,m,ncell", [
    (1, ["dirichlet"], 3, [12]),
    (2, ["dirichlet", "neumann"], 2, [6, 5]),
    (2, ["neumann", "periodic"], 2, [5, 6]),
    (3, ["dirichlet", "dirichlet", "neumann"], 1, [3, 4, 3]),
])
def test_walled_solver_glue(fake_gpu, dim, walls, m, ncell):
    import test_walls as T
    nd = T._doubled(ncell, walls)
    nq = (m + 1) ** dim
    nn = int(np.prod(nd))
    rng = np.random.default_rng(300 + dim + m)
    p, u = T._symmetrize(rng.uniform(-1, 1, (nn, nq)), rng.uniform(-1, 1, (dim, nn, nq)), dim, m, nd, walls)
    dt = I.cfl_dt(nd)
    ref_p, ref_u = T._restrict_doubled(*oracle.run(dim, m, nd, dt, p, u, 5), dim, m, ncell, walls)
    s = W.WalledSolver(dim, m, ncell, dt, walls, length=T._lengths(walls))
    try:
        s.set_initial(*T._restrict_doubled(p, u, dim, m, ncell, walls))
        s.step(5)
        got_p, got_u = s.fields()
    finally:
        s.close()
    assert _rel(got_p, ref_p) < 1e-12 and _rel(got_u, ref_u) < 1e-12


@pytest.mark.parametrize("dim,m,ncell,world", [(1, 3, [11], 2), (2, 2, [5, 7], 3), (3, 1, [3, 3, 5], 2)])
def test_slab_solver_glue(fake_gpu, dim, m, ncell, world):
    st = I.random_state(dim, m, ncell, seed=40 + world)
    dt = I.cfl_dt(ncell)
    ref_p, ref_u = oracle.run(dim, m, ncell, dt, st.p, st.u, 4)
    slabs = [halo.SlabSolver(dim, m, ncell, dt, pl) for pl in halo.slab_planes(ncell[-1], world)]
    for s in slabs:
        s.set_initial(st.p, st.u)
    halo.step_slabs(slabs, 4)
    parts = [s.owned_fields() for s in slabs]
    for s in slabs:
        s.close()
    np.testing.assert_array_equal(np.concatenate([x[0] for x in parts], axis=0), ref_p)
    np.testing.assert_array_equal(np.concatenate([x[1] for x in parts], axis=1), ref_u)
