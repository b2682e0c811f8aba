"""Slab decomposition with ghost-plane exchange, checked on the CPU with the oracle as the
per-rank stepper: slabs stepped one step at a time with their ghosts refreshed in between
must reproduce the undivided grid bit for bit (every owned node sees the same operands), in
one process (1 to 4 slabs, ragged plane counts) and over two or three gloo ranks."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1808_10481_gb300 import halo
from paper_1808_10481_gb300 import inputs as I

CASES = [
    (1, 3, [13]),
    (2, 2, [7, 11]),
    (2, 3, [5, 6]),
    (3, 1, [4, 3, 7]),
]


def test_slab_planes_partition_and_balance():
    for n in (2, 5, 7, 64, 101):
        for world in range(1, min(n, 6) + 1):
            parts = halo.slab_planes(n, world)
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a < b for a, b in parts)
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        halo.slab_planes(3, 4)
    with pytest.raises(ValueError):
        halo.slab_planes(3, 0)


def test_local_planes_wrap():
    assert list(halo.local_planes(10, (0, 4))) == [9, 0, 1, 2, 3, 4]
    assert list(halo.local_planes(10, (7, 10))) == [6, 7, 8, 9, 0]
    assert list(halo.local_planes(3, (0, 3))) == [2, 0, 1, 2, 0]
    assert halo.local_ncell([8, 10], (7, 10)) == [8, 5]


def test_extract_and_owned_round_trip():
    d, m, ncell = 2, 1, [3, 7]
    nq = (m + 1) ** d
    rng = np.random.default_rng(3)
    u = rng.standard_normal((d, 21, nq))
    parts = halo.slab_planes(ncell[-1], 3)
    back = np.concatenate([halo.owned(halo.extract(u, ncell, nq, d, pl), ncell, nq, d, pl) for pl in parts], axis=1)
    np.testing.assert_array_equal(back, u)
    # the ghost planes hold the periodic neighbours' planes
    loc = halo.extract(u, ncell, nq, d, parts[0]).reshape(d, -1, 3, nq)
    np.testing.assert_array_equal(loc[:, 0], u.reshape(d, 7, 3, nq)[:, 6])
    np.testing.assert_array_equal(loc[:, -1], u.reshape(d, 7, 3, nq)[:, parts[0][1]])


def _state(d, m, ncell, seed):
    st = I.random_state(d, m, ncell, seed=seed)
    return np.ascontiguousarray(st.p), np.ascontiguousarray(st.u)


def _plane_nodes(ncell):
    return int(np.prod(ncell[:-1])) if len(ncell) > 1 else 1


def _slab_step(d, m, ncell, dt, lp, lu, planes):
    """One oracle step of one slab (its ghosts already refreshed)."""
    return oracle.run(d, m, halo.local_ncell(ncell, planes), dt, lp, lu, 1, inv_h=halo.spacing(ncell))


@pytest.mark.parametrize("d,m,ncell", CASES)
@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_slabs_in_one_process_equal_the_undivided_grid(d, m, ncell, world):
    if ncell[-1] < world:
        pytest.skip("fewer planes than ranks")
    nq = (m + 1) ** d
    dt = I.cfl_dt(ncell)
    p, u = _state(d, m, ncell, seed=10 * d + m + world)
    steps = 5
    ref_p, ref_u = oracle.run(d, m, ncell, dt, p, u, steps)
    parts = halo.slab_planes(ncell[-1], world)
    lps = [np.ascontiguousarray(halo.extract(p.reshape(1, -1, nq), ncell, nq, 1, pl)[0]) for pl in parts]
    lus = [np.ascontiguousarray(halo.extract(u, ncell, nq, d, pl)) for pl in parts]
    pn = _plane_nodes(ncell)
    for _ in range(steps):
        halo.exchange_local([halo.plane_view(x, 1, x.shape[0] // pn, pn, nq, "host") for x in lps])
        halo.exchange_local([halo.plane_view(x, d, x.shape[1] // pn, pn, nq, "host") for x in lus])
        for r, pl in enumerate(parts):
            lps[r], lus[r] = _slab_step(d, m, ncell, dt, lps[r], lus[r], pl)
    got_p = np.concatenate([halo.owned(x[None], ncell, nq, 1, pl)[0] for x, pl in zip(lps, parts)], axis=0)
    got_u = np.concatenate([halo.owned(x, ncell, nq, d, pl) for x, pl in zip(lus, parts)], axis=1)
    np.testing.assert_array_equal(got_p, ref_p)
    np.testing.assert_array_equal(got_u, ref_u)


def test_skipping_the_exchange_breaks_the_result():
    """Guards against a vacuous pass: slabs whose ghosts go stale differ from the grid."""
    d, m, ncell = 2, 2, [7, 11]
    nq = (m + 1) ** d
    dt = I.cfl_dt(ncell)
    p, u = _state(d, m, ncell, seed=5)
    ref_p, _ = oracle.run(d, m, ncell, dt, p, u, 3)
    parts = halo.slab_planes(ncell[-1], 2)
    lps = [np.ascontiguousarray(halo.extract(p.reshape(1, -1, nq), ncell, nq, 1, pl)[0]) for pl in parts]
    lus = [np.ascontiguousarray(halo.extract(u, ncell, nq, d, pl)) for pl in parts]
    for _ in range(3):
        for r, pl in enumerate(parts):
            lps[r], lus[r] = _slab_step(d, m, ncell, dt, lps[r], lus[r], pl)
    got_p = np.concatenate([halo.owned(x[None], ncell, nq, 1, pl)[0] for x, pl in zip(lps, parts)], axis=0)
    assert np.abs(got_p - ref_p).max() > 1e-6 * np.abs(ref_p).max()


# ----------------------------------------------------------------------------- two gloo ranks
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, d, m, ncell, steps, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.set_threads(1)
        nq = (m + 1) ** d
        dt = I.cfl_dt(ncell)
        p, u = _state(d, m, ncell, seed=77)      # every rank draws the same global state
        pl = halo.slab_planes(ncell[-1], world)[rank]
        lp = np.ascontiguousarray(halo.extract(p.reshape(1, -1, nq), ncell, nq, 1, pl)[0])
        lu = np.ascontiguousarray(halo.extract(u, ncell, nq, d, pl))
        pn = _plane_nodes(ncell)
        for _ in range(steps):
            tp, tu = torch.from_numpy(lp), torch.from_numpy(lu)     # share memory with lp, lu
            halo.exchange(halo.plane_view(tp, 1, lp.shape[0] // pn, pn, nq, "host"), rank, world, dist)
            halo.exchange(halo.plane_view(tu, d, lu.shape[1] // pn, pn, nq, "host"), rank, world, dist)
            lp, lu = _slab_step(d, m, ncell, dt, lp, lu, pl)
        q.put((rank, halo.owned(lp[None], ncell, nq, 1, pl)[0], halo.owned(lu, ncell, nq, d, pl)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("d,m,ncell,world", [(2, 3, [6, 9], 2), (3, 1, [3, 4, 5], 2), (2, 2, [5, 7], 3)])
def test_gloo_ranks_equal_the_undivided_grid(d, m, ncell, world):
    """Two ranks are each other's upper and lower neighbour (the tags keep the messages
    apart); three ranks have distinct neighbours."""
    steps = 4
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, d, m, ncell, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted((q.get(timeout=180) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    p0, u0 = _state(d, m, ncell, seed=77)
    ref_p, ref_u = oracle.run(d, m, ncell, I.cfl_dt(ncell), p0, u0, steps)
    np.testing.assert_array_equal(np.concatenate([r[1] for r in results], axis=0), ref_p)
    np.testing.assert_array_equal(np.concatenate([r[2] for r in results], axis=1), ref_u)


def test_extract_and_owned_work_on_torch_tensors():
    torch = pytest.importorskip("torch")
    d, m, ncell = 3, 1, [3, 2, 5]
    nq = (m + 1) ** d
    u = np.random.default_rng(9).standard_normal((d, 30, nq))
    for pl in halo.slab_planes(ncell[-1], 2):
        want = halo.extract(u, ncell, nq, d, pl)
        got = halo.extract(torch.from_numpy(u), ncell, nq, d, pl)
        np.testing.assert_array_equal(got.numpy(), want)
        np.testing.assert_array_equal(halo.owned(got, ncell, nq, d, pl).numpy(), halo.owned(want, ncell, nq, d, pl))
