"""Host logic of the learned correction's data-parallel training
(paper_1808_10481_gb300/learned.py) on CPU with two gloo ranks.

The GPU step (hl_mlp_loss_grad) is replaced by the oracle's network gradient on each rank's
own rows; everything else is the product's code: the shard of the training rows, the in-place
all-reduce mean of the gradient, then one Adam step per rank.  The averaged gradient must be
the gradient of the mean loss over both ranks' rows (one process over all rows), and both
replicas must hold identical weights after the step."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

from oracle import mlp as omlp
from paper_1808_10481_gb300 import learned

KEYS = ("W1", "b1", "W2", "b2", "W3", "b3")


def flat(P):
    return np.concatenate([P[k].ravel() for k in KEYS])


def unflat(v, like):
    out, o = {}, 0
    for k in KEYS:
        n = like[k].size
        out[k] = v[o:o + n].reshape(like[k].shape)
        o += n
    return out


def data(rows=64, seed=3):
    rng = np.random.default_rng(seed)
    P = omlp.init_params(rng)
    X = rng.standard_normal((rows, omlp.N_IN))
    T = rng.standard_normal((rows, omlp.N_OUT)) * 0.1
    return P, X, T


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P, X, T = data()
        lo, hi = learned.shard_range(X.shape[0], world, rank)
        _, grads = omlp.loss_and_grads(P, X[lo:hi], T[lo:hi])
        g = torch.from_numpy(flat(grads).astype(np.float64))
        learned.allreduce_mean_(g, tdist)
        Pn = {k: v.copy() for k, v in P.items()}
        omlp.adam_step(Pn, unflat(g.numpy(), P), {k: np.zeros_like(v) for k, v in P.items()},
                       {k: np.zeros_like(v) for k, v in P.items()}, 1, 1e-3)
        q.put((rank, g.numpy().copy(), flat(Pn)))
    except Exception as e:  # report instead of leaving the parent waiting
        q.put((rank, None, repr(e)))
    finally:
        tdist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_range_partitions_the_rows():
    for n in (0, 1, 7, 64, 1000):
        for world in (1, 2, 3, 8):
            parts = [learned.shard_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        learned.shard_range(4, 2, 2)


def test_allreduce_is_a_no_op_on_one_rank():
    t = torch.arange(5, dtype=torch.float64)
    learned.allreduce_mean_(t, None)
    assert torch.equal(t, torch.arange(5, dtype=torch.float64))


def test_two_ranks_average_to_the_full_batch_gradient_and_stay_identical():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (g, w)) for r, g, w in (q.get(timeout=120) for _ in range(world)))
    for r in range(world):
        assert res[r][0] is not None, res[r][1]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    P, X, T = data()
    _, full = omlp.loss_and_grads(P, X, T)
    g_full = flat(full)
    for r in range(world):
        g, _ = res[r]
        assert np.allclose(g, g_full, rtol=1e-12, atol=1e-15 * np.abs(g_full).max())
    assert np.array_equal(res[0][1], res[1][1])      # identical replicas after the Adam step
    # a rank that skipped the reduction would hold its half's gradient instead
    _, half = omlp.loss_and_grads(P, X[:32], T[:32])
    assert not np.allclose(flat(half), g_full, rtol=1e-6)
