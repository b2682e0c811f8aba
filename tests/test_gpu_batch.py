"""Batched multi-shot solves (one launch per half-step over all shots, captured as a
CUDA graph) and tile-shape autotuning, through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1808_10481_gb300 import hl
from paper_1808_10481_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1808_10481_gb300 import build
    build.build()
    hl.load()


def rel_err(got, ref):
    scale = float(np.abs(ref).max())
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max()) / (scale if scale > 0 else 1.0)


def _shots(d, sizes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        ncell = [n] * d if np.isscalar(n) else list(n)
        dt = I.cfl_dt(ncell)
        st = I.random_state(d, 3 if d < 3 else 2, ncell, seed=seed + i)
        src = dict(x0=list(rng.random(d)), sigma=0.05, f0=float(rng.uniform(10, 20)), amp=1.0)
        out.append((ncell, dt, st, src))
    return out


def _run_single(d, m, ncell, dt, p, u, steps, src=None, tile=None):
    h = hl.hl_create(d, m, ncell, dt)
    try:
        if tile is not None:
            hl.hl_set_option(h, hl.HL_OPT_TILE, tile)
            hl.hl_set_option(h, hl.HL_OPT_KERNEL_PATH, 2)
        hl.hl_set_initial(h, p, u)
        if src:
            hl.hl_set_source(h, src["x0"], src["sigma"], src["f0"], src["amp"])
        hl.hl_step(h, steps)
        pg, ug, _, _ = hl.hl_get_fields(h)
        return pg, ug
    finally:
        hl.hl_destroy(h)


def _run_batch(d, m, shots, steps, with_src, graph=1, chunks=1):
    h = hl.hl_create_batch(d, m, [s[0] for s in shots], [s[1] for s in shots])
    try:
        hl.hl_set_option(h, hl.HL_OPT_GRAPH, graph)
        p = np.concatenate([s[2].p.ravel() for s in shots])
        u = np.concatenate([s[2].u.ravel() for s in shots])
        hl.hl_set_initial(h, p, u)
        if with_src:
            hl.hl_set_sources(h, [s[3]["x0"] for s in shots], [s[3]["sigma"] for s in shots],
                              [s[3]["f0"] for s in shots], [s[3]["amp"] for s in shots])
        for _ in range(chunks):
            hl.hl_step(h, steps // chunks)
        pb = np.empty(p.size)
        ub = np.empty(u.size)
        hl.hl_get_fields(h, pb, ub)
    finally:
        hl.hl_destroy(h)
    outs, po, uo = [], 0, 0
    for ncell, _, st, _ in shots:
        outs.append((pb[po:po + st.p.size].reshape(st.p.shape), ub[uo:uo + st.u.size].reshape(st.u.shape)))
        po += st.p.size
        uo += st.u.size
    return outs


@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("with_src", [False, True])
def test_batch_equals_each_shot_alone_bitwise(graph, with_src):
    d, m = 2, 3
    shots = _shots(d, [17, (40, 23), 64, 9, 31], seed=3)
    steps = 12
    outs = _run_batch(d, m, shots, steps, with_src, graph=graph, chunks=2)
    for (ncell, dt, st, src), (pb, ub) in zip(shots, outs):
        ps, us = _run_single(d, m, ncell, dt, st.p, st.u, steps, src if with_src else None)
        np.testing.assert_array_equal(pb, ps)
        np.testing.assert_array_equal(ub, us)


@pytest.mark.parametrize("d", [1, 3])
def test_batch_other_dimensions_match_oracle(d):
    m = 3 if d == 1 else 2
    sizes = [33, 7, 100] if d == 1 else [(6, 5, 4), (9, 8, 7)]
    shots = _shots(d, sizes, seed=9)
    steps = 8
    outs = _run_batch(d, m, shots, steps, True)
    for (ncell, dt, st, src), (pb, ub) in zip(shots, outs):
        po, uo = oracle.run_source(d, m, ncell, dt, st.p, st.u, steps, **src)
        assert rel_err(pb, po) <= 1e-12 and rel_err(ub, uo) <= 1e-12


def test_ricker_batch_from_rest_matches_oracle():
    """The batched workload's set-up in miniature: zero fields, one Ricker source per
    shot (f0 in [10, 20], seeded position), uneven grid sizes."""
    d, m = 2, 3
    rng = np.random.default_rng(77)
    sizes = [int(x) for x in rng.integers(24, 72, size=6)]
    shots = []
    for n in sizes:
        ncell = [n, n]
        nnode, nq = n * n, (m + 1) ** d
        st = I.InitialData(np.zeros((nnode, nq)), np.zeros((d, nnode, nq)), {})
        src = dict(x0=list(rng.random(2)), sigma=0.01, f0=float(rng.uniform(10, 20)), amp=1.0)
        shots.append((ncell, I.cfl_dt(ncell), st, src))
    steps = 40
    outs = _run_batch(d, m, shots, steps, True)
    for (ncell, dt, st, src), (pb, ub) in zip(shots, outs):
        # 40 steps: compared with the oracle's double-double build (see test_gpu_parity)
        po, uo = oracle.run_source(d, m, ncell, dt, st.p, st.u, steps, **src, prec="dd")
        assert np.abs(po).max() > 0
        assert rel_err(pb, po) <= 1e-12 and rel_err(ub, uo) <= 1e-12


@pytest.mark.parametrize("d,m,ncell", [(2, 3, [45, 37]), (2, 4, [21, 19]), (3, 2, [13, 11, 7]), (3, 1, [9, 7, 5])])
def test_tile_shape_does_not_change_results(d, m, ncell):
    """Every tile shape, paired (two nodes per thread along y, odd row counts leave
    a lone last row) or not, gives bitwise the same result."""
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=12)
    ref = _run_single(d, m, ncell, dt, st.p, st.u, 6, tile=0)
    for t in range(1, hl.HL_NUM_TILES):
        got = _run_single(d, m, ncell, dt, st.p, st.u, 6, tile=t)
        np.testing.assert_array_equal(got[0], ref[0], err_msg=f"tile {hl.TILES[t]}")
        np.testing.assert_array_equal(got[1], ref[1], err_msg=f"tile {hl.TILES[t]}")


def test_autotune_picks_a_tile_and_leaves_state_untouched():
    d, m = 2, 3
    shots = _shots(d, [128, 96, 200], seed=5)
    h = hl.hl_create_batch(d, m, [s[0] for s in shots], [s[1] for s in shots])
    try:
        p = np.concatenate([s[2].p.ravel() for s in shots])
        u = np.concatenate([s[2].u.ravel() for s in shots])
        hl.hl_set_initial(h, p, u)
        best, ms = hl.hl_autotune(h, 2)
        assert 0 <= best < hl.HL_NUM_TILES
        assert ms[best] > 0 and all(x < 0 or x >= ms[best] for x in ms)
        pb = np.empty(p.size)
        ub = np.empty(u.size)
        _, _, _, _ = hl.hl_get_fields(h, pb, ub)
        np.testing.assert_array_equal(pb, p)
        np.testing.assert_array_equal(ub, u)
        assert hl.hl_info(h)[2] == 0
    finally:
        hl.hl_destroy(h)
