"""Mixed-precision modes: the contraction on the FP32 pipe (HL_FP32, HL_FP32_COMP) or
as exact FP16 tensor-core digit products (HL_TC_SPLIT, 2D and 3D), the node data and their
updates in binary64.

Their error against the FP64 oracle is stated and bounded by the arithmetic, not held to
the FP64 bar.  One half-step rounds inputs and sums to the mode's unit roundoff eps
(2^-24 for HL_FP32, about 2^-47 for the float-float HL_FP32_COMP), amplified by the
operator's absolute row sum (cancellation in the high-order stencil).  The bound after n
steps is 4 * eps * rowsum * n (tc_bound for the digit split, whose quantisation is
relative to block and column maxima); the measured errors are printed for the record."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1808_10481_gb300 import hl
from paper_1808_10481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EPS = {1: 2.0 ** -24, 2: 2.0 ** -47}
_ROW = {}
_COLS = {}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1808_10481_gb300 import build
    build.build()
    hl.load()


def rel_err(got, ref):
    scale = float(np.abs(ref).max())
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max()) / (scale if scale > 0 else 1.0)


def _vertex_operator(d, m):
    """The p-half's vertex-form operator from the oracle: row k = (component, vertex, slot)."""
    if (d, m) not in _COLS:
        nq = (m + 1) ** d
        cols = []
        for c in range(d):
            for v in range(1 << d):
                for l in range(nq):
                    vtx = np.zeros((d, 1 << d, nq))
                    vtx[c, v, l] = 1.0
                    cols.append(oracle.node_update(d, m, [0.45] * d, 0, vtx)[0])
        _COLS[(d, m)] = np.abs(np.array(cols))
    return _COLS[(d, m)]


def rowsum(d, m):
    if (d, m) not in _ROW:
        _ROW[(d, m)] = float(_vertex_operator(d, m).sum(axis=0).max())
    return _ROW[(d, m)]


def tc_bound(d, m, steps):
    """HL_TC_SPLIT quantises data and operator columns to 46 bits below their block and
    column maxima (relative error 2^-47 of the maximum each) and drops digit levels of
    weight <= 2^-45: per half-step and output at most 2^-46 max|data| (rowsum + K colmax)
    + 2^-44 max|data| colmax, K the number of terms.  Four times that per step."""
    W = _vertex_operator(d, m)
    K = W.shape[0]
    per = 2.0 ** -46 * (rowsum(d, m) + K * W.max(axis=0).max()) + 2.0 ** -44 * W.max()
    return 4 * per * steps


def gpu_run(d, m, ncell, dt, st, steps, mode):
    h = hl.hl_create(d, m, ncell, dt)
    try:
        hl.hl_set_precision(h, mode)
        hl.hl_set_initial(h, st.p, st.u)
        hl.hl_step(h, steps)
        pg, ug, _, _ = hl.hl_get_fields(h)
        return pg, ug
    finally:
        hl.hl_destroy(h)


CASES = [
    (1, 3, [64], "standing", 200),
    (2, 3, [48, 40], "gaussian", 40),
    (3, 2, [16, 14, 12], "plane", 20),
]


@pytest.mark.parametrize("d,m,ncell,kind,steps", CASES)
def test_mixed_modes_error_against_oracle(d, m, ncell, kind, steps):
    dt = I.cfl_dt(ncell)
    if kind == "standing":
        st = I.standing_mode(d, m, ncell, dt, wave=[3])
    elif kind == "gaussian":
        st = I.gaussian_pulse(d, m, ncell, dt, seed=2, width=0.1)
    else:
        st = I.plane_wave(m, ncell, dt, seed=3, kmax=2.0)
    po, uo = oracle.run(d, m, ncell, dt, st.p, st.u, steps, prec="dd")
    errs = {}
    for mode in (hl.HL_FP32, hl.HL_FP32_COMP):
        pg, ug = gpu_run(d, m, ncell, dt, st, steps, mode)
        errs[mode] = max(rel_err(pg, po), rel_err(ug, uo))
        bound = 4 * EPS[mode] * rowsum(d, m) * steps
        assert errs[mode] <= bound, (mode, errs[mode], bound)
    print(f"mixed-precision error d={d} m={m} steps={steps}: FP32 {errs[hl.HL_FP32]:.2e}, "
          f"FP32_COMP {errs[hl.HL_FP32_COMP]:.2e}")
    assert errs[hl.HL_FP32_COMP] * 1e3 < errs[hl.HL_FP32]


def test_compensated_mode_keeps_the_discretisation_error():
    """At equal grid the compensated mode's L2 error against the exact solution equals
    the FP64 solver's to 1%; the plain FP32 mode's is reported beside it."""
    d, m, ncell = 3, 2, [32, 32, 32]
    dt = I.cfl_dt(ncell)
    st = I.plane_wave(m, ncell, dt, seed=3, kmax=3.0)
    steps = 30
    ex = I.plane_wave(m, ncell, dt, seed=3, kmax=3.0, t0=steps * dt)
    e = {}
    for mode in (hl.HL_FP64, hl.HL_FP32, hl.HL_FP32_COMP):
        pg, _ = gpu_run(d, m, ncell, dt, st, steps, mode)
        e[mode] = I.l2_error(d, ncell, pg, ex.p)
    print("L2 error vs exact (FP64, FP32, FP32_COMP):", e[hl.HL_FP64], e[hl.HL_FP32], e[hl.HL_FP32_COMP])
    assert abs(e[hl.HL_FP32_COMP] - e[hl.HL_FP64]) <= 0.01 * e[hl.HL_FP64]


def test_mixed_with_point_source_matches_oracle():
    """The source updates the binary64 data and the shadows together."""
    d, m, ncell = 2, 3, [40, 36]
    dt = I.cfl_dt(ncell)
    nnode, nq = 40 * 36, 16
    p, u = np.zeros((nnode, nq)), np.zeros((2, nnode, nq))
    src = dict(x0=[0.3, 0.6], sigma=0.05, f0=12.0, amp=1.0)
    steps = 30
    po, uo = oracle.run_source(d, m, ncell, dt, p, u, steps, **src, prec="dd")
    h = hl.hl_create(d, m, ncell, dt)
    try:
        hl.hl_set_precision(h, hl.HL_FP32_COMP)
        hl.hl_set_initial(h, p, u)
        hl.hl_set_source(h, src["x0"], src["sigma"], src["f0"], src["amp"])
        hl.hl_step(h, steps)
        pg, ug, _, _ = hl.hl_get_fields(h)
    finally:
        hl.hl_destroy(h)
    bound = 4 * EPS[2] * rowsum(d, m) * steps
    assert max(rel_err(pg, po), rel_err(ug, uo)) <= bound


def test_mixed_batch_matches_each_shot_alone():
    """A batch shares one FP32 operator table (shot 0's; every shot has dt/h = 0.9, so
    the tables agree to the last bits of lam): batch and single runs agree to the mode's
    rounding level."""
    d, m = 2, 3
    sizes = [20, 33, 47]
    cells = [[n, n] for n in sizes]
    dts = [I.cfl_dt(c) for c in cells]
    sts = [I.random_state(d, m, c, seed=40 + i) for i, c in enumerate(cells)]
    h = hl.hl_create_batch(d, m, cells, dts)
    try:
        hl.hl_set_precision(h, hl.HL_FP32_COMP)
        p = np.concatenate([s.p.ravel() for s in sts])
        u = np.concatenate([s.u.ravel() for s in sts])
        hl.hl_set_initial(h, p, u)
        hl.hl_step(h, 9)
        pb, ub = np.empty(p.size), np.empty(u.size)
        hl.hl_get_fields(h, pb, ub)
    finally:
        hl.hl_destroy(h)
    po = uo = 0
    for c, dt, s in zip(cells, dts, sts):
        ps, us = gpu_run(d, m, c, dt, s, 9, hl.HL_FP32_COMP)
        assert rel_err(pb[po:po + s.p.size], ps.ravel()) <= 4 * EPS[2] * rowsum(d, m) * 9
        assert rel_err(ub[uo:uo + s.u.size], us.ravel()) <= 4 * EPS[2] * rowsum(d, m) * 9
        po += s.p.size
        uo += s.u.size


def test_precision_mode_validation():
    h = hl.hl_create(3, 3, [4, 4, 4], 0.1)
    try:
        with pytest.raises(hl.HLError):
            hl.hl_set_precision(h, hl.HL_FP32)
        with pytest.raises(hl.HLError):
            hl.hl_set_precision(h, 7)
    finally:
        hl.hl_destroy(h)


@pytest.mark.parametrize("m,ncell,kind,steps", [(3, [48, 40], "gaussian", 40), (3, [17, 13], "random", 6),
                                                (2, [19, 16], "random", 6), (1, [23, 9], "random", 6),
                                                (0, [16, 16], "random", 6)])
def test_tc_split_error_against_oracle(m, ncell, kind, steps):
    d = 2
    dt = I.cfl_dt(ncell)
    st = I.gaussian_pulse(d, m, ncell, dt, seed=2, width=0.1) if kind == "gaussian" else \
        I.random_state(d, m, ncell, seed=60 + m)
    po, uo = oracle.run(d, m, ncell, dt, st.p, st.u, steps, prec="dd")
    pg, ug = gpu_run(d, m, ncell, dt, st, steps, hl.HL_TC_SPLIT)
    err = max(rel_err(pg, po), rel_err(ug, uo))
    pf, uf = gpu_run(d, m, ncell, dt, st, steps, hl.HL_FP32)
    err32 = max(rel_err(pf, po), rel_err(uf, uo))
    print(f"tensor-core split error d=2 m={m} n={ncell} steps={steps}: {err:.2e} (FP32 {err32:.2e}, "
          f"bound {tc_bound(d, m, steps):.2e})")
    assert err <= tc_bound(d, m, steps)
    assert err * 1e3 < err32


def test_tc_split_keeps_the_discretisation_error():
    """2D standing mode, m = 3: the tensor-core split mode's L2 error against the exact
    solution equals the FP64 solver's to 1%."""
    d, m, ncell = 2, 3, [32, 32]
    dt = I.cfl_dt(ncell)
    st = I.standing_mode(d, m, ncell, dt, wave=[2, 3])
    steps = 60
    ex = I.standing_mode_exact(d, m, ncell, [2, 3], steps * dt, (steps + 0.5) * dt)
    e = {}
    for mode in (hl.HL_FP64, hl.HL_TC_SPLIT):
        pg, _ = gpu_run(d, m, ncell, dt, st, steps, mode)
        e[mode] = I.l2_error(d, ncell, pg, ex.p)
    print("2D L2 error vs exact (FP64, TC_SPLIT):", e[hl.HL_FP64], e[hl.HL_TC_SPLIT])
    assert abs(e[hl.HL_TC_SPLIT] - e[hl.HL_FP64]) <= 0.01 * e[hl.HL_FP64]


def test_tc_split_every_tile_shape_and_source():
    """Every tile shape (the block scale differs per tile), with a point source."""
    d, m, ncell = 2, 3, [45, 37]
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=71)
    src = dict(x0=[0.3, 0.6], sigma=0.05, f0=12.0, amp=1.0)
    steps = 5
    po, uo = oracle.run_source(d, m, ncell, dt, st.p, st.u, steps, **src, prec="dd")
    for t in range(hl.HL_NUM_TILES):
        h = hl.hl_create(d, m, ncell, dt)
        try:
            hl.hl_set_option(h, hl.HL_OPT_TILE, t)
            hl.hl_set_precision(h, hl.HL_TC_SPLIT)
            hl.hl_set_initial(h, st.p, st.u)
            hl.hl_set_source(h, src["x0"], src["sigma"], src["f0"], src["amp"])
            hl.hl_step(h, steps)
            pg, ug, _, _ = hl.hl_get_fields(h)
        finally:
            hl.hl_destroy(h)
        assert max(rel_err(pg, po), rel_err(ug, uo)) <= tc_bound(d, m, steps), hl.TILES[t]


def test_tc_split_batch_matches_each_shot_alone():
    d, m = 2, 3
    sizes = [20, 33, 47]
    cells = [[n, n] for n in sizes]
    dts = [I.cfl_dt(c) for c in cells]
    sts = [I.random_state(d, m, c, seed=80 + i) for i, c in enumerate(cells)]
    h = hl.hl_create_batch(d, m, cells, dts)
    try:
        hl.hl_set_precision(h, hl.HL_TC_SPLIT)
        p = np.concatenate([s.p.ravel() for s in sts])
        u = np.concatenate([s.u.ravel() for s in sts])
        hl.hl_set_initial(h, p, u)
        hl.hl_step(h, 7)
        pb, ub = np.empty(p.size), np.empty(u.size)
        hl.hl_get_fields(h, pb, ub)
    finally:
        hl.hl_destroy(h)
    po = uo = 0
    for c, dt, s in zip(cells, dts, sts):
        pr, ur = oracle.run(d, m, c, dt, s.p, s.u, 7)
        assert rel_err(pb[po:po + s.p.size], pr.ravel()) <= tc_bound(d, m, 7)
        assert rel_err(ub[uo:uo + s.u.size], ur.ravel()) <= tc_bound(d, m, 7)
        po += s.p.size
        uo += s.u.size


def test_tc_split_validation():
    for d, m, nc in ((3, 1, [4, 4, 4]), (1, 3, [16]), (2, 4, [8, 8])):
        h = hl.hl_create(d, m, nc, 0.9 / max(nc))
        try:
            with pytest.raises(hl.HLError):
                hl.hl_set_precision(h, hl.HL_TC_SPLIT)
        finally:
            hl.hl_destroy(h)
    # 3D runs one shot
    h = hl.hl_create_batch(3, 2, [[4, 4, 4], [5, 4, 4]], [0.05, 0.05])
    try:
        with pytest.raises(hl.HLError):
            hl.hl_set_precision(h, hl.HL_TC_SPLIT)
    finally:
        hl.hl_destroy(h)


# 3D (m = 2): the partner field cut once per half-step at the field's exponent, groups
# of 4 vertices x 27 slots accumulated exactly on the tensor cores and drained into
# float-float sums.  Grids: one tile ragged in x, several tiles with a ragged last one
# (130 = 128 + 2), an exact tile multiple, and a cube with odd sizes per axis.
@pytest.mark.parametrize("ncell,kind,steps", [([9, 7, 5], "random", 4), ([130, 3, 2], "random", 3),
                                              ([128, 4, 3], "random", 3), ([16, 14, 12], "plane", 20),
                                              ([2, 2, 2], "random", 5)])
def test_tc_split_3d_error_against_oracle(ncell, kind, steps):
    d, m = 3, 2
    dt = I.cfl_dt(ncell)
    st = I.plane_wave(m, ncell, dt, seed=3, kmax=2.0) if kind == "plane" else I.random_state(d, m, ncell, seed=140)
    po, uo = oracle.run(d, m, ncell, dt, st.p, st.u, steps, prec="dd")
    pg, ug = gpu_run(d, m, ncell, dt, st, steps, hl.HL_TC_SPLIT)
    err = max(rel_err(pg, po), rel_err(ug, uo))
    pf, uf = gpu_run(d, m, ncell, dt, st, steps, hl.HL_FP32)
    err32 = max(rel_err(pf, po), rel_err(uf, uo))
    print(f"tensor-core split error d=3 m=2 n={ncell} steps={steps}: {err:.2e} (FP32 {err32:.2e}, "
          f"bound {tc_bound(d, m, steps):.2e})")
    assert err <= tc_bound(d, m, steps)
    assert err * 1e3 < err32


def test_tc_split_3d_keeps_the_discretisation_error():
    """3D plane wave, m = 2: the L2 error against the exact solution equals FP64's to 1%."""
    d, m, ncell = 3, 2, [20, 20, 20]
    dt = I.cfl_dt(ncell)
    st = I.plane_wave(m, ncell, dt, seed=5, kmax=3.0)
    steps = 40
    ex = I.plane_wave(m, ncell, dt, seed=5, kmax=3.0, t0=steps * dt)
    e = {}
    for mode in (hl.HL_FP64, hl.HL_TC_SPLIT):
        pg, _ = gpu_run(d, m, ncell, dt, st, steps, mode)
        e[mode] = I.l2_error(d, ncell, pg, ex.p)
    print("3D L2 error vs exact (FP64, TC_SPLIT):", e[hl.HL_FP64], e[hl.HL_TC_SPLIT])
    assert abs(e[hl.HL_TC_SPLIT] - e[hl.HL_FP64]) <= 0.01 * e[hl.HL_FP64]


def test_tc_split_3d_with_source_and_graph():
    """A point source inside the tensor-core steps, launched plainly and from a graph."""
    d, m, ncell = 3, 2, [12, 11, 10]
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=141)
    src = dict(x0=[0.3, 0.6, 0.5], sigma=0.08, f0=6.0, amp=1.0)
    steps = 4
    po, uo = oracle.run_source(d, m, ncell, dt, st.p, st.u, steps, **src, prec="dd")
    for graph in (0, 1):
        h = hl.hl_create(d, m, ncell, dt)
        try:
            hl.hl_set_option(h, hl.HL_OPT_GRAPH, graph)
            hl.hl_set_precision(h, hl.HL_TC_SPLIT)
            hl.hl_set_initial(h, st.p, st.u)
            hl.hl_set_source(h, src["x0"], src["sigma"], src["f0"], src["amp"])
            hl.hl_step(h, steps)
            pg, ug, _, _ = hl.hl_get_fields(h)
        finally:
            hl.hl_destroy(h)
        assert max(rel_err(pg, po), rel_err(ug, uo)) <= tc_bound(d, m, steps), graph


@pytest.mark.parametrize("mode", ["fp32_comp", "tc_split"])
def test_autotune_in_mixed_modes_leaves_state_untouched(mode):
    """The autotuner times every tile shape in the handle's precision mode on scratch copies:
    the state and the step counter are unchanged, and stepping afterwards still matches the
    oracle within the mode's bound."""
    prec = {"fp32_comp": hl.HL_FP32_COMP, "tc_split": hl.HL_TC_SPLIT}[mode]
    d, m, ncell = 2, 3, [40, 36]
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=91)
    h = hl.hl_create(d, m, ncell, dt)
    try:
        hl.hl_set_precision(h, prec)
        hl.hl_set_initial(h, st.p, st.u)
        best, ms = hl.hl_autotune(h, 1)
        assert 0 <= best < hl.HL_NUM_TILES and ms[best] > 0
        p0, u0, _, _ = hl.hl_get_fields(h)
        np.testing.assert_array_equal(p0, st.p.reshape(p0.shape))
        np.testing.assert_array_equal(u0, st.u.reshape(u0.shape))
        assert hl.hl_info(h)[2] == 0
        hl.hl_step(h, 4)
        pg, ug, _, _ = hl.hl_get_fields(h)
    finally:
        hl.hl_destroy(h)
    po, uo = oracle.run(d, m, ncell, dt, st.p, st.u, 4)
    bound = tc_bound(d, m, 4) if mode == "tc_split" else 4 * EPS[2] * rowsum(d, m) * 4
    assert max(rel_err(pg, po), rel_err(ug, uo)) <= bound
