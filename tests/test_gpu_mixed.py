"""Mixed-precision modes (FP32 contraction, FP64 node data and accumulation).

Their error against the FP64 oracle is stated, not held to the FP64 bar: per half-step
each mode rounds the gathered data and the operator to binary32 (HL_FP32, relative
2^-24 ~ 6e-8 per input) or keeps a hi/lo split of both (HL_FP32_COMP, inputs exact to
~2^-48 with FP32 accumulation of the main and correction sums).  The bounds below are
those per-step figures times the operator's amplification and the step count, with
margin; the measured errors are printed for the record."""
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


# (bound for HL_FP32, bound for HL_FP32_COMP) on the relative error after the run
CASES = [
    (1, 3, [64], "standing", 200, 5e-6, 5e-7),
    (2, 3, [48, 40], "gaussian", 40, 5e-6, 5e-7),
    (3, 2, [16, 14, 12], "plane", 20, 5e-6, 5e-7),
]


@pytest.mark.parametrize("d,m,ncell,kind,steps,b32,bcomp", CASES)
def test_mixed_modes_error_against_oracle(d, m, ncell, kind, steps, b32, bcomp):
    dt = I.cfl_dt(ncell)
    if kind == "standing":
        st = I.standing_mode(d, m, ncell, dt, wave=[3])
    elif kind == "gaussian":
        st = I.gaussian_pulse(d, m, ncell, dt, seed=2, width=0.1)
    else:
        st = I.plane_wave(m, ncell, dt, seed=3, kmax=2.0)
    po, uo = oracle.run(d, m, ncell, dt, st.p, st.u, steps)
    errs = {}
    for mode, bound in ((hl.HL_FP32, b32), (hl.HL_FP32_COMP, bcomp)):
        pg, ug = gpu_run(d, m, ncell, dt, st, steps, mode)
        errs[mode] = max(rel_err(pg, po), rel_err(ug, uo))
        assert errs[mode] <= bound, (mode, errs[mode], bound)
    print(f"mixed-precision error d={d} m={m}: FP32 {errs[hl.HL_FP32]:.2e}, FP32_COMP {errs[hl.HL_FP32_COMP]:.2e}")
    assert errs[hl.HL_FP32_COMP] < errs[hl.HL_FP32]


def test_mixed_keeps_the_discretisation_error():
    """At equal grid the FP32 modes' L2 error against the exact solution equals the FP64
    solver's to within 1% (the discretisation error dominates the rounding)."""
    d, m, ncell = 3, 2, [32, 32, 32]
    dt = I.cfl_dt(ncell)
    st = I.plane_wave(m, ncell, dt, seed=3, kmax=3.0)
    steps = 30
    t_p = steps * dt
    ex = I.plane_wave(m, ncell, dt, seed=3, kmax=3.0, t0=t_p)
    e = {}
    for mode in (hl.HL_FP64, hl.HL_FP32, hl.HL_FP32_COMP):
        pg, _ = gpu_run(d, m, ncell, dt, st, steps, mode)
        e[mode] = I.l2_error(d, ncell, pg, ex.p)
    print("L2 error vs exact:", e)
    assert abs(e[hl.HL_FP32] - e[hl.HL_FP64]) <= 0.01 * e[hl.HL_FP64]
    assert abs(e[hl.HL_FP32_COMP] - e[hl.HL_FP64]) <= 0.01 * e[hl.HL_FP64]


def test_mixed_batch_equals_each_shot_alone():
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
        np.testing.assert_array_equal(pb[po:po + s.p.size], ps.ravel())
        np.testing.assert_array_equal(ub[uo:uo + s.u.size], us.ravel())
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
