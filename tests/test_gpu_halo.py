"""Slabs of one grid on the GPU: hl_create_spacing, and slabs with ghost planes stepped by
the CUDA kernels with their ghosts refreshed between steps (the ranks of a slab
decomposition emulated in one process: separate launches in stream order, nothing waits
on another launch).  The owned planes must match the CPU oracle's undivided grid at the
FP64 parity bar, 1e-12 of the field's maximum."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1808_10481_gb300 import halo, hl
from paper_1808_10481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1808_10481_gb300 import build
    build.build()
    hl.load()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _run(h, p, u, steps):
    hl.hl_set_initial(h, p, u)
    hl.hl_step(h, steps)
    out_p, out_u, _, _ = hl.hl_get_fields(h)
    return out_p, out_u


def test_spacing_of_the_unit_box_equals_create():
    d, m, ncell = 2, 3, [37, 29]
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=21)
    a = hl.hl_create(d, m, ncell, dt)
    b = hl.hl_create_spacing(d, m, ncell, [float(n) for n in ncell], dt)
    try:
        pa, ua = _run(a, st.p, st.u, 6)
        pb, ub = _run(b, st.p, st.u, 6)
    finally:
        hl.hl_destroy(a)
        hl.hl_destroy(b)
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(ua, ub)


@pytest.mark.parametrize("d,m,ncell,world", [
    (1, 3, [50], 2),
    (2, 3, [37, 29], 2),
    (2, 3, [37, 29], 3),
    (2, 2, [16, 5], 4),
    (3, 2, [9, 7, 11], 2),
])
def test_slabs_on_one_gpu_match_the_oracle(d, m, ncell, world):
    import torch
    dt = I.cfl_dt(ncell)
    steps = 8
    st = I.random_state(d, m, ncell, seed=31 + world)
    slabs = [halo.SlabSolver(d, m, ncell, dt, pl) for pl in halo.slab_planes(ncell[-1], world)]
    try:
        for s in slabs:
            s.set_initial(st.p, st.u)
        halo.step_slabs(slabs, steps)
        torch.cuda.synchronize()
        parts = [s.owned_fields() for s in slabs]
    finally:
        for s in slabs:
            s.close()
    got_p = np.concatenate([x[0] for x in parts], axis=0)
    got_u = np.concatenate([x[1] for x in parts], axis=1)
    ref_p, ref_u = oracle.run(d, m, ncell, dt, st.p, st.u, steps)
    assert _rel(got_p, ref_p) <= TOL
    assert _rel(got_u, ref_u) <= TOL


def test_point_source_needs_the_unit_box():
    h = hl.hl_create_spacing(2, 3, [16, 6], [16.0, 16.0], I.cfl_dt([16, 16]))
    try:
        with pytest.raises(hl.HLError) as ei:
            hl.hl_set_source(h, [0.5, 0.5], 0.01, 15.0, 1.0)
        assert ei.value.code == hl.HL_EINVAL
    finally:
        hl.hl_destroy(h)
