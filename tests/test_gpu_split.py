"""The split two-kernel form of the FP64 half-step (HL_OPT_SPLIT; Section 6's interpolation
and evolution kernels) through the C ABI: against the oracle on random data in 1D, 2D and 3D
for every supported order, on ragged grids smaller and larger than one block of nodes, and
against the fused kernels over a longer run."""
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
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def run(d, m, ncell, dt, st, steps, split):
    h = hl.hl_create(d, m, ncell, dt)
    try:
        hl.hl_set_option(h, hl.HL_OPT_KERNEL_PATH, 2)
        hl.hl_set_option(h, hl.HL_OPT_SPLIT, split)
        hl.hl_set_initial(h, st.p, st.u)
        hl.hl_step(h, steps)
        pg, ug, _, _ = hl.hl_get_fields(h)
        return pg, ug
    finally:
        hl.hl_destroy(h)


@pytest.mark.parametrize("d,m,ncell,steps", [
    (1, 0, [5], 6), (1, 3, [300], 5), (2, 0, [7, 5], 4), (2, 1, [19, 13], 4), (2, 2, [40, 9], 3),
    (2, 3, [70, 11], 3), (3, 0, [6, 5, 4], 3), (3, 1, [40, 7, 5], 2), (3, 2, [20, 9, 7], 2), (3, 3, [11, 6, 5], 2),
])
def test_split_matches_oracle(d, m, ncell, steps):
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=700 + 10 * d + m)
    pg, ug = run(d, m, ncell, dt, st, steps, 1)
    po, uo = oracle.run(d, m, ncell, dt, st.p, st.u, steps)
    assert rel_err(pg, po) <= 1e-12 and rel_err(ug, uo) <= 1e-12, (rel_err(pg, po), rel_err(ug, uo))


def test_split_equals_fused_over_a_plane_wave_run():
    d, m, ncell, steps = 3, 2, [24, 20, 16], 30
    dt = I.cfl_dt(ncell)
    st = I.plane_wave(m, ncell, dt, seed=3, kmax=3.0)
    ps, us = run(d, m, ncell, dt, st, steps, 1)
    pf, uf = run(d, m, ncell, dt, st, steps, 0)
    assert rel_err(ps, pf) <= 1e-12 and rel_err(us, uf) <= 1e-12


def test_split_validation():
    h = hl.hl_create(2, 3, [8, 8], 0.1)
    try:
        hl.hl_set_precision(h, hl.HL_FP32)
        with pytest.raises(hl.HLError):
            hl.hl_set_option(h, hl.HL_OPT_SPLIT, 1)
        hl.hl_set_precision(h, hl.HL_FP64)
        hl.hl_set_option(h, hl.HL_OPT_SPLIT, 1)
        with pytest.raises(hl.HLError):
            hl.hl_set_precision(h, hl.HL_FP32)
        with pytest.raises(hl.HLError):
            hl.hl_set_option(h, hl.HL_OPT_SPLIT, 2)
    finally:
        hl.hl_destroy(h)
    h = hl.hl_create(2, 4, [8, 8], 0.1)
    try:
        with pytest.raises(hl.HLError):
            hl.hl_set_option(h, hl.HL_OPT_SPLIT, 1)
    finally:
        hl.hl_destroy(h)
