"""The variable-wave-speed kernels (Section 4.2, 1D) through the C ABI against the oracle in
oracle/variable.py: random data with random positive speed tables on small, tiny and ragged
grids, the paper's c^2 = 1 + sin(x)/2 over long runs, unit speed against the constant-speed
kernels, and argument validation."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import variable as V
from paper_1808_10481_gb300 import hl
from paper_1808_10481_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1808_10481_gb300 import build
    build.build()
    hl.load()


def rel_err(got, ref):
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / max(np.abs(ref).max(), 1e-300))


def random_tables(n, m, seed):
    rng = np.random.default_rng(seed)
    A = 2 * m + 2
    tabs = []
    for _ in range(2):
        t = rng.uniform(-1, 1, (n, A)) * 0.3 ** np.arange(A)
        t[:, 0] = rng.uniform(0.5, 1.2, n)
        tabs.append(t)
    return tabs


def gpu(m, n, dt, p, u, cp, cd, steps):
    h = hl.hl_create(1, m, [n], dt)
    try:
        hl.hl_set_wave_speed(h, cp, cd)
        hl.hl_set_initial(h, p, u.reshape(1, n, m + 1))
        hl.hl_step(h, steps)
        pg, ug, _, _ = hl.hl_get_fields(h)
        return pg, ug[0]
    finally:
        hl.hl_destroy(h)


@pytest.mark.parametrize("m,n,steps", [(0, 2, 9), (1, 3, 7), (2, 37, 11), (3, 64, 9), (3, 1000, 5),
                                       (4, 129, 4), (5, 40, 3), (6, 33, 2)])
def test_random_data_and_speed_match_oracle(m, n, steps):
    cp, cd = random_tables(n, m, 500 + m)
    dt = 0.8 / n / np.sqrt(1.2)
    st = I.random_state(1, m, [n], seed=510 + m)
    pg, ug = gpu(m, n, dt, st.p, st.u[0], cp, cd, steps)
    po, uo = V.run(m, n, dt, st.p, st.u[0], cp, cd, steps)
    tol = 1e-12 if m <= 4 else 64 * 2.0 ** -52 * {5: 2e3, 6: 3e4}[m] * steps
    assert rel_err(pg, po) <= tol and rel_err(ug, uo) <= tol, (rel_err(pg, po), rel_err(ug, uo))


@pytest.mark.parametrize("m", [2, 3])
def test_sine_speed_long_run_matches_oracle(m):
    """c^2 = 1 + sin(2 pi x)/2 (the paper's speed on the unit interval), a travelling sine
    without forcing, 300 steps at C_CFL = 0.9 of the fastest speed."""
    n = 96
    dt = 0.9 / n / I.c2_max()
    p, u, _, _ = I.variable_speed_wave(m, n, dt)
    cp, cd = I.c2_taylor_table(n, m, False), I.c2_taylor_table(n, m, True)
    pg, ug = gpu(m, n, dt, p, u, cp, cd, 300)
    po, uo = V.run(m, n, dt, p, u, cp, cd, 300, dtype=np.longdouble)   # long run: extended-precision reference
    assert rel_err(pg, po) <= 1e-12 and rel_err(ug, uo) <= 1e-12


def test_unit_speed_matches_the_constant_speed_kernels():
    m, n, steps = 3, 200, 40
    dt = 0.9 / n
    st = I.random_state(1, m, [n], seed=520)
    ones = np.zeros((n, 2 * m + 2))
    ones[:, 0] = 1.0
    pv, uv = gpu(m, n, dt, st.p, st.u[0], ones, ones, steps)
    h = hl.hl_create(1, m, [n], dt)
    try:
        hl.hl_set_initial(h, st.p, st.u)
        hl.hl_step(h, steps)
        pc, uc, _, _ = hl.hl_get_fields(h)
    finally:
        hl.hl_destroy(h)
    assert rel_err(pv, pc) <= 1e-12 and rel_err(uv, uc[0]) <= 1e-12


def test_wave_speed_validation():
    m, n = 2, 16
    ones = np.zeros((n, 2 * m + 2))
    ones[:, 0] = 1.0
    h2 = hl.hl_create(2, m, [n, n], 0.9 / n)
    try:
        with pytest.raises(hl.HLError):
            hl.hl_set_wave_speed(h2, np.tile(ones, (n, 1)), np.tile(ones, (n, 1)))
    finally:
        hl.hl_destroy(h2)
    h = hl.hl_create(1, m, [n], 0.9 / n)
    try:
        fast = ones.copy()
        fast[:, 0] = 2.0        # c = sqrt(2): c dt > h at dt = 0.9 h
        with pytest.raises(hl.HLError):
            hl.hl_set_wave_speed(h, fast, fast)
        neg = ones.copy()
        neg[3, 0] = -1.0
        with pytest.raises(hl.HLError):
            hl.hl_set_wave_speed(h, neg, ones)
        hl.hl_set_wave_speed(h, ones, ones)
        with pytest.raises(hl.HLError):
            hl.hl_set_precision(h, hl.HL_FP32)
        hl.hl_set_wave_speed(h, None, None)
        hl.hl_set_precision(h, hl.HL_FP32)
    finally:
        hl.hl_destroy(h)
