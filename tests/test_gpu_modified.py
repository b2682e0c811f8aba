"""The modified Hermite-leapfrog kernels (Section 4.3, 1D, both fields on both grids) through
the C ABI against the oracle in oracle/modified.py: random data on small and ragged grids for
every order, long runs of the paper's standing wave, the uniform 2m+2 convergence on the GPU,
and the library's error handling."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import modified as MO
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


def gpu(m, n, dt, st, steps):
    h = hl.hl_mod_create(m, n, dt)
    try:
        hl.hl_mod_set_initial(h, *st)
        hl.hl_mod_step(h, steps)
        return hl.hl_mod_get_fields(h)
    finally:
        hl.hl_mod_destroy(h)


def tol(m, steps):
    """1e-12 for m <= 4; beyond, the oracle's own binary64 interpolation cancels heavily
    (H's entries grow with m), so the bar is 64 eps times the operator row sum per step."""
    if m <= 4:
        return 1e-12
    rowsum = {5: 2e3, 6: 3e4}[m]
    return 64 * 2.0 ** -52 * rowsum * steps


@pytest.mark.parametrize("m,n,steps", [(0, 2, 5), (1, 3, 7), (2, 37, 11), (3, 64, 9), (3, 1000, 4),
                                       (4, 257, 6), (5, 50, 3), (6, 41, 3)])
def test_random_data_matches_oracle(m, n, steps):
    rng = np.random.default_rng(100 + m)
    st = tuple(rng.uniform(-1, 1, (n, m + 1)) for _ in range(4))
    dt = 0.9 / n
    got = gpu(m, n, dt, st, steps)
    ref = MO.run(m, n, dt, *st, steps)
    for g, r, name in zip(got, ref, ("p primal", "u primal", "p dual", "u dual")):
        assert rel_err(g, r) <= tol(m, steps), (name, rel_err(g, r))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_standing_wave_long_run_matches_oracle(m):
    n, steps = 64, 400
    dt = 0.9 / n
    st = I.standing_mode_1d_both_grids(m, n, dt, 3)
    got = gpu(m, n, dt, st, steps)
    # long runs are compared with the oracle in extended precision: the binary64 oracle's
    # own rounding drifts about 2e-12 over 400 steps at m = 3
    ref = MO.run(m, n, dt, *st, steps, dtype=np.longdouble)
    for g, r in zip(got, ref):
        assert rel_err(g, r) <= 1e-12


def test_gpu_convergence_is_uniform_2m_plus_2():
    """m = 3 on the GPU: the standing-wave error falls at order 8 (Table 4: 7.97 at C_CFL 0.9)."""
    m, T, errs, Ns = 3, 4.13 / 2, [], [16, 24, 32, 48]
    for N in Ns:
        steps = math.ceil(T / (0.9 / N))
        dt = T / steps
        got = gpu(m, N, dt, I.standing_mode_1d_both_grids(m, N, dt, 3), steps)
        ex = I.standing_mode_1d_both_grids(m, N, dt, 3, t0=steps * dt)
        errs.append(math.sqrt(np.sum((got[0][:, 0] - ex[0][:, 0]) ** 2) / N))
    rate = float(np.polyfit(np.log(1.0 / np.array(Ns)), np.log(errs), 1)[0])
    assert abs(rate - 7.97) <= 0.35, rate


def test_nonfinite_and_validation():
    with pytest.raises(hl.HLError):
        hl.hl_mod_create(7, 16, 0.01)
    with pytest.raises(hl.HLError):
        hl.hl_mod_create(2, 16, 1.0 / 16)
    n, m = 16, 2
    st = [np.zeros((n, m + 1)) for _ in range(4)]
    st[2][3, 1] = np.nan
    h = hl.hl_mod_create(m, n, 0.05)
    try:
        hl.hl_mod_set_initial(h, *st)
        hl.hl_mod_step(h, 1)
        with pytest.raises(hl.HLError) as ei:
            hl.hl_mod_get_fields(h)
        assert ei.value.code == hl.HL_ENONFINITE
        steps, tp, td = hl.hl_mod_info(h)
        assert steps == 1 and tp == pytest.approx(0.05) and td == pytest.approx(0.075)
    finally:
        hl.hl_mod_destroy(h)
