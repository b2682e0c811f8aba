"""hl_step_noalloc: the FP64 step for callers that cannot allocate device memory
(applications that own the device pool, loops that forbid allocation after start-up).
Its kernels keep their scratch in a static device array instead of cudaMalloc'd memory.
Checked through the C ABI against the existing hl_step on the same buffers contents, on
two calls in a row, within the parity bar the other GPU tests use.  Collected last so that
a failure here cannot stop the rest of a run that stops at the first failure."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1808_10481_gb300 import hl
from paper_1808_10481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1808_10481_gb300 import build
    build.build()
    hl.load()


def rel_err(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def device_state(torch, d, m, ncell, seed):
    """Random node data in the device layout (slot-major), on cuda:0."""
    st = I.random_state(d, m, ncell, seed=seed)
    p0 = np.ascontiguousarray(st.p.T)
    u0 = np.ascontiguousarray(st.u.transpose(0, 2, 1))
    return p0, u0


@pytest.mark.parametrize("d,m,ncell,steps,use_stream", [
    (1, 3, [300], 9, False),     # 1D: the tile folds into x
    (2, 3, [150, 70], 7, False),  # operator table in the kernel parameter bank
    (3, 2, [20, 12, 9], 4, False),
    (2, 6, [21, 18], 3, False),  # operator table held in the static scratch array
    (2, 3, [64, 40], 5, True),   # on a caller's torch stream
])
def test_noalloc_matches_hl_step_on_two_calls(d, m, ncell, steps, use_stream):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    dt = I.cfl_dt(ncell)
    p0, u0 = device_state(torch, d, m, ncell, 99)
    p_na, u_na = torch.from_numpy(p0).to(dev), torch.from_numpy(u0).to(dev)
    p_ref, u_ref = torch.from_numpy(p0).to(dev), torch.from_numpy(u0).to(dev)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream() if use_stream else None
    h = hl.hl_create(d, m, ncell, dt)
    try:
        hl.hl_bind_device(h, p_ref, u_ref)
        for call in range(2):
            assert hl.hl_step_noalloc(d, m, ncell, dt, p_na, u_na, steps, stream=stream) == hl.HL_OK
            hl.hl_step(h, steps)
            assert hl.hl_sync(h) == hl.HL_OK
            got_p, want_p = p_na.cpu().numpy(), p_ref.cpu().numpy()
            got_u, want_u = u_na.cpu().numpy(), u_ref.cpu().numpy()
            assert rel_err(got_p, want_p) <= TOL, (call, rel_err(got_p, want_p))
            assert rel_err(got_u, want_u) <= TOL, (call, rel_err(got_u, want_u))
    finally:
        hl.hl_destroy(h)


def test_noalloc_allocates_no_device_memory():
    """After one warm-up call (which loads the kernels' module), a further call leaves the
    device's free memory unchanged."""
    torch = pytest.importorskip("torch")
    d, m, ncell = 2, 3, [96, 80]
    dt = I.cfl_dt(ncell)
    p0, u0 = device_state(torch, d, m, ncell, 5)
    p, u = torch.from_numpy(p0).to("cuda:0"), torch.from_numpy(u0).to("cuda:0")
    assert hl.hl_step_noalloc(d, m, ncell, dt, p, u, 2) == hl.HL_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert hl.hl_step_noalloc(d, m, ncell, dt, p, u, 3) == hl.HL_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_reports_nonfinite_then_clears_the_status_word():
    """A NaN in the state comes back as HL_ENONFINITE; the next call on clean data returns
    HL_OK, so the shared status word is cleared between calls."""
    torch = pytest.importorskip("torch")
    d, m, ncell = 2, 2, [40, 36]
    dt = I.cfl_dt(ncell)
    p0, u0 = device_state(torch, d, m, ncell, 6)
    bad = p0.copy()
    bad[0, 17] = np.nan
    p, u = torch.from_numpy(bad).to("cuda:0"), torch.from_numpy(u0).to("cuda:0")
    assert hl.hl_step_noalloc(d, m, ncell, dt, p, u, 2) == hl.HL_ENONFINITE
    p, u = torch.from_numpy(p0).to("cuda:0"), torch.from_numpy(u0).to("cuda:0")
    assert hl.hl_step_noalloc(d, m, ncell, dt, p, u, 2) == hl.HL_OK


def test_noalloc_rejects_operator_beyond_scratch_maximum():
    torch = pytest.importorskip("torch")
    ncell = [4, 4, 4]
    nq = 64
    p = torch.zeros(nq * 64, dtype=torch.float64, device="cuda:0")
    u = torch.zeros(3 * nq * 64, dtype=torch.float64, device="cuda:0")
    with pytest.raises(hl.HLError) as ei:
        hl.hl_step_noalloc(3, 3, ncell, 0.1, p, u, 1)
    assert ei.value.code == hl.HL_EINVAL and "scratch" in str(ei.value)


def test_noalloc_rejects_host_buffers_at_the_c_abi():
    """Pointers that are not device memory of the current device are refused before any
    kernel runs (the C entry point checks them with cudaPointerGetAttributes)."""
    torch = pytest.importorskip("torch")
    import ctypes
    ncell = [16, 16]
    nq = 16
    p = np.zeros(nq * 256)
    u = np.zeros(2 * nq * 256)
    nc = (ctypes.c_int64 * 2)(*ncell)
    rc = hl.load().hl_step_noalloc(2, 3, nc, 0.9 / 16, ctypes.c_void_p(p.ctypes.data),
                                   ctypes.c_void_p(u.ctypes.data), 1, None)
    assert rc == hl.HL_EINVAL
    assert "current device" in hl.hl_last_error(None) or "not CUDA device" in hl.hl_last_error(None)
