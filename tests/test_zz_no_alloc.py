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


@pytest.mark.parametrize("d,m,ncell,steps", [
    (2, 3, [150, 70], 7),        # operator table in the kernel parameter bank
    (3, 2, [20, 12, 9], 4),
    (2, 6, [21, 18], 3),         # operator table held in the static scratch array
])
def test_noalloc_matches_hl_step_on_two_calls(d, m, ncell, steps):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    dt = I.cfl_dt(ncell)
    st = I.random_state(d, m, ncell, seed=99)
    # device layout (slot-major) buffers owned by the caller
    p0 = np.ascontiguousarray(st.p.T)
    u0 = np.ascontiguousarray(st.u.transpose(0, 2, 1))
    p_na, u_na = torch.from_numpy(p0).to(dev), torch.from_numpy(u0).to(dev)
    p_ref, u_ref = torch.from_numpy(p0).to(dev), torch.from_numpy(u0).to(dev)
    torch.cuda.synchronize()
    h = hl.hl_create(d, m, ncell, dt)
    try:
        hl.hl_bind_device(h, p_ref, u_ref)
        for call in range(2):
            assert hl.hl_step_noalloc(d, m, ncell, dt, p_na, u_na, steps) == hl.HL_OK
            hl.hl_step(h, steps)
            assert hl.hl_sync(h) == hl.HL_OK
            got_p, want_p = p_na.cpu().numpy(), p_ref.cpu().numpy()
            got_u, want_u = u_na.cpu().numpy(), u_ref.cpu().numpy()
            assert rel_err(got_p, want_p) <= TOL, (call, rel_err(got_p, want_p))
            assert rel_err(got_u, want_u) <= TOL, (call, rel_err(got_u, want_u))
    finally:
        hl.hl_destroy(h)


def test_noalloc_rejects_operator_beyond_scratch_maximum():
    torch = pytest.importorskip("torch")
    ncell = [4, 4, 4]
    nq = 64
    p = torch.zeros(nq * 64, dtype=torch.float64, device="cuda:0")
    u = torch.zeros(3 * nq * 64, dtype=torch.float64, device="cuda:0")
    with pytest.raises(hl.HLError) as ei:
        hl.hl_step_noalloc(3, 3, ncell, 0.1, p, u, 1)
    assert ei.value.code == hl.HL_EINVAL and "scratch" in str(ei.value)
