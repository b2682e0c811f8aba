"""Learned coarse-grid correction: the project's own GPU kernels (tensor-core MLP
forward/backward, Adam, feature gather, restriction targets, FP64 correction) against
the FP64 oracle in oracle/mlp.py, and what a trained network gains on held-out data."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp as M
from paper_1808_10481_gb300 import hl
from paper_1808_10481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1808_10481_gb300 import build
    build.build()
    hl.load()


def unpack(flat):
    o, out = 0, {}
    for name, shape in (("W1", (M.N_IN, M.N_H)), ("b1", (M.N_H,)), ("W2", (M.N_H, M.N_H)), ("b2", (M.N_H,)),
                        ("W3", (M.N_H, M.N_OUT)), ("b3", (M.N_OUT,))):
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    assert o == flat.size
    return out


def pack(params):
    return np.concatenate([params[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture()
def net():
    m = hl.hl_mlp_create(1234)
    yield m
    hl.hl_mlp_destroy(m)


def _batch(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, M.N_IN)).astype(np.float32)
    T = rng.standard_normal((rows, M.N_OUT)).astype(np.float32)
    return X, T


def test_forward_matches_oracle(net):
    rows = 333                                     # ragged against the 64-row tiles
    X, _ = _batch(rows, 1)
    Xd = torch.from_numpy(X).to(DEV)
    Yd = torch.empty((rows, M.N_OUT), dtype=torch.float32, device=DEV)
    hl.hl_mlp_forward(net, Xd, rows, Yd)
    torch.cuda.synchronize()
    params, _ = hl.hl_mlp_params(net)
    P = unpack(params)
    # the oracle with the operands the tensor cores see: weights and inputs rounded to BF16
    Pb = {k: (bf16(v) if k.startswith("W") else v) for k, v in P.items()}
    Y_ref, _ = M.forward(Pb, bf16(X))
    assert rel(Yd.cpu().numpy(), Y_ref) < 2e-2


def test_gradients_match_oracle(net):
    rows = 517
    X, T = _batch(rows, 2)
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    loss = hl.hl_mlp_loss_grad(net, Xd, Td, rows)
    params, grads = hl.hl_mlp_params(net, want_grads=True)
    P, G = unpack(params), unpack(grads)
    loss_ref, G_ref = M.loss_and_grads(P, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    for k in G_ref:
        assert rel(G[k], G_ref[k]) < 5e-2, (k, rel(G[k], G_ref[k]))


def test_adam_training_fits_a_smooth_map(net):
    """The kernels learn: a fixed random smooth map is fitted to a fraction of its variance."""
    rows = 4096
    rng = np.random.default_rng(3)
    X = rng.standard_normal((rows, M.N_IN)).astype(np.float32) * 0.5
    A = rng.standard_normal((M.N_IN, M.N_OUT)) / np.sqrt(M.N_IN)
    T = np.tanh(X.astype(np.float64) @ A).astype(np.float32)
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    first = hl.hl_mlp_loss_grad(net, Xd, Td, rows)
    for _ in range(300):
        hl.hl_mlp_loss_grad(net, Xd, Td, rows, want_loss=False)
        hl.hl_mlp_adam_step(net, 2e-3)
    last = hl.hl_mlp_loss_grad(net, Xd, Td, rows)
    assert last < 0.1 * first, (first, last)


def _solver(ncell, st, steps):
    h = hl.hl_create(2, 3, ncell, I.cfl_dt(ncell))
    hl.hl_set_initial(h, st.p, st.u)
    hl.hl_step(h, steps)
    hl.hl_sync(h)
    return h


def _splitmix64_nth(seed, n):
    """n-th output (n >= 1) of SplitMix64 seeded with `seed` (Steele, Lea and Flood 2014)."""
    mask = (1 << 64) - 1
    z = (seed + n * 0x9E3779B97F4A7C15) & mask
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    return z ^ (z >> 31)


def test_device_minibatch_draw_follows_splitmix64(net):
    pool, rows, seed = 1000, 64, 12345
    rng = np.random.default_rng(8)
    Xp = torch.from_numpy(rng.standard_normal((pool, M.N_IN)).astype(np.float32)).to(DEV)
    Tp = torch.from_numpy(rng.standard_normal((pool, M.N_OUT)).astype(np.float32)).to(DEV)
    X = torch.empty((rows, M.N_IN), dtype=torch.float32, device=DEV)
    T = torch.empty((rows, M.N_OUT), dtype=torch.float32, device=DEV)
    for step in (0, 1, 77):
        hl.hl_mlp_sample(net, Xp, Tp, rows, seed, step, X, T)
        torch.cuda.synchronize()
        idx = [_splitmix64_nth(seed, step * rows + i + 1) % pool for i in range(rows)]
        assert torch.equal(X.cpu(), Xp.cpu()[idx])
        assert torch.equal(T.cpu(), Tp.cpu()[idx])


def test_features_and_targets_match_oracle():
    nc, r = [20, 12], 4
    nf = [nc[0] * r, nc[1] * r]
    stc = I.gaussian_pulse(2, 3, nc, I.cfl_dt(nc), seed=4, width=0.15)
    stf = I.gaussian_pulse(2, 3, nf, I.cfl_dt(nf), seed=4, width=0.15)
    hc = _solver(nc, stc, 6)
    hf = _solver(nf, stf, 24)
    try:
        pc, uc, _, _ = hl.hl_get_fields(hc)
        pf, _, _, _ = hl.hl_get_fields(hf)
        nodes = np.array([0, 5, 19, 20, 100, 239], dtype=np.int32)
        nd = torch.from_numpy(nodes).to(DEV)
        X = torch.empty((nodes.size, M.N_IN), dtype=torch.float32, device=DEV)
        T = torch.empty((nodes.size, M.N_OUT), dtype=torch.float32, device=DEV)
        hl.hl_features(hc, nd, nodes.size, 0.75, 0.5, X)
        hl.hl_targets(hf, r, hc, nd, nodes.size, 1e-3, T)
        hl.hl_sync(hc)
        # the kernel rounds p to binary32 and then scales in binary32: within 2 ulp of the
        # oracle's single rounding of the scaled binary64 value
        Xr = M.features(pc, uc, nc, nodes, 0.75, 0.5).astype(np.float32)
        np.testing.assert_allclose(X.cpu().numpy(), Xr, rtol=2.5e-7, atol=0)
        Tr = ((M.restrict_p(pf, nf, r) - pc)[nodes] / 1e-3).astype(np.float32)
        np.testing.assert_allclose(T.cpu().numpy(), Tr, rtol=1e-6, atol=1e-6 * np.abs(Tr).max())
    finally:
        hl.hl_destroy(hc)
        hl.hl_destroy(hf)


def _trajectory(seed, nc, r, steps):
    """Coarse and fine solutions of one seeded pulse at the same time (fine = reference)."""
    rng = np.random.default_rng(seed)
    width = float(rng.uniform(0.06, 0.12))
    nf = [nc[0] * r, nc[1] * r]
    stc = I.gaussian_pulse(2, 3, nc, I.cfl_dt(nc), seed=seed, width=width)
    stf = I.gaussian_pulse(2, 3, nf, I.cfl_dt(nf), seed=seed, width=width)
    return _solver(nc, stc, steps), _solver(nf, stf, steps * r)


def test_learned_correction_gains_on_held_out_pulses():
    """Train on 24 seeded pulses (coarse 32^2 vs fine 128^2, m = 3, 12 coarse steps) and
    evaluate on 8 held-out seeds: the corrected coarse solution must be closer to the fine
    one than the plain coarse solution.  The gain is printed."""
    nc, r, steps = [32, 32], 4, 12
    rows = nc[0] * nc[1]
    Xs, Ts = [], []
    held = []
    for seed in range(32):
        hc, hf = _trajectory(seed, nc, r, steps)
        X = torch.empty((rows, M.N_IN), dtype=torch.float32, device=DEV)
        T = torch.empty((rows, M.N_OUT), dtype=torch.float32, device=DEV)
        hl.hl_features(hc, None, rows, 1.0, 0.0, X)
        hl.hl_targets(hf, r, hc, None, rows, 1.0, T)
        hl.hl_sync(hc)
        if seed < 24:
            Xs.append(X)
            Ts.append(T)
            hl.hl_destroy(hc)
            hl.hl_destroy(hf)
        else:
            held.append((hc, hf, T))
    X = torch.cat(Xs)
    T = torch.cat(Ts)
    out_scale = float(T.pow(2).mean().sqrt())
    T = T / out_scale
    n = X.shape[0]
    m = hl.hl_mlp_create(7)
    try:
        g = torch.Generator(device="cpu").manual_seed(0)
        for it in range(1500):
            idx = torch.randint(0, n, (2048,), generator=g).to(DEV)
            hl.hl_mlp_loss_grad(m, X[idx].contiguous(), T[idx].contiguous(), 2048, want_loss=False)
            hl.hl_mlp_adam_step(m, 1e-3 if it < 1000 else 3e-4)
        plain, corr = 0.0, 0.0
        for hc, hf, Tt in held:
            plain += float(Tt.pow(2).sum())
            hl.hl_apply_correction(hc, m, 1.0, 0.0, out_scale)
            T2 = torch.empty_like(Tt)
            hl.hl_targets(hf, r, hc, None, rows, 1.0, T2)
            hl.hl_sync(hc)
            corr += float(T2.pow(2).sum())
        gain = (plain / corr) ** 0.5
        print(f"learned correction: held-out error ratio plain/corrected = {gain:.2f}")
        assert gain > 1.0
    finally:
        hl.hl_mlp_destroy(m)
        for hc, hf, _ in held:
            hl.hl_destroy(hc)
            hl.hl_destroy(hf)
