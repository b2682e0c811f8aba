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


# ---------------------------------------------------------------------------------------
# Element-wise comparison of the GPU network with the FP64 oracle.  The kernels round every
# GEMM operand to BF16 (unit roundoff 2^-8) and accumulate in FP32.  The reference is the
# oracle run with the same operand rounding (oracle.mlp, operand_round = BF16), so the
# differences left are the FP32 accumulation (at most (K + 2) 2^-23 times the sum of the
# magnitudes of the terms, truncating worst case), the roundings that the accumulation
# error can flip (a value within that error of a BF16 rounding boundary), and ReLU masks it
# can flip (a pre-activation within that error of zero).  Two checks per element:
#   * a rigorous bound that propagates all three through the network (every element);
#   * a tight one: |GPU - reference| <= 2^-12 sum |terms| for all but at most 1% of the
#     elements (flips are rare), so one wrong output column, row or bias block fails.
U_BF16 = 2.0 ** -8
TIGHT = 2.0 ** -12


def g32(k):
    return (k + 2) * 2.0 ** -23


def rounded(a, ea, nonneg=False):
    """The reference's BF16 value of a and the bound of |bf16(a_gpu) - bf16(a)| given
    |a_gpu - a| <= ea (rounding is monotone: bf16(a_gpu) lies between the roundings of the
    interval's ends)."""
    ab = bf16(a)
    lo = np.maximum(a - ea, 0.0) if nonneg else a - ea
    return ab, np.maximum(np.abs(bf16(a + ea) - ab), np.abs(bf16(lo) - ab))


def product_bound(A, dA, B, dB):
    """|GPU(A B) - A B| for BF16 operands whose GPU values differ from A, B by at most dA, dB,
    with FP32 accumulation over the inner dimension."""
    aA, aB = np.abs(A), np.abs(B)
    return dA @ aB + aA @ dB + dA @ dB + g32(A.shape[1]) * ((aA + dA) @ (aB + dB))


def masked(P, eP, Z, eZ):
    """ReLU mask of a backward product: where |Z| <= eZ the GPU's mask may differ."""
    on = Z > 0
    return P * on, np.where(np.abs(Z) <= eZ, np.abs(P) + eP, eP * on)


def colsum_bound(D, eD, rows):
    return eD.sum(axis=0) + g32(rows) * (np.abs(D) + eD).sum(axis=0)


def forward_reference(P, X):
    """The oracle's forward with BF16 operands, its element-wise bounds and the magnitude
    sums of the output products."""
    Wb = {k: bf16(P[k]) for k in ("W1", "W2", "W3")}
    Xb = bf16(X)
    Y, (_, Z1, H1, Z2, H2) = M.forward(P, X, operand_round=bf16)
    z = np.zeros_like
    eZ1 = product_bound(Xb, z(Xb), Wb["W1"], z(Wb["W1"])) + 2.0 ** -23 * np.abs(Z1)
    H1b, d1 = rounded(H1, eZ1, True)
    eZ2 = product_bound(H1b, d1, Wb["W2"], z(Wb["W2"])) + 2.0 ** -23 * np.abs(Z2)
    H2b, d2 = rounded(H2, eZ2, True)
    eY = product_bound(H2b, d2, Wb["W3"], z(Wb["W3"])) + 2.0 ** -23 * np.abs(Y)
    mag = np.abs(H2b) @ np.abs(Wb["W3"]) + np.abs(P["b3"])
    return Y, eY, mag, dict(Wb=Wb, Xb=Xb, Z1=Z1, Z2=Z2, H1b=H1b, H2b=H2b, d1=d1, d2=d2, eZ1=eZ1, eZ2=eZ2)


def check_elementwise(name, got, ref, bound, mag):
    err = np.abs(np.asarray(got, dtype=np.float64) - ref)
    assert np.all(err <= bound), (name, "rigorous", float((err / bound).max()))
    frac = float(np.mean(err > TIGHT * mag + 1e-30))
    assert frac <= 0.01, (name, "tight", frac)


def test_forward_matches_oracle_elementwise(net):
    rows = 333                                     # ragged against the 64-row tiles
    X, _ = _batch(rows, 1)
    Xd = torch.from_numpy(X).to(DEV)
    Yd = torch.empty((rows, M.N_OUT), dtype=torch.float32, device=DEV)
    hl.hl_mlp_forward(net, Xd, rows, Yd)
    torch.cuda.synchronize()
    params, _ = hl.hl_mlp_params(net)
    P = unpack(params)
    Y_ref, eY, mag, _ = forward_reference(P, X.astype(np.float64))
    check_elementwise("Y", Yd.cpu().numpy(), Y_ref, eY, mag)


@pytest.mark.parametrize("rows,offset", [(2 * 152 * 128 + 77, 0), (333, 1)])
def test_forward_paths_match_oracle_elementwise(net, rows, offset):
    """Both forward paths against the oracle, element by element.  offset 0: the tcgen05
    kernel with 305 tiles of 128 rows, so its persistent CTAs (one per SM) take up to three
    tiles each, the last one ragged.  offset 1: X starts one float past a 16-byte boundary,
    which sends the call to the per-layer GEMMs."""
    X, _ = _batch(rows, 2)
    buf = torch.zeros(rows * M.N_IN + offset, dtype=torch.float32, device=DEV)
    buf[offset:] = torch.from_numpy(X.ravel()).to(DEV)
    Yd = torch.full((rows, M.N_OUT), float("nan"), dtype=torch.float32, device=DEV)
    hl.hl_mlp_forward(net, buf[offset:], rows, Yd)
    torch.cuda.synchronize()
    params, _ = hl.hl_mlp_params(net)
    P = unpack(params)
    Y_ref, eY, mag, _ = forward_reference(P, X.astype(np.float64))
    check_elementwise("Y", Yd.cpu().numpy(), Y_ref, eY, mag)


def test_gradients_match_oracle_elementwise(net):
    rows = 517
    X, T = _batch(rows, 2)
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    loss = hl.hl_mlp_loss_grad(net, Xd, Td, rows)
    params, grads = hl.hl_mlp_params(net, want_grads=True)
    P, G = unpack(params), unpack(grads)
    X64, T64 = X.astype(np.float64), T.astype(np.float64)
    Y, eY, _, c = forward_reference(P, X64)
    loss_ref, G_ref = M.loss_and_grads(P, X64, T64, operand_round=bf16)
    n = Y.size
    R = Y - T64
    assert abs(loss - loss_ref) <= float(np.sum(2 * np.abs(R) * eY + eY * eY) / n) + 1e-12 * loss_ref
    Wb, z = c["Wb"], np.zeros_like
    dY = 2.0 * R / n
    edY = 2.0 * eY / n + 2 * 2.0 ** -23 * np.abs(dY)
    dYb, ddY = rounded(dY, edY)
    bounds, mags = {}, {}
    bounds["W3"] = product_bound(c["H2b"].T, c["d2"].T, dYb, ddY)
    mags["W3"] = np.abs(c["H2b"]).T @ np.abs(dYb)
    bounds["b3"], mags["b3"] = colsum_bound(dY, edY, rows), np.abs(dY).sum(axis=0)
    P2 = dYb @ Wb["W3"].T
    dH2, edH2 = masked(P2, product_bound(dYb, ddY, Wb["W3"].T, z(Wb["W3"].T)), c["Z2"], c["eZ2"])
    dH2b, ddH2 = rounded(dH2, edH2)
    bounds["W2"] = product_bound(c["H1b"].T, c["d1"].T, dH2b, ddH2)
    mags["W2"] = np.abs(c["H1b"]).T @ np.abs(dH2b)
    bounds["b2"], mags["b2"] = colsum_bound(dH2, edH2, rows), np.abs(dH2).sum(axis=0)
    P1 = dH2b @ Wb["W2"].T
    dH1, edH1 = masked(P1, product_bound(dH2b, ddH2, Wb["W2"].T, z(Wb["W2"].T)), c["Z1"], c["eZ1"])
    dH1b, ddH1 = rounded(dH1, edH1)
    bounds["W1"] = product_bound(c["Xb"].T, z(c["Xb"].T), dH1b, ddH1)   # the GPU's BF16 X is Xb exactly
    mags["W1"] = np.abs(c["Xb"]).T @ np.abs(dH1b)
    bounds["b1"], mags["b1"] = colsum_bound(dH1, edH1, rows), np.abs(dH1).sum(axis=0)
    for k in G_ref:
        check_elementwise(k, G[k], G_ref[k], bounds[k], mags[k])


def test_adam_step_matches_oracle_elementwise(net):
    """hl_mlp_adam_step against the oracle's FP64 Adam, from the same weights and the same
    gradient, after 1 and after 5 steps (the gradient is not recomputed in between)."""
    rows = 200
    X, T = _batch(rows, 9)
    hl.hl_mlp_loss_grad(net, torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), rows, want_loss=False)
    params, grads = hl.hl_mlp_params(net, want_grads=True)
    w = {k: v.copy() for k, v in unpack(params).items()}
    g = unpack(grads)
    m1 = {k: np.zeros_like(v) for k, v in w.items()}
    m2 = {k: np.zeros_like(v) for k, v in w.items()}
    lr = 1e-3
    t = 0
    for n_steps in (1, 4):
        for _ in range(n_steps):
            hl.hl_mlp_adam_step(net, lr)
            t += 1
            M.adam_step(w, g, m1, m2, t, lr)
        got, _ = hl.hl_mlp_params(net)
        Gw = unpack(got)
        for k in w:
            # FP32 arithmetic of the kernel: a few ulp of the weight plus a relative 1e-5 of
            # the accumulated step (lr per step at most)
            tol = 4 * 2.0 ** -23 * np.abs(w[k]) + 1e-5 * lr * t + 1e-12
            assert np.all(np.abs(Gw[k] - w[k]) <= tol), (k, t, float(np.abs(Gw[k] - w[k]).max()))


def test_grad_buffer_is_the_gradient_adam_reads():
    """hl_mlp_grad_tensor shares the network's gradient: it equals the host copy after
    hl_mlp_loss_grad, and an in-place change (as a data-parallel all-reduce makes) is what
    the next Adam step uses: zeroed, the first step leaves every weight unchanged."""
    m = hl.hl_mlp_create(77)
    try:
        rows = 128
        X, T = _batch(rows, 21)
        hl.hl_mlp_loss_grad(m, torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), rows, want_loss=False)
        g = hl.hl_mlp_grad_tensor(m)
        torch.cuda.synchronize()
        w0, g_host = hl.hl_mlp_params(m, want_grads=True)
        assert g.shape == (hl.HL_MLP_NPARAMS,) and np.array_equal(g.cpu().numpy(), g_host)
        g.zero_()
        hl.hl_mlp_adam_step(m, 1e-3)
        w1, g2 = hl.hl_mlp_params(m, want_grads=True)
        assert not g2.any() and np.array_equal(w0, w1)
    finally:
        hl.hl_mlp_destroy(m)


def test_data_parallel_train_on_one_rank_is_the_plain_loop():
    """learned.train on a single rank (no all-reduce) equals the draw / loss-and-gradient /
    Adam loop bitwise."""
    from paper_1808_10481_gb300 import learned
    rows, batch, iters = 4096, 256, 5
    X, T = _batch(rows, 22)
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    a, b = hl.hl_mlp_create(5), hl.hl_mlp_create(5)
    try:
        st = torch.cuda.current_stream()
        hl.hl_mlp_set_stream(a, st)
        hl.hl_mlp_set_stream(b, st)
        learned.train(a, Xd, Td, iters, batch, lambda it: 1e-3, seed=3)
        Xb = torch.empty((batch, hl.HL_MLP_IN), dtype=torch.float32, device=DEV)
        Tb = torch.empty((batch, hl.HL_MLP_OUT), dtype=torch.float32, device=DEV)
        for it in range(iters):
            hl.hl_mlp_sample(b, Xd, Td, batch, 3, it, Xb, Tb)
            hl.hl_mlp_loss_grad(b, Xb, Tb, batch, want_loss=False)
            hl.hl_mlp_adam_step(b, 1e-3)
        wa, _ = hl.hl_mlp_params(a)
        wb, _ = hl.hl_mlp_params(b)
        assert np.array_equal(wa, wb)
    finally:
        hl.hl_mlp_destroy(a)
        hl.hl_mlp_destroy(b)


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
        assert gain > 2.0
    finally:
        hl.hl_mlp_destroy(m)
        for hc, hf, _ in held:
            hl.hl_destroy(hc)
            hl.hl_destroy(hf)


def _pulse_solver(ncell, seed=3):
    st = I.gaussian_pulse(2, 3, ncell, I.cfl_dt(ncell), seed=seed, width=0.1)
    h = hl.hl_create(2, 3, ncell, I.cfl_dt(ncell))
    hl.hl_set_initial(h, st.p, st.u)
    return h


@pytest.mark.parametrize("graph", [0, 1])
def test_set_correction_equals_the_manual_loop_bitwise(graph):
    """hl_set_correction(k = 4) over 12 steps of one hl_step call gives, bit for bit, what
    three rounds of hl_step(4) + hl_apply_correction give; with a permissive fallback bound
    all three corrections are applied (also inside a captured CUDA graph)."""
    nc = [32, 24]
    net = hl.hl_mlp_create(99)
    try:
        a = _pulse_solver(nc)
        b = _pulse_solver(nc)
        try:
            hl.hl_set_option(a, hl.HL_OPT_GRAPH, graph)
            hl.hl_set_correction(a, net, 4, 1.0, 0.0, 1e-4, 1e30)
            hl.hl_step(a, 12)
            pa, ua, _, _ = hl.hl_get_fields(a)
            assert hl.hl_correction_stats(a) == (3, 0)
            for _ in range(3):
                hl.hl_step(b, 4)
                hl.hl_apply_correction(b, net, 1.0, 0.0, 1e-4)
            pb, ub, _, _ = hl.hl_get_fields(b)
            np.testing.assert_array_equal(pa, pb)
            np.testing.assert_array_equal(ua, ub)
        finally:
            hl.hl_destroy(a)
            hl.hl_destroy(b)
    finally:
        hl.hl_mlp_destroy(net)


@pytest.mark.parametrize("bad", ["huge", "nan"])
def test_correction_fallback_keeps_the_plain_step(bad):
    """Weights injected on the host make the correction far larger than a plain step's change
    (or non-finite): every correction is skipped and the state equals the plain solver's bit
    for bit; the skips are counted."""
    nc = [32, 24]
    net = hl.hl_mlp_create(5)
    try:
        params, _ = hl.hl_mlp_params(net)
        params = params.copy()
        if bad == "huge":
            params[-16:] = 1e6          # output bias: every correction is 1e6 * out_scale
        else:
            params[-16:] = np.nan
        hl.hl_mlp_params(net, set_params=params)
        a = _pulse_solver(nc)
        b = _pulse_solver(nc)
        try:
            hl.hl_set_correction(a, net, 3, 1.0, 0.0, 1.0, 2.0)
            hl.hl_step(a, 9)
            hl.hl_step(b, 9)
            pa, ua, _, _ = hl.hl_get_fields(a)
            pb, ub, _, _ = hl.hl_get_fields(b)
            np.testing.assert_array_equal(pa, pb)
            np.testing.assert_array_equal(ua, ub)
            assert hl.hl_correction_stats(a) == (0, 3)
        finally:
            hl.hl_destroy(a)
            hl.hl_destroy(b)
    finally:
        hl.hl_mlp_destroy(net)


def test_set_correction_validation():
    net = hl.hl_mlp_create(1)
    h3 = hl.hl_create(2, 2, [16, 16], 0.05)
    h = _pulse_solver([16, 16])
    try:
        with pytest.raises(hl.HLError):
            hl.hl_set_correction(h3, net, 2, 1.0, 0.0, 1.0, 1.0)   # m = 2: the network is for m = 3
        with pytest.raises(hl.HLError):
            hl.hl_set_correction(h, net, 0, 1.0, 0.0, 1.0, 1.0)
        with pytest.raises(hl.HLError):
            hl.hl_set_correction(h, net, 2, 1.0, 0.0, -1.0, 1.0)
        hl.hl_set_correction(h, net, 2, 1.0, 0.0, 1e-6, 1.0)
        hl.hl_set_correction(h, None)
        hl.hl_step(h, 4)
        assert hl.hl_correction_stats(h) == (0, 0)
    finally:
        hl.hl_destroy(h)
        hl.hl_destroy(h3)
        hl.hl_mlp_destroy(net)
