"""The arithmetic of the tensor-core split mode (HL_TC_SPLIT), emulated on the CPU.

The GPU kernel cuts the partner data and the operator into base-256 digits after a
power-of-two scaling, multiplies digit pairs on the tensor cores with FP32 accumulation,
and relies on each level's sum staying an integer below 2^24 so that the FP32 sums are
exact.  This test replays that scheme with numpy (FP32 digit extraction with the
1.5 * 2^23 rounding constant, float-float remainder) on the operator the oracle defines,
checks the exactness bound on worst-case data, and checks that the recombined result
matches the exact product to the scheme's precision.  It does not run the kernel; the GPU
tests compare the kernel with the oracle."""
from __future__ import annotations

import numpy as np

import oracle

F = np.float32
MAGIC = F(12582912.0)


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    e = F(F(a - F(s - bb)) + F(b - bb))
    return s, e


def partner_digits(hi, lo, E):
    """Digits d_0..d_5 of (hi + lo) 2^-E, |.| < 1, as the kernel cuts them (FP32 ops)."""
    sc = F(2.0 ** -E)
    h, q = F(hi * sc), F(lo * sc)
    out = []
    for _ in range(6):
        t = F(h * F(256))
        d = F(F(t + MAGIC) - MAGIC)
        h, q = two_sum(F(t - d), F(q * F(256)))
        out.append(int(d))
    return out


def operator_digits(w, e):
    X = int(round(np.ldexp(w, 46 - e)))
    d = [0] * 6
    for j in range(5, -1, -1):
        r = X & 255
        if r >= 128:
            r -= 256
        d[j] = r
        X = (X - r) >> 8
    assert X == 0
    return d


def vertex_operator(d=2, m=3):
    nq = (m + 1) ** d
    cols = []
    for c in range(d):
        for v in range(1 << d):
            for l in range(nq):
                vtx = np.zeros((d, 1 << d, nq))
                vtx[c, v, l] = 1.0
                cols.append(oracle.node_update(d, m, [0.45] * d, 0, vtx)[0])
    return np.array(cols)          # [K = 128][N = 16]


def test_digit_products_are_exact_and_recombine_to_the_product():
    W = vertex_operator()
    K, N = W.shape
    rng = np.random.default_rng(3)
    # worst case for the level sums: every value near the block maximum, random signs
    x = rng.choice([-1.0, 1.0], K) * (1.0 - rng.random(K) * 1e-3)
    x *= 3.7                                           # block maximum below 2^E with E = 2
    hi = x.astype(F)
    lo = (x - hi.astype(np.float64)).astype(F)
    E = 2
    A = np.array([partner_digits(h, l, E) for h, l in zip(hi, lo)])      # [K][6]
    assert np.abs(A[:, 0]).max() <= 256 and np.abs(A[:, 1:]).max() <= 128
    # the digits reproduce the value to 2^-49 of the block scale
    rec = (A * (256.0 ** -np.arange(1, 7))).sum(axis=1) * 2.0 ** E
    assert np.abs(rec - (hi.astype(np.float64) + lo)).max() <= 2.0 ** (E - 48)
    approx = np.zeros(N)
    for n in range(N):
        col = W[:, n]
        e = int(np.frexp(np.abs(col).max())[1]) if np.abs(col).max() > 0 else 0
        B = np.array([operator_digits(w, e) for w in col])             # [K][6]
        for L in range(7):
            # the level sum over one partner component (64 terms), in exact integers
            for comp in range(2):
                ks = slice(comp * 64, (comp + 1) * 64)
                s = sum(int(A[ks, i] @ B[ks, L - i]) for i in range(6) if 0 <= L - i < 6)
                assert abs(s) < 2 ** 24                               # FP32 holds it exactly
                approx[n] += s * 2.0 ** (E + e - 14 - 8 * L)
    exact = (hi.astype(np.float64) + lo) @ W
    scale = np.abs(x).max() * np.abs(W).sum(axis=0).max()
    assert np.abs(approx - exact).max() <= 2.0 ** -44 * scale   # measured 2^-46.7
