"""The operator images the tcgen05 tensor-core kernels load (built on the host by the
library, hl_tc_image) against the oracle, in the layouts the kernels read them.

Every entry is the FP16 bit pattern of a balanced base-256 digit (an integer in
[-128, 127], exact in FP16); reassembled with its column exponent it must equal the vertex
form of the fused operator (the oracle's node increment per unit of one partner slot at one
cell vertex) within half the column's quantum 2^(e - 47), plus the oracle's own rounding.
The zero digit block (j = 6), the padded slots and the padded output columns must be zero."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1808_10481_gb300 import hl


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1808_10481_gb300 import build
    build.build()
    hl.load()


def f16(bits):
    return np.asarray(bits, dtype=np.uint16).view(np.float16).astype(np.float64)


def reassemble(d):
    """Digit rows d[j] (j = 0..6, most significant first) -> sum_j d_j 256^(5-j)."""
    return sum(d[j] * 256.0 ** (5 - j) for j in range(6))


@pytest.mark.parametrize("m", [0, 3])
def test_2d_images_reassemble_the_vertex_operator(m):
    lam = [0.45, 0.3]
    img, ex = hl.hl_tc_image(2, m, lam)
    d = f16(img)
    assert np.all(d == np.round(d)) and d.min() >= -128 and d.max() <= 127
    nq = (m + 1) ** 2
    # p-half: blocks b = c*4 + v of [2 chunks][112 rows n = j*16 + s][8]
    P = d[0].reshape(8, 2, 7, 16, 8)                        # (b, ch, j, s, k)
    assert np.all(P[:, :, 6] == 0.0)
    for c in range(2):
        for v in range(4):
            for l in range(16):
                col = reassemble(P[c * 4 + v, l // 8, :, :, l % 8]) * 2.0 ** (ex[0] - 46)   # (s,)
                if l >= nq:
                    assert np.all(col == 0.0)
                    continue
                vtx = np.zeros((2, 4, nq))
                vtx[c, v, l] = 1.0
                want = np.zeros(16)
                want[:nq] = oracle.node_update(2, m, lam, 0, vtx)[0]
                assert np.all(np.abs(col - want) <= 2.0 ** (ex[0] - 47) + 1e-14 * np.abs(want).max()), (c, v, l)
    # u-half: blocks b = v of [2 chunks][224 rows n = j*32 + i*16 + s][8]
    U = d[1].reshape(4, 2, 7, 2, 16, 8)                     # (v, ch, j, i, s, k)
    assert np.all(U[:, :, 6] == 0.0)
    for v in range(4):
        for l in range(nq):
            vtx = np.zeros((1, 4, nq))
            vtx[0, v, l] = 1.0
            inc = oracle.node_update(2, m, lam, 1, vtx)
            for i in range(2):
                col = reassemble(U[v, l // 8, :, i, :, l % 8]) * 2.0 ** (ex[1 + i] - 46)
                want = np.zeros(16)
                want[:nq] = inc[i]
                assert np.all(np.abs(col - want) <= 2.0 ** (ex[1 + i] - 47) + 1e-14 * np.abs(want).max()), (v, l, i)


def test_3d_image_reassembles_the_vertex_operator():
    m, nq = 2, 27
    lam = [0.45, 0.4, 0.35]
    img, ex = hl.hl_tc_image(3, m, lam)
    d = f16(img)                                            # (half, unit, vv, ch, n, k)
    assert np.all(d == np.round(d)) and d.min() >= -128 and d.max() <= 127
    D = d.reshape(2, 12, 4, 2, 7, 32, 8)                    # (half, unit, vv, ch, j, s, k)
    assert np.all(D[:, :, :, :, 6] == 0.0)
    assert np.all(D[:, :, :, :, :, nq:] == 0.0)             # padded output columns
    W = {}
    for half in range(2):
        for i in range(3):
            for vz in range(2):
                for kh in range(2):
                    u = (i * 2 + vz) * 2 + kh
                    for vv in range(4):
                        v = vv + 4 * vz
                        for ch in range(2):
                            for k in range(8):
                                l = kh * 16 + ch * 8 + k
                                W[(half, i, v, l)] = reassemble(D[half, u, vv, ch, :, :, k])    # (32,)
    # padded partner slots are zero
    for (half, i, v, l), col in W.items():
        if l >= nq:
            assert np.all(col == 0.0), (half, i, v, l)
    # p-half against the oracle: W(c, v, l)[s] 2^(e_s - 46) = increment of p slot s
    colmax_p = np.zeros(nq)
    ref_p = {}
    for c in range(3):
        for v in range(8):
            for l in range(nq):
                vtx = np.zeros((3, 8, nq))
                vtx[c, v, l] = 1.0
                ref_p[(c, v, l)] = oracle.node_update(3, m, lam, 0, vtx)[0]
                colmax_p = np.maximum(colmax_p, np.abs(ref_p[(c, v, l)]))
    for s in range(nq):
        e = int(ex[0, s])
        assert colmax_p[s] < 2.0 ** e <= 2 * colmax_p[s] * (1 + 1e-12), (s, e)
    for (c, v, l), want in ref_p.items():
        got = W[(0, c, v, l)][:nq] * 2.0 ** (ex[0, :nq] - 46)
        assert np.all(np.abs(got - want) <= 2.0 ** (ex[0, :nq] - 47) + 1e-14 * colmax_p), (c, v, l)
    # u-half: W(i, v, l)[s] 2^(e_{1+i,s} - 46) = increment of u_i slot s per unit of p slot l at v
    for v in range(8):
        for l in range(nq):
            vtx = np.zeros((1, 8, nq))
            vtx[0, v, l] = 1.0
            inc = oracle.node_update(3, m, lam, 1, vtx)
            for i in range(3):
                got = W[(1, i, v, l)][:nq] * 2.0 ** (ex[1 + i, :nq] - 46)
                assert np.all(np.abs(got - inc[i]) <= 2.0 ** (ex[1 + i, :nq] - 47) + 1e-13 * np.abs(inc[i]).max()), (v, l, i)


def test_image_arguments_are_checked():
    for dim, m in ((1, 3), (2, 4), (3, 1), (3, 3)):
        with pytest.raises(hl.HLError):
            hl.hl_tc_image(dim, m, [0.45] * max(dim, 2))
