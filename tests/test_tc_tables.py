"""The operator digit tables of the tensor-core split mode (built on the host by the
library, hl_tc_tables) against the oracle.

Reassembled from its base-256 digits and column exponents, every entry must equal the
vertex form of the operator (the oracle's node increment per unit of one partner slot at
one cell vertex) rounded to the table's quantum 2^(e_n - 46): within half a quantum, plus
the oracle's own rounding.  The digits must be the balanced ones the tensor-core products
assume (integers in [-128, 127], exact in BF16), and the padding must be zero."""
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


def _bf16_to_float(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("m", [0, 1, 2, 3])
@pytest.mark.parametrize("lam", [(0.45, 0.45), (0.45, 0.3)])
def test_tc_tables_reassemble_the_vertex_operator(m, lam):
    dig, ex = hl.hl_tc_tables(m, list(lam))
    d = _bf16_to_float(dig)                                       # (op, j, s, k)
    assert np.all(d == np.round(d)) and d.min() >= -128 and d.max() <= 127
    W = sum(d[:, j] * 256.0 ** (5 - j) for j in range(6)) * 2.0 ** (ex[:, :, None] - 46)   # (op, s, k)
    nq = (m + 1) ** 2
    ref = np.zeros_like(W)
    for op in range(3):
        ncomp = 2 if op == 0 else 1
        for c in range(ncomp):
            for v in range(4):
                for l in range(nq):
                    vtx = np.zeros((ncomp, 4, nq))
                    vtx[c, v, l] = 1.0
                    inc = oracle.node_update(2, m, list(lam), 0 if op == 0 else 1, vtx)
                    ref[op, :nq, (c * 4 + v) * 16 + l] = inc[0] if op == 0 else inc[op - 1]
    for op in range(3):
        for s in range(16):
            col, want = W[op, s], ref[op, s]
            mx = np.abs(want).max()
            if mx == 0.0:
                assert np.all(col == 0.0), (op, s)
                continue
            e = int(ex[op, s])
            assert mx < 2.0 ** e <= 2 * mx * (1 + 1e-12), (op, s, e, mx)      # e is the column's exponent
            assert np.abs(col - want).max() <= 2.0 ** (e - 47) + 1e-14 * mx, (op, s)
    # padding: slots beyond nq, rows of absent components, rows k >= 128
    assert np.all(W[:, nq:, :] == 0.0)
    assert np.all(W[:, :, 128:] == 0.0)
    assert np.all(W[1:, :, 64:] == 0.0)


def test_tc_tables_reject_bad_arguments():
    with pytest.raises(hl.HLError):
        hl.hl_tc_tables(4, [0.45, 0.45])
