"""The integer bit logic of the tensor-core split mode's digit scheme
(csrc/hl_tc_bits.cuh), built for the host from the same header and checked against exact
rational arithmetic:

* t5_fixed(v, emax) = trunc(v 2^(48 - E)) + 0x8080808080 with 2^E = 2^(emax - 1022) above
  |v| (zero for zero, subnormal and non-finite v);
* the digit words of two such values decode, after the packed FP16 subtraction the kernels
  apply (1152, or 1536 for the top digit), to balanced base-256 digits (top digit in
  [-256, 256], the others in [-128, 127]) whose sum d_i 256^(5-i) is the fixed-point value;
* t5_scaled_f64(f, k) = f 2^k exactly.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
BIAS = 0x8080808080


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    out = str(tmp_path_factory.mktemp("tcbits") / "libtcbits.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CUDA_INC,
                    "-D__device__=", "-D__forceinline__=inline",
                    os.path.join(HERE, "tc_bits_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    L.fixed_many.argtypes = [P, P, P, ctypes.c_long]
    L.digit_words_many.argtypes = [P, P, ctypes.c_long]
    L.scaled_many.argtypes = [P, P, P, ctypes.c_long]
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _bexp(v):
    return int((np.float64(v).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF))


def _fixed(L, v, emax):
    v = np.ascontiguousarray(v, np.float64)
    e = np.ascontiguousarray(emax, np.int32)
    y = np.empty(v.size, np.int64)
    L.fixed_many(_p(v), _p(e), _p(y), v.size)
    return y


def _trunc(fr: Fraction) -> int:
    q = abs(fr.numerator) // fr.denominator
    return q if fr >= 0 else -q


def test_fixed_point_is_the_truncated_scaled_value(lib):
    rng = np.random.default_rng(11)
    n = 20000
    v = rng.uniform(-1, 1, n) * 2.0 ** rng.integers(-60, 60, n)
    v[::17] = 0.0
    emax = np.array([_bexp(x) for x in v]) + rng.integers(0, 4, n)
    emax[v == 0.0] = 1023
    y = _fixed(lib, v, emax)
    for x, e, got in zip(v[:4000], emax[:4000], y[:4000]):
        want = _trunc(Fraction(float(x)) * Fraction(2) ** (48 - (int(e) - 1022)))
        assert abs(want) < 2 ** 48
        assert int(got) - BIAS == want, (x, e)
    # zero, subnormal and non-finite values give zero
    odd = np.array([0.0, -0.0, 5e-324, -2e-310, np.inf, -np.inf, np.nan])
    assert np.all(_fixed(lib, odd, np.full(odd.size, 1023)) == BIAS)


def _f16_value(bits):
    return np.asarray(bits, np.uint16).view(np.float16).astype(np.float64)


def test_digit_words_decode_to_the_balanced_digits(lib):
    rng = np.random.default_rng(12)
    n = 20000
    v = rng.uniform(-1, 1, 2 * n) * 2.0 ** rng.integers(-30, 30, 2 * n)
    v[::11] = 0.0
    v[1::13] = -v[1::13]
    emax = np.array([_bexp(x) for x in v]) + rng.integers(0, 3, 2 * n)
    emax[v == 0.0] = 1023
    y = _fixed(lib, v, emax)
    # extremes of the 48-bit range: all-ones and the largest negative
    y[:4] = BIAS + np.array([2 ** 48 - 1, -(2 ** 48 - 1), 2 ** 40, -(2 ** 40)], dtype=np.int64)
    w = np.empty(6 * n, np.uint32)
    lib.digit_words_many(_p(y), _p(w), n)
    w = w.reshape(n, 6)
    for half, shift in ((0, 0), (1, 16)):
        bits = ((w >> np.uint32(shift)) & np.uint32(0xFFFF)).astype(np.uint16)
        vals = _f16_value(bits)
        d = vals - np.array([1536.0] + [1152.0] * 5)
        assert np.all(d == np.round(d))
        assert d[:, 0].min() >= -256 and d[:, 0].max() <= 256
        assert d[:, 1:].min() >= -128 and d[:, 1:].max() <= 127
        X = sum(d[:, i].astype(np.int64) * (256 ** (5 - i)) for i in range(6))
        assert np.array_equal(X, y[half::2] - BIAS)


def test_scaled_is_exact(lib):
    rng = np.random.default_rng(13)
    n = 5000
    f = (rng.uniform(-1, 1, n) * 2.0 ** rng.integers(-100, 100, n)).astype(np.float32)
    f[::9] = 0.0
    k = rng.integers(-200, 200, n).astype(np.int32)
    out = np.empty(n)
    lib.scaled_many(_p(f), _p(k), _p(out), n)
    for a, kk, got in zip(f, k, out):
        assert Fraction(float(got)) == Fraction(float(a)) * Fraction(2) ** int(kk), (a, kk)
