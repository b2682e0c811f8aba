"""The binary64 <-> binary32 conversions and float-float operations of the mixed-precision
kernels (csrc/hl_split.cuh), built for the host from the same header and checked against
exact rational arithmetic:

* split_f64(x) = (hi, lo): hi is x rounded to nearest-even binary32, lo is x - hi truncated
  to 24 significant bits, |x - hi - lo| <= 2^-47 |x|; magnitudes below 2^-126 flush to zero;
  Inf/NaN pass through (and a hi that rounds past the binary32 range becomes Inf);
* f32_to_f64 is exact on normal binary32 values and flushes subnormals;
* TwoSum is error-free: s = fl(a + b) and s + e = a + b exactly;
* a float-float dot product (ff_fma) keeps the error of 64 terms far below binary32's.
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
F32_MIN_NORMAL = 2.0 ** -126


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("split") / "libsplit.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-I", CUDA_INC,
                    os.path.join(HERE, "split_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    for name, n in (("split_many", 3), ("widen_many", 2), ("two_sum_many", 4)):
        getattr(L, name).argtypes = [P] * n + [ctypes.c_long]
    L.ff_dot_many.argtypes = [P] * 4 + [ctypes.c_long, ctypes.c_long, P, P]
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _split(L, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    hi, lo = np.empty(x.size, np.float32), np.empty(x.size, np.float32)
    L.split_many(_p(x), _p(hi), _p(lo), x.size)
    return hi, lo


def _edge_values():
    f = [0.0, -0.0, 5e-324, -2.2250738585072014e-308, F32_MIN_NORMAL, -F32_MIN_NORMAL,
         F32_MIN_NORMAL * (1 - 2.0 ** -53), F32_MIN_NORMAL * (1 + 2.0 ** -52),
         1.0, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 1 + 2.0 ** -24 + 2.0 ** -60, 1 - 2.0 ** -25,
         2 - 2.0 ** -52, -(2 - 2.0 ** -52), 2.0 ** -100 + 2.0 ** -160, 1.0 / 3.0, -0.1,
         float(np.finfo(np.float32).max), (2 - 2.0 ** -24) * 2.0 ** 127, (2 - 2.0 ** -23.5) * 2.0 ** 127,
         2.0 ** 128, 1e300, -1e300, float("inf"), float("-inf"), float("nan")]
    return np.array(f, dtype=np.float64)


def _random_doubles(rng, n):
    ex = rng.integers(1023 - 140, 1023 + 129, n).astype(np.uint64)
    mant = rng.integers(0, 2 ** 52, n, dtype=np.uint64)
    sign = rng.integers(0, 2, n).astype(np.uint64)
    return ((sign << np.uint64(63)) | (ex << np.uint64(52)) | mant).view(np.float64)


def _expected_lo(x: float, hi: float) -> float:
    rem = Fraction(x) - Fraction(hi)
    if rem == 0:
        return 0.0
    a = abs(rem)
    E = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** E > a:
        E -= 1
    if E < -126:
        return 0.0
    q = Fraction(2) ** (E - 23)
    t = (a / q).__floor__() * q
    return float(t if rem > 0 else -t)


def test_split_f64_rounds_truncates_and_flushes(lib):
    rng = np.random.default_rng(2024)
    x = np.concatenate([_edge_values(), _random_doubles(rng, 20000)])
    hi, lo = _split(lib, x)
    with np.errstate(over="ignore"):
        rne = x.astype(np.float32)
    bound = Fraction(1, 2 ** 47)
    for i, xi in enumerate(x.tolist()):
        h, l = float(hi[i]), float(lo[i])
        if np.isnan(xi):
            assert np.isnan(h) and l == 0.0
            continue
        if np.isinf(xi) or np.isinf(rne[i]):
            assert h == float(rne[i]) and l == 0.0, xi
            continue
        if abs(xi) < F32_MIN_NORMAL:
            assert h == 0.0 and l == 0.0 and np.signbit(h) == np.signbit(xi), xi
            continue
        assert h == float(rne[i]), (xi, h, float(rne[i]))
        want = _expected_lo(xi, h)
        assert l == want, (xi, l, want)
        if want != 0.0 or Fraction(xi) == Fraction(h):
            assert abs(Fraction(xi) - Fraction(h) - Fraction(l)) <= bound * abs(Fraction(xi))


def test_f32_to_f64_is_exact_on_normals(lib):
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32)
    extra = np.array([0x00000000, 0x80000000, 0x00000001, 0x807FFFFF, 0x00800000, 0x7F7FFFFF,
                      0x7F800000, 0xFF800000, 0x7FC00000], dtype=np.uint32)
    f = np.concatenate([extra, bits]).view(np.float32)
    out = np.empty(f.size, np.float64)
    lib.widen_many(_p(f), _p(out), f.size)
    with np.errstate(invalid="ignore"):
        ref = f.astype(np.float64)
    sub = (np.abs(ref) < F32_MIN_NORMAL) & (ref != 0)
    nan = np.isnan(ref)
    ok = ~sub & ~nan
    assert np.array_equal(out[ok], ref[ok])
    assert np.all(out[sub] == 0.0) and np.array_equal(np.signbit(out[sub]), np.signbit(ref[sub]))
    assert np.all(np.isnan(out[nan]))


def test_two_sum_is_error_free(lib):
    rng = np.random.default_rng(11)
    n = 20000
    a = (rng.standard_normal(n) * 2.0 ** rng.integers(-30, 30, n)).astype(np.float32)
    b = (rng.standard_normal(n) * 2.0 ** rng.integers(-30, 30, n)).astype(np.float32)
    s, e = np.empty(n, np.float32), np.empty(n, np.float32)
    lib.two_sum_many(_p(a), _p(b), _p(s), _p(e), n)
    assert np.array_equal(s, a + b)                      # numpy float32 addition: fl(a + b)
    for i in range(0, n, 7):
        assert Fraction(float(a[i])) + Fraction(float(b[i])) == Fraction(float(s[i])) + Fraction(float(e[i]))


def test_float_float_dot_product_keeps_about_46_bits(lib):
    """64-term dot products of float-float operands: the error stays below 2^-40 of
    sum |c x| (binary32 accumulation would sit near 2^-24; a dropped error term of the
    product or of the sum shows up at that level)."""
    rng = np.random.default_rng(5)
    rows, k = 300, 64
    c = rng.uniform(-1, 1, k) * 2.0 ** rng.integers(-6, 6, k)
    x = rng.uniform(-1, 1, (rows, k))
    ch, cl = _split(lib, c)
    xh, xl = _split(lib, x.ravel())
    oh, ol = np.empty(rows, np.float32), np.empty(rows, np.float32)
    lib.ff_dot_many(_p(ch), _p(cl), _p(xh), _p(xl), rows, k, _p(oh), _p(ol))
    worst = 0.0
    for r in range(rows):
        cs = [Fraction(float(ch[j])) + Fraction(float(cl[j])) for j in range(k)]
        xs = [Fraction(float(xh[r * k + j])) + Fraction(float(xl[r * k + j])) for j in range(k)]
        exact = sum(ci * xi for ci, xi in zip(cs, xs))
        scale = sum(abs(ci * xi) for ci, xi in zip(cs, xs))
        got = Fraction(float(oh[r])) + Fraction(float(ol[r]))
        worst = max(worst, float(abs(got - exact) / scale))
    assert worst < 2.0 ** -40, worst
