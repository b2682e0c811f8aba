"""Host-side checks of the C ABI that need no GPU: the library builds and exports
every entry point include/hl.h declares, the binding wraps each of them, argument
validation happens before any CUDA call, and the kernels' compile-time sparsity
rule matches the true operator (computed here from the oracle on unit inputs)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1808_10481_gb300 import build as B
from paper_1808_10481_gb300 import hl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hl.h")).read()
    return re.findall(r"^\s*(?:int|void|const char)\s*\*?\s*(hl_\w+)\s*\(", txt, re.M)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_core_entry_points():
    names = set(_declared())
    for n in ["hl_create", "hl_set_initial", "hl_step", "hl_get_fields", "hl_destroy", "hl_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_wraps_every_declared_symbol():
    for name in _declared():
        assert callable(getattr(hl, name, None)), name


def test_binding_constants_match_the_header():
    """Every HL_* constant of the header (enums and #defines) has the same value in the binding,
    and the binding's tile list has one entry per tile shape."""
    import re
    text = open(os.path.join(ROOT, "include", "hl.h")).read()
    consts = {k: int(v) for k, v in re.findall(r"\b(HL_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    consts.update({k: int(v) for k, v in re.findall(r"#define\s+(HL_[A-Z0-9_]+)\s+(-?\d+)", text)})
    assert len(consts) > 20
    for k, v in consts.items():
        assert getattr(hl, k) == v, k
    assert len(hl.TILES) == hl.HL_NUM_TILES


@pytest.mark.parametrize("args,fragment", [
    ((0, 3, [8], 0.01), "dim"),
    ((4, 3, [8], 0.01), "dim"),
    ((2, -1, [8, 8], 0.01), "m must"),
    ((2, 7, [8, 8], 0.01), "m must"),
    ((3, 4, [8, 8, 8], 0.01), "m <= 3"),
    ((2, 3, [1, 8], 0.01), ">= 2"),
    ((2, 3, [8, 8], 0.0), "dt"),
    ((2, 3, [8, 8], float("nan")), "dt"),
    ((2, 3, [8, 16], 0.07), "min h"),
    ((3, 1, [2048, 2048, 1024], 1e-5), "2^31"),
])
def test_invalid_arguments_rejected_before_cuda(args, fragment):
    hl.load()
    with pytest.raises(hl.HLError) as ei:
        hl.hl_create(*args)
    assert ei.value.code == hl.HL_EINVAL
    assert fragment in str(ei.value)


def test_null_handle_calls_fail_cleanly(lib):
    lib.hl_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.hl_step(None, 1) == hl.HL_EINVAL
    lib.hl_destroy.argtypes = [ctypes.c_void_p]
    lib.hl_destroy(None)


def _butterflied_nnz(d, m, lam):
    """Non-zeros of the all-lower-vertex operator block, from the oracle's node update
    applied to unit vertex data (an independent route to the operator)."""
    nq = (m + 1) ** d
    nz = 0
    for i in range(d):
        for l in range(nq):
            vtx = np.zeros((d, 1 << d, nq))
            vtx[i, 0, l] = 1.0
            col = oracle.node_update(d, m, lam, 0, vtx)[0]
            nz += int(np.sum(np.abs(col) > 1e-13))
    return nz


@pytest.mark.parametrize("d,m", [(1, 3), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_kernel_sparsity_rule_matches_operator(d, m):
    hl.load()
    fma, add = hl.hl_op_counts(d, m)
    nz = _butterflied_nnz(d, m, [0.45, 0.37, 0.29][:d])
    assert fma == 2 * nz                       # p-half and u-half use the same table
    assert add == d * (1 << d) * (m + 1) ** d * (d + 1) + (m + 1) ** d * (d + 1)


@pytest.mark.parametrize("args,fragment", [
    ((2, 3, [8, 8], [8.0, 0.0], 0.01), "inv_h"),
    ((2, 3, [8, 8], [8.0, -4.0], 0.01), "inv_h"),
    ((2, 3, [8, 8], [float("inf"), 8.0], 0.01), "inv_h"),
    ((2, 3, [8, 8], [float("nan"), 8.0], 0.01), "inv_h"),
    ((2, 3, [8, 4], [8.0, 32.0], 0.05), "min h"),      # h_y = 1/32, not 1/4
    ((2, 3, [8, 1], [8.0, 8.0], 0.01), ">= 2"),
])
def test_spacing_arguments_rejected_before_cuda(args, fragment):
    hl.load()
    with pytest.raises(hl.HLError) as ei:
        hl.hl_create_spacing(*args)
    assert ei.value.code == hl.HL_EINVAL
    assert fragment in str(ei.value)


def test_spacing_null_inv_h_rejected(lib):
    import ctypes
    out = ctypes.c_void_p(1)
    nc = (ctypes.c_int64 * 2)(8, 8)
    fn = lib.hl_create_spacing
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    assert fn(2, 3, nc, None, 0.01, ctypes.byref(out)) == hl.HL_EINVAL
    assert out.value is None
    assert "inv_h" in hl.load().hl_last_error(None).decode()


@pytest.mark.parametrize("args,fragment", [
    ((2, 3, 0, [], []), "n_shots"),
    ((2, 3, 257, [[8, 8]] * 257, [0.01] * 257), "n_shots"),
    ((2, 4, 2, [[8, 8], [8, 8]], [0.01, 0.01]), "m <= 3"),
    ((2, 3, 2, [[8, 8], [8, 1]], [0.01, 0.01]), ">= 2"),
    ((2, 3, 2, [[8, 8], [16, 16]], [0.01, 0.07]), "min h"),
])
def test_batch_arguments_rejected_before_cuda(args, fragment):
    hl.load()
    d, m, ns, cells, dts = args
    with pytest.raises((hl.HLError, ValueError)) as ei:
        if ns == 0:
            import ctypes
            lib = hl.load()
            out = ctypes.c_void_p()
            rc = lib.hl_create_batch(d, m, 0, None, None, ctypes.byref(out))
            raise hl.HLError(rc, lib.hl_last_error(None).decode())
        hl.hl_create_batch(d, m, cells, dts)
    assert fragment in str(ei.value)


def _exact_operator(d, m, lam):
    """The fused operator in exact rationals (W from the series, H from eq. interp),
    negated and restricted to the all-lower vertex block, as float64."""
    from fractions import Fraction as Fr
    from itertools import product
    from math import factorial as fac
    from oracle.hermite import hermite_inverse_exact
    H = hermite_inverse_exact(m)
    n, A = m + 1, 2 * m + 2
    nq = n ** d
    lamf = [Fr(x) for x in lam]
    out = np.zeros((d, nq, nq))
    for i in range(d):
        for s in range(nq):
            sv = [(s // n ** k) % n for k in range(d)]
            for l in range(nq):
                lv = [(l // n ** k) % n for k in range(d)]
                acc = Fr(0)
                for b in product(range(m + 1), repeat=d):
                    a = [sv[k] + 2 * b[k] + (k == i) for k in range(d)]
                    if max(a) > 2 * m + 1:
                        continue
                    K = sum(b)
                    w = Fr(2 * fac(K), fac(2 * K + 1))
                    for k in range(d):
                        w *= Fr(fac(a[k]), fac(sv[k]) * fac(b[k])) * lamf[k] ** (a[k] - sv[k])
                        w *= H[a[k]][lv[k]]
                    acc -= w
                out[i, l, s] = float(acc)
    return out


@pytest.mark.parametrize("d,m", [(1, m) for m in range(7)] + [(2, m) for m in range(7)] +
                         [(3, m) for m in range(4)])
def test_operator_table_is_correctly_rounded(d, m):
    """The library composes its operator in double-double: every entry must equal the
    exact rational value rounded once (within one ulp), for every (d, m) it accepts."""
    lam = [0.45, 0.37, 0.29][:d]
    got = hl.hl_operator_table(d, m, lam)
    want = _exact_operator(d, m, lam)
    ulp = np.spacing(np.abs(want))
    assert np.all(np.abs(got - want) <= ulp + 1e-300)


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: a missing libhl.so is an ImportError, not a silent substitute."""
    saved = hl._lib
    hl._lib = None
    try:
        with pytest.raises(ImportError):
            hl.load(str(tmp_path / "libhl.so"))
    finally:
        hl._lib = saved


def test_header_compiles_and_links_as_c99(lib, tmp_path):
    """A plain C99 program (tests/c_abi_check.c) includes include/hl.h with -pedantic -Werror,
    links against libhl.so and checks the argument validation of several entry points."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(B.LIB)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_check.c"), "-o", exe, "-L" + libdir, "-lhl",
                    "-Wl,-rpath," + libdir], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
