"""CPU oracle for the Hermite-leapfrog method (arXiv 1808.10481).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: it is a plain, slow
implementation of the method in the paper's order (gather, Hermite-Birkhoff
reconstruction one axis at a time, Cauchy-Kowalevsky series term by term,
leapfrog subtraction), written in C (``hl_oracle.c``) with the exact-rational
operator H from ``hermite.py``.

Two builds of the same source: ``prec="f64"`` (IEEE binary64, the paper's
precision and the timed CPU baseline) and ``prec="dd"`` (double-double, about
106 significant bits, ``dd.hpp``; the same bits on every platform).  Long runs
are compared with the ``dd`` build, because the binary64 build's own
accumulated rounding after hundreds of steps (about 1e-12 to 5e-12 relative on
the 1D and 2D workloads) is as large as the parity bar.  Arrays passed to a
``dd`` call become (hi, lo = 0) pairs; results come back rounded to float64.

Every function is pinned by ``tests/test_oracle_pins.py`` against facts the
paper and the mathematics fix (polynomial reproduction, exact local evolution
by a matrix exponential, the Yee special case, conservation, Fourier
stability, convergence rates of Tables 1 and 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .hermite import hermite_inverse, hermite_inverse_exact, interp_system

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hl_oracle.c")
_LIBS = {"f64": os.path.join(_HERE, "_build", "liboracle.so"),
         "dd": os.path.join(_HERE, "_build", "liboracle_dd.so")}
_DEPS = [_SRC, os.path.join(_HERE, "dd.hpp")]


class DD(ctypes.Structure):
    """A double-double scalar as the double-double build passes it by value."""
    _fields_ = [("hi", ctypes.c_double), ("lo", ctypes.c_double)]
_libs: dict = {}


def build(force: bool = False) -> str:
    """Compile both builds of the oracle (gcc, OpenMP): binary64 as C, double-double as C++."""
    for prec, path in _LIBS.items():
        os.makedirs(os.path.dirname(path), exist_ok=True)
        newest = max(os.path.getmtime(f) for f in _DEPS)
        if not force and os.path.exists(path) and os.path.getmtime(path) >= newest:
            continue
        tmp = path + f".tmp{os.getpid()}"
        if prec == "dd":
            cmd = ["g++", "-O2", "-std=c++17", "-x", "c++", "-DORC_DD", "-I" + _HERE, "-ffp-contract=off",
                   "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        else:
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return _LIBS["f64"]


def _dtype(prec: str):
    return np.float64


def _load(prec: str = "f64"):
    if prec in _libs:
        return _libs[prec]
    if prec not in _LIBS:
        raise ValueError("prec must be 'f64' or 'dd'")
    build()
    lib = ctypes.CDLL(_LIBS[prec])
    R = ctypes.c_double if prec == "f64" else DD
    rp = ctypes.POINTER(R)
    i64p = ctypes.POINTER(ctypes.c_int64)
    I, L = ctypes.c_int, ctypes.c_int64
    sig = {
        "oracle_node_update": [I, I, rp, rp, I, rp, rp],
        "oracle_half_step": [I, I, i64p, rp, rp, I, rp, rp],
        "oracle_half_step_nodes": [I, I, i64p, rp, rp, I, rp, rp, i64p, L, rp],
        "oracle_run": [I, I, i64p, rp, rp, rp, rp, L],
        "oracle_add_source": [I, I, i64p, rp, R, R, R, R, R, rp],
        "oracle_run_source": [I, I, i64p, rp, rp, R, rp, R, R, R, L, rp, rp, L],
        "oracle_set_threads": [I],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = None
    lib.oracle_threads.restype = ctypes.c_int
    _libs[prec] = lib
    return lib


def _ptr(a: np.ndarray):
    """Pointer to a float64 array (binary64) or to a (..., 2) hi/lo array (double-double)."""
    ct = DD if (a.ndim and a.shape[-1] == 2 and getattr(a, "_is_dd", False)) else ctypes.c_double
    return a.ctypes.data_as(ctypes.POINTER(ct))


class _DDArray(np.ndarray):
    _is_dd = True


def _arr(a, prec: str, copy: bool = False) -> np.ndarray:
    x = np.array(a, dtype=np.float64, order="C", copy=True) if copy else np.ascontiguousarray(a, dtype=np.float64)
    if prec == "f64":
        return x
    y = np.zeros(x.shape + (2,), dtype=np.float64)
    y[..., 0] = x
    return y.view(_DDArray)


def _scalar(x: float, prec: str):
    return float(x) if prec == "f64" else DD(float(x), 0.0)


def _h_array(m: int, prec: str = "f64") -> np.ndarray:
    # H is dyadic (exact in binary64) for every m <= 6, so the conversion is exact
    return _arr(np.array(hermite_inverse(m), dtype=np.float64), prec)


def _nc(ncell):
    return np.array(list(ncell) + [1] * (3 - len(ncell)), dtype=np.int64)


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _out(a: np.ndarray, raw: bool = False):
    """float64 result; for a double-double array hi + lo (rounded once), or the pair if raw."""
    if a.ndim and getattr(a, "_is_dd", False):
        a = np.asarray(a)
        return a if raw else a[..., 0] + a[..., 1]
    return a


def lambdas(ncell, dt: float, prec: str = "f64", inv_h=None) -> np.ndarray:
    """lam_k = dt / (2 h_k), computed in binary64 as dt * (1/h_k) / 2.  By default
    h_k = 1/ncell_k (periodic unit box); inv_h gives 1/h_k explicitly (a grid of
    ncell_k nodes spaced h_k apart, e.g. one slab of a larger grid)."""
    inv = list(ncell) if inv_h is None else list(inv_h)
    lam = np.array([dt * float(n) / 2.0 for n in inv] + [0.0] * (3 - len(inv)), dtype=np.float64)
    return _arr(lam, prec)


def set_threads(n: int) -> None:
    for prec in _LIBS:
        _load(prec).oracle_set_threads(int(n))


def threads() -> int:
    return int(_load().oracle_threads())


def node_update(d: int, m: int, lam, mode: int, vtx: np.ndarray, prec: str = "f64") -> np.ndarray:
    """Increment of one target node from its 2^d vertices' partner data.

    vtx has shape (ncomp_src, 2^d, (m+1)^d); returns (ncomp_dst, (m+1)^d).
    mode 0 = p-half (src = d velocity components), mode 1 = u-half.
    """
    lib = _load(prec)
    nq = (m + 1) ** d
    ncs, ncd = (d, 1) if mode == 0 else (1, d)
    vtx = _arr(np.asarray(vtx, dtype=np.float64).reshape(ncs, 1 << d, nq), prec)
    out = _arr(np.zeros((ncd, nq)), prec)
    lam3 = np.zeros(3)
    lam3[:d] = np.asarray(lam, dtype=np.float64)[:d]
    lib.oracle_node_update(d, m, _ptr(_arr(lam3, prec)), _ptr(_h_array(m, prec)), mode, _ptr(vtx), _ptr(out))
    return _out(out)


def half_step(d: int, m: int, ncell, dt: float, mode: int, src: np.ndarray, dst: np.ndarray) -> None:
    """One binary64 half-step in place on dst (host layout f[comp][node][q])."""
    lib = _load("f64")
    assert src.dtype == np.float64 and dst.dtype == np.float64
    assert src.flags.c_contiguous and dst.flags.c_contiguous
    lib.oracle_half_step(d, m, _i64p(_nc(ncell)), _ptr(lambdas(ncell, dt)), _ptr(_h_array(m)), mode, _ptr(src),
                         _ptr(dst))


def half_step_nodes(d: int, m: int, ncell, dt: float, mode: int, src: np.ndarray, dst: np.ndarray,
                    nodes, prec: str = "f64") -> np.ndarray:
    """The half-step at the listed target nodes only; returns (ncomp_dst, len(nodes), nq).

    src/dst are full fields in host layout (dst is not modified)."""
    lib = _load(prec)
    nq = (m + 1) ** d
    ncd = 1 if mode == 0 else d
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64))
    src = _arr(src, prec)
    dst = _arr(dst, prec)
    out = _arr(np.empty((ncd, nodes.size, nq)), prec)
    lib.oracle_half_step_nodes(d, m, _i64p(_nc(ncell)), _ptr(lambdas(ncell, dt, prec)), _ptr(_h_array(m, prec)),
                               mode, _ptr(src), _ptr(dst), _i64p(nodes), nodes.size, _ptr(out))
    return _out(out)


def run(d: int, m: int, ncell, dt: float, p: np.ndarray, u: np.ndarray, n_steps: int, prec: str = "f64",
        raw: bool = False, inv_h=None):
    """n_steps leapfrog steps; returns new (p, u) arrays (inputs untouched).

    p has shape (nnode, nq), u (d, nnode, nq); node index x-fastest,
    slot q = a_0 + (m+1)(a_1 + (m+1) a_2).  inv_h: see lambdas()."""
    lib = _load(prec)
    p = _arr(p, prec, copy=True)
    u = _arr(u, prec, copy=True)
    lib.oracle_run(d, m, _i64p(_nc(ncell)), _ptr(lambdas(ncell, dt, prec, inv_h)), _ptr(_h_array(m, prec)),
                   _ptr(p), _ptr(u), int(n_steps))
    return _out(p, raw), _out(u, raw)


def add_source(d: int, m: int, ncell, x0, sigma: float, f0: float, amp: float, t_mid: float, dt: float,
               p: np.ndarray) -> None:
    """p~ += dt * amp * R(t_mid) * g~ in place (binary64; Ricker wavelet times a Gaussian)."""
    lib = _load("f64")
    assert p.dtype == np.float64 and p.flags.c_contiguous
    x = np.zeros(3)
    x[:d] = np.asarray(x0, dtype=np.float64)[:d]
    lib.oracle_add_source(d, m, _i64p(_nc(ncell)), _ptr(x), float(sigma), float(f0), float(amp), float(t_mid),
                          float(dt), _ptr(p))


def run_source(d: int, m: int, ncell, dt: float, p, u, n_steps: int, x0, sigma: float, f0: float, amp: float,
               step0: int = 0, prec: str = "f64", raw: bool = False):
    """run() with the point source injected after every p-half; returns new (p, u)."""
    lib = _load(prec)
    p = _arr(p, prec, copy=True)
    u = _arr(u, prec, copy=True)
    x = np.zeros(3)
    x[:d] = np.asarray(x0, dtype=np.float64)[:d]
    x = _arr(x, prec)
    lib.oracle_run_source(d, m, _i64p(_nc(ncell)), _ptr(lambdas(ncell, dt, prec)), _ptr(_h_array(m, prec)),
                          _scalar(dt, prec), _ptr(x), _scalar(sigma, prec), _scalar(f0, prec), _scalar(amp, prec),
                          int(step0), _ptr(p), _ptr(u), int(n_steps))
    return _out(p, raw), _out(u, raw)


__all__ = [
    "build", "node_update", "half_step", "half_step_nodes", "run", "add_source", "run_source", "lambdas",
    "set_threads", "threads", "hermite_inverse", "hermite_inverse_exact", "interp_system",
]
