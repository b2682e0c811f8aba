"""CPU oracle for the Hermite-leapfrog method (arXiv 1808.10481).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: it is a plain, slow, FP64
implementation of the method in the paper's order (gather, Hermite-Birkhoff
reconstruction one axis at a time, Cauchy-Kowalevsky series term by term,
leapfrog subtraction), written in C (``hl_oracle.c``) with the exact-rational
operator H from ``hermite.py``.

Every function here is pinned by ``tests/test_oracle_pins.py`` against facts
the paper and the mathematics fix (polynomial reproduction, exact local
evolution by a matrix exponential, the Yee special case, conservation,
Fourier stability, convergence rates of Tables 1 and 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

from .hermite import hermite_inverse, hermite_inverse_exact, interp_system

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hl_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_node_update.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, dp, dp]
    lib.oracle_node_update.restype = None
    lib.oracle_half_step.argtypes = [ctypes.c_int, ctypes.c_int, i64p, dp, dp, ctypes.c_int, dp, dp]
    lib.oracle_half_step.restype = None
    lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, i64p, dp, dp, dp, dp, ctypes.c_int64]
    lib.oracle_run.restype = None
    lib.oracle_half_step_nodes.argtypes = [ctypes.c_int, ctypes.c_int, i64p, dp, dp, ctypes.c_int, dp, dp,
                                            i64p, ctypes.c_int64, dp]
    lib.oracle_half_step_nodes.restype = None
    lib.oracle_add_source.argtypes = [ctypes.c_int, ctypes.c_int, i64p, dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    lib.oracle_add_source.restype = None
    lib.oracle_run_source.argtypes = [ctypes.c_int, ctypes.c_int, i64p, dp, dp, ctypes.c_double, dp,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64, dp, dp,
                                       ctypes.c_int64]
    lib.oracle_run_source.restype = None
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _h_array(m: int) -> np.ndarray:
    return np.ascontiguousarray(np.array(hermite_inverse(m), dtype=np.float64))


def lambdas(ncell, dt: float) -> np.ndarray:
    """lam_k = dt / (2 h_k) with h_k = 1/ncell_k (periodic unit box)."""
    return np.array([dt * n / 2.0 for n in ncell] + [0.0] * (3 - len(ncell)), dtype=np.float64)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def threads() -> int:
    return int(_load().oracle_threads())


def node_update(d: int, m: int, lam, mode: int, vtx: np.ndarray) -> np.ndarray:
    """Increment of one target node from its 2^d vertices' partner data.

    vtx has shape (ncomp_src, 2^d, (m+1)^d); returns (ncomp_dst, (m+1)^d).
    mode 0 = p-half (src = d velocity components), mode 1 = u-half.
    """
    lib = _load()
    nq = (m + 1) ** d
    ncs, ncd = (d, 1) if mode == 0 else (1, d)
    vtx = np.ascontiguousarray(vtx, dtype=np.float64).reshape(ncs, 1 << d, nq)
    out = np.zeros((ncd, nq), dtype=np.float64)
    lam3 = np.zeros(3)
    lam3[:d] = np.asarray(lam, dtype=np.float64)[:d]
    lib.oracle_node_update(d, m, _dptr(lam3), _dptr(_h_array(m)), mode, _dptr(vtx), _dptr(out))
    return out


def half_step(d: int, m: int, ncell, dt: float, mode: int, src: np.ndarray, dst: np.ndarray) -> None:
    """One half-step in place on dst (host layout f[comp][node][q])."""
    lib = _load()
    nc = np.array(list(ncell) + [1] * (3 - len(ncell)), dtype=np.int64)
    assert src.dtype == np.float64 and dst.dtype == np.float64
    assert src.flags.c_contiguous and dst.flags.c_contiguous
    lam = lambdas(ncell, dt)
    lib.oracle_half_step(d, m, nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(lam),
                         _dptr(_h_array(m)), mode, _dptr(src), _dptr(dst))


def half_step_nodes(d: int, m: int, ncell, dt: float, mode: int, src: np.ndarray, dst: np.ndarray,
                    nodes) -> np.ndarray:
    """The half-step at the listed target nodes only; returns (ncomp_dst, len(nodes), nq).

    src/dst are full fields in host layout (dst is not modified)."""
    lib = _load()
    nq = (m + 1) ** d
    ncd = 1 if mode == 0 else d
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64))
    src = np.ascontiguousarray(src, dtype=np.float64)
    dst = np.ascontiguousarray(dst, dtype=np.float64)
    out = np.empty((ncd, nodes.size, nq), dtype=np.float64)
    nc = np.array(list(ncell) + [1] * (3 - len(ncell)), dtype=np.int64)
    lam = lambdas(ncell, dt)
    lib.oracle_half_step_nodes(d, m, nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(lam),
                               _dptr(_h_array(m)), mode, _dptr(src), _dptr(dst),
                               nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nodes.size, _dptr(out))
    return out


def run(d: int, m: int, ncell, dt: float, p: np.ndarray, u: np.ndarray, n_steps: int):
    """n_steps leapfrog steps; returns new (p, u) arrays (inputs untouched).

    p has shape (nnode, nq) (or anything with that many float64 values), u
    (d, nnode, nq); node index x-fastest, slot q = a_0 + (m+1)(a_1 + (m+1) a_2).
    """
    lib = _load()
    p = np.array(p, dtype=np.float64, order="C", copy=True)
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    nc = np.array(list(ncell) + [1] * (3 - len(ncell)), dtype=np.int64)
    lam = lambdas(ncell, dt)
    lib.oracle_run(d, m, nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(lam),
                   _dptr(_h_array(m)), _dptr(p), _dptr(u), int(n_steps))
    return p, u


def _nc(ncell):
    return np.array(list(ncell) + [1] * (3 - len(ncell)), dtype=np.int64)


def add_source(d: int, m: int, ncell, x0, sigma: float, f0: float, amp: float, t_mid: float, dt: float,
               p: np.ndarray) -> None:
    """p~ += dt * amp * R(t_mid) * g~ in place (Ricker wavelet times a Gaussian, midpoint rule)."""
    lib = _load()
    assert p.dtype == np.float64 and p.flags.c_contiguous
    x = np.zeros(3)
    x[:d] = np.asarray(x0, dtype=np.float64)[:d]
    nc = _nc(ncell)
    lib.oracle_add_source(d, m, nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(x), float(sigma),
                          float(f0), float(amp), float(t_mid), float(dt), _dptr(p))


def run_source(d: int, m: int, ncell, dt: float, p, u, n_steps: int, x0, sigma: float, f0: float, amp: float,
               step0: int = 0):
    """run() with the point source injected after every p-half; returns new (p, u)."""
    lib = _load()
    p = np.array(p, dtype=np.float64, order="C", copy=True)
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    x = np.zeros(3)
    x[:d] = np.asarray(x0, dtype=np.float64)[:d]
    nc = _nc(ncell)
    lib.oracle_run_source(d, m, nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(lambdas(ncell, dt)),
                          _dptr(_h_array(m)), float(dt), _dptr(x), float(sigma), float(f0), float(amp),
                          int(step0), _dptr(p), _dptr(u), int(n_steps))
    return p, u


__all__ = ["add_source", "run_source",
    "build", "node_update", "half_step", "half_step_nodes", "run", "lambdas", "set_threads", "threads",
    "hermite_inverse", "hermite_inverse_exact", "interp_system",
]
