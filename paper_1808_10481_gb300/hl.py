"""Thin Python binding of the C ABI in include/hl.h (libhl.so): argument marshalling only.

Every call here forwards to the CUDA library of the same name; no step of the
method runs in Python.  Host buffers are numpy float64 arrays (or CPU torch
tensors); device buffers are CUDA torch tensors (anything with ``data_ptr()``).
If libhl.so has not been built, loading fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhl.so")

HL_OK, HL_EINVAL, HL_ENOMEM, HL_ECUDA, HL_ETIMEOUT, HL_ENONFINITE, HL_ESTATE = 0, -1, -2, -3, -4, -5, -6
HL_FP64 = 0
HL_FP32 = 1
HL_FP32_COMP = 2
HL_TC_SPLIT = 3
TC_SPLIT_DIMS = (2, 3)   # HL_TC_SPLIT: dim 2 (m <= 3), dim 3 (m = 2, one shot)
HL_OPT_KERNEL_PATH = 1
HL_OPT_TIMING = 2
HL_OPT_GRAPH = 3
HL_OPT_TILE = 4
HL_OPT_STEP = 5
HL_OPT_SPLIT = 6
HL_WALL_PERIODIC, HL_WALL_DIRICHLET, HL_WALL_NEUMANN = 0, 1, 2
HL_NUM_TILES = 14
HL_NOALLOC_SCRATCH_BYTES = 65536
HL_TC_TABLE_ELEMS, HL_TC_EXPO_ELEMS = 39168, 48
HL_TC_IMAGE2_ELEMS, HL_TC_IMAGE3_ELEMS, HL_TC_EXPO3_ELEMS = 28672, 344064, 128
HL_MLP_IN, HL_MLP_HIDDEN, HL_MLP_OUT, HL_MLP_NPARAMS = 288, 128, 16, 55568
TILES = [(128, 1), (256, 1), (64, 2), (32, 4), (32, 8), (64, 4), (16, 8), (16, 16),
         (32, 4, "paired"), (32, 8, "paired"), (64, 4, "paired"), (16, 16, "paired"),
         (32, 8, "paired p-half"), (64, 4, "paired p-half")]
CODE_NAMES = {0: "HL_OK", -1: "HL_EINVAL", -2: "HL_ENOMEM", -3: "HL_ECUDA", -4: "HL_ETIMEOUT",
              -5: "HL_ENONFINITE", -6: "HL_ESTATE"}


class HLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{CODE_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double

# (name, restype, argtypes): mirrors include/hl.h
_SIGNATURES = [
    ("hl_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_I64), _D, ctypes.POINTER(_P)]),
    ("hl_create_batch", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_I64),
                                        ctypes.POINTER(_D), ctypes.POINTER(_P)]),
    ("hl_create_spacing", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_I64), ctypes.POINTER(_D),
                                          _D, ctypes.POINTER(_P)]),
    ("hl_set_initial", ctypes.c_int, [_P, _P, _P]),
    ("hl_set_initial_device", ctypes.c_int, [_P, _P, _P]),
    ("hl_get_fields_device", ctypes.c_int, [_P, _P, _P]),
    ("hl_step", ctypes.c_int, [_P, _I64]),
    ("hl_get_fields", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("hl_sync", ctypes.c_int, [_P]),
    ("hl_destroy", None, [_P]),
    ("hl_last_error", ctypes.c_char_p, [_P]),
    ("hl_set_stream", ctypes.c_int, [_P, _P]),
    ("hl_bind_device", ctypes.c_int, [_P, _P, _P]),
    ("hl_set_source", ctypes.c_int, [_P, ctypes.POINTER(_D), _D, _D, _D]),
    ("hl_set_sources", ctypes.c_int, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                       ctypes.POINTER(_D)]),
    ("hl_autotune", ctypes.c_int, [_P, _I64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_D)]),
    ("hl_set_precision", ctypes.c_int, [_P, ctypes.c_int]),
    ("hl_set_wave_speed", ctypes.c_int, [_P, _P, _P]),
    ("hl_set_walls", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    ("hl_set_option", ctypes.c_int, [_P, ctypes.c_int, _I64]),
    ("hl_kernel_times", ctypes.c_int, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    ("hl_operator_table", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("hl_tc_tables", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_D), _P, _P]),
    ("hl_tc_image", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_D), _P, _I64, _P, _I64]),
    ("hl_mlp_create", ctypes.c_int, [ctypes.c_uint64, ctypes.POINTER(_P)]),
    ("hl_mlp_destroy", None, [_P]),
    ("hl_mlp_last_error", ctypes.c_char_p, [_P]),
    ("hl_mlp_set_stream", ctypes.c_int, [_P, _P]),
    ("hl_mlp_params", ctypes.c_int, [_P, _P, _P, _P]),
    ("hl_mlp_forward", ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    ("hl_mlp_loss_grad", ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(_D)]),
    ("hl_mlp_adam_step", ctypes.c_int, [_P, ctypes.c_float]),
    ("hl_mlp_grad_buffer", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p)]),
    ("hl_mlp_sample", ctypes.c_int, [_P, _P, _P, _I64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _P, _P]),
    ("hl_features", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float, _P]),
    ("hl_targets", ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _D, _P]),
    ("hl_apply_correction", ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_float, _D]),
    ("hl_set_correction", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float, _D, _D]),
    ("hl_correction_stats", ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    ("hl_step_noalloc", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_I64), _D, _P, _P, _I64, _P]),
    ("hl_op_counts", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("hl_mod_create", ctypes.c_int, [ctypes.c_int, _I64, _D, ctypes.POINTER(_P)]),
    ("hl_mod_destroy", None, [_P]),
    ("hl_mod_last_error", ctypes.c_char_p, [_P]),
    ("hl_mod_set_stream", ctypes.c_int, [_P, _P]),
    ("hl_mod_set_initial", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("hl_mod_step", ctypes.c_int, [_P, _I64]),
    ("hl_mod_get_fields", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("hl_mod_info", ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("hl_info", ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
]


def load(path: str = LIB_PATH):
    """Load libhl.so (raises if it is missing: the library has no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhl.so not found at {path}; build it with paper_1808_10481_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


@dataclass
class Handle:
    """Opaque solver pointer plus the sizes needed to marshal buffers.

    For a batch, n_cells is a tuple of per-shot tuples and dt a tuple of floats."""
    ptr: ctypes.c_void_p
    dim: int
    m: int
    n_cells: tuple
    dt: float
    n_shots: int = 1

    @property
    def nnode(self) -> int:
        if self.n_shots == 1:
            return int(np.prod(self.n_cells))
        return int(sum(int(np.prod(c)) for c in self.n_cells))

    @property
    def nq(self) -> int:
        return (self.m + 1) ** self.dim


def _err(h) -> str:
    return load().hl_last_error(h.ptr if isinstance(h, Handle) else h).decode(errors="replace")


def _check(h, rc: int) -> int:
    if rc != HL_OK:
        raise HLError(rc, _err(h))
    return rc


def _host_ptr(a, count: int, writable: bool):
    if hasattr(a, "data_ptr"):            # CPU torch tensor
        if a.is_cuda:
            raise ValueError("expected a host buffer")
        if str(a.dtype) != "torch.float64" or not a.is_contiguous() or a.numel() != count:
            raise ValueError("host buffer must be contiguous float64 with the solver's size")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous or a.size != count:
        raise ValueError("host buffer must be a C-contiguous float64 numpy array with the solver's size")
    if writable and not a.flags.writeable:
        raise ValueError("host output buffer is read-only")
    return ctypes.c_void_p(a.ctypes.data)


def _dev_ptr(t, count: int):
    if t is None:
        return None
    if not hasattr(t, "data_ptr") or not getattr(t, "is_cuda", False):
        raise ValueError("expected a CUDA tensor")
    if str(t.dtype) != "torch.float64" or not t.is_contiguous() or t.numel() != count:
        raise ValueError("device buffer must be contiguous float64 with the solver's size")
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------------- entry points
def hl_create(dim: int, m: int, n_cells, dt: float) -> Handle:
    lib = load()
    if 1 <= dim <= 3 and len(n_cells) != dim:   # other dims are the C library's to reject
        raise ValueError("n_cells must hold dim entries")
    nc = (_I64 * len(n_cells))(*[int(x) for x in n_cells])
    out = _P()
    rc = lib.hl_create(int(dim), int(m), nc, float(dt), ctypes.byref(out))
    if rc != HL_OK:
        raise HLError(rc, lib.hl_last_error(None).decode(errors="replace"))
    return Handle(out, int(dim), int(m), tuple(int(x) for x in n_cells), float(dt))


def hl_create_spacing(dim: int, m: int, n_cells, inv_h, dt: float) -> Handle:
    """inv_h: dim entries, 1/h_k (nodes per unit length) of a periodic grid of n_cells nodes."""
    lib = load()
    if len(n_cells) != dim or len(inv_h) != dim:
        raise ValueError("n_cells and inv_h must hold dim entries")
    nc = (_I64 * dim)(*[int(x) for x in n_cells])
    ih = (_D * dim)(*[float(x) for x in inv_h])
    out = _P()
    rc = lib.hl_create_spacing(int(dim), int(m), nc, ih, float(dt), ctypes.byref(out))
    if rc != HL_OK:
        raise HLError(rc, lib.hl_last_error(None).decode(errors="replace"))
    return Handle(out, int(dim), int(m), tuple(int(x) for x in n_cells), float(dt))


def hl_create_batch(dim: int, m: int, n_cells, dt) -> Handle:
    """n_cells: sequence of per-shot node counts (each dim long); dt: per-shot steps."""
    lib = load()
    flat = [int(x) for c in n_cells for x in c]
    ns = len(dt)
    if len(flat) != ns * dim:
        raise ValueError("n_cells must hold dim entries per shot")
    nc = (_I64 * len(flat))(*flat)
    dts = (_D * ns)(*[float(x) for x in dt])
    out = _P()
    rc = lib.hl_create_batch(int(dim), int(m), ns, nc, dts, ctypes.byref(out))
    if rc != HL_OK:
        raise HLError(rc, lib.hl_last_error(None).decode(errors="replace"))
    return Handle(out, int(dim), int(m), tuple(tuple(int(x) for x in c) for c in n_cells),
                  tuple(float(x) for x in dt), ns)


def hl_set_initial(h: Handle, p, u) -> None:
    n = h.nnode * h.nq
    _check(h, load().hl_set_initial(h.ptr, _host_ptr(p, n, False), _host_ptr(u, n * h.dim, False)))


def hl_set_initial_device(h: Handle, p_dev, u_dev) -> None:
    n = h.nnode * h.nq
    _check(h, load().hl_set_initial_device(h.ptr, _dev_ptr(p_dev, n), _dev_ptr(u_dev, n * h.dim)))


def hl_get_fields_device(h: Handle, p_dev=None, u_dev=None) -> None:
    n = h.nnode * h.nq
    _check(h, load().hl_get_fields_device(h.ptr, _dev_ptr(p_dev, n), _dev_ptr(u_dev, n * h.dim)))


def hl_step(h: Handle, n_steps: int) -> None:
    _check(h, load().hl_step(h.ptr, int(n_steps)))


def hl_get_fields(h: Handle, p=None, u=None, raise_nonfinite: bool = True):
    """Copy the state to host arrays (allocated if None); returns (p, u, t_p, t_u)."""
    n = h.nnode * h.nq
    if p is None:
        p = np.empty((h.nnode, h.nq), dtype=np.float64)
    if u is None:
        u = np.empty((h.dim, h.nnode, h.nq), dtype=np.float64)
    tp, tu = _D(), _D()
    rc = load().hl_get_fields(h.ptr, _host_ptr(p, n, True), _host_ptr(u, n * h.dim, True),
                              ctypes.byref(tp), ctypes.byref(tu))
    if rc != HL_OK and (rc != HL_ENONFINITE or raise_nonfinite):
        raise HLError(rc, _err(h))
    return p, u, tp.value, tu.value


def hl_sync(h: Handle) -> int:
    """Returns HL_OK or HL_ENONFINITE; raises on CUDA failure."""
    rc = load().hl_sync(h.ptr)
    if rc not in (HL_OK, HL_ENONFINITE):
        raise HLError(rc, _err(h))
    return rc


def hl_destroy(h: Handle) -> None:
    if h is not None and h.ptr:
        load().hl_destroy(h.ptr)
        h.ptr = _P()


def hl_last_error(h: Handle | None) -> str:
    return load().hl_last_error(h.ptr if h is not None else None).decode(errors="replace")


def hl_set_stream(h: Handle, stream) -> None:
    raw = getattr(stream, "cuda_stream", stream)
    _check(h, load().hl_set_stream(h.ptr, ctypes.c_void_p(int(raw) if raw else 0)))


def hl_bind_device(h: Handle, p_dev, u_dev) -> None:
    n = h.nnode * h.nq
    _check(h, load().hl_bind_device(h.ptr, _dev_ptr(p_dev, n), _dev_ptr(u_dev, n * h.dim)))


def hl_set_source(h: Handle, x0, sigma: float, f0: float, amp: float) -> None:
    x = (_D * 3)(*([float(v) for v in x0] + [0.0] * (3 - len(x0))))
    _check(h, load().hl_set_source(h.ptr, x, float(sigma), float(f0), float(amp)))


def hl_set_sources(h: Handle, x0, sigma, f0, amp) -> None:
    ns = h.n_shots
    flat = [float(v) for row in x0 for v in row]
    if len(flat) != ns * h.dim:
        raise ValueError("x0 must hold dim coordinates per shot")
    arr = lambda v: (_D * ns)(*[float(x) for x in v])
    _check(h, load().hl_set_sources(h.ptr, (_D * len(flat))(*flat), arr(sigma), arr(f0), arr(amp)))


def hl_autotune(h: Handle, steps_per_trial: int = 2):
    """Returns (best tile index, [ms per step of each tile shape or -1])."""
    best = ctypes.c_int()
    ms = (_D * HL_NUM_TILES)()
    _check(h, load().hl_autotune(h.ptr, int(steps_per_trial), ctypes.byref(best), ms))
    return best.value, list(ms)


def hl_set_precision(h: Handle, mode: int) -> None:
    _check(h, load().hl_set_precision(h.ptr, int(mode)))


def hl_set_wave_speed(h: Handle, c2_primal, c2_dual) -> None:
    """c2 tables (nnode, 2m+2) of scaled Taylor coefficients of c^2 at the primal and dual
    nodes (dim = 1); None for both restores unit speed."""
    if c2_primal is None and c2_dual is None:
        _check(h, load().hl_set_wave_speed(h.ptr, None, None))
        return
    n = h.nnode * (2 * h.m + 2)
    cp = np.ascontiguousarray(c2_primal, dtype=np.float64)   # kept alive across the call
    cd = np.ascontiguousarray(c2_dual, dtype=np.float64)
    _check(h, load().hl_set_wave_speed(h.ptr, _host_ptr(cp, n, False), _host_ptr(cd, n, False)))


def hl_set_walls(h: Handle, kinds) -> None:
    """kinds: one HL_WALL_* per axis (or the names 'periodic'/'dirichlet'/'neumann'); None removes them."""
    if kinds is None:
        _check(h, load().hl_set_walls(h.ptr, None))
        return
    names = {"periodic": HL_WALL_PERIODIC, "dirichlet": HL_WALL_DIRICHLET, "neumann": HL_WALL_NEUMANN}
    vals = [names[k] if isinstance(k, str) else int(k) for k in kinds]
    if len(vals) != h.dim:
        raise ValueError("one wall kind per axis")
    _check(h, load().hl_set_walls(h.ptr, (ctypes.c_int * h.dim)(*vals)))


def hl_set_option(h: Handle, option: int, value: int) -> None:
    _check(h, load().hl_set_option(h.ptr, int(option), int(value)))


def hl_kernel_times(h: Handle):
    """Returns ({'p_half','u_half','small'}: total ms, same keys: launch counts) and resets."""
    ms = (_D * 3)()
    n = (_I64 * 3)()
    _check(h, load().hl_kernel_times(h.ptr, ms, n))
    keys = ("p_half", "u_half", "small")
    return dict(zip(keys, list(ms))), dict(zip(keys, list(n)))


def hl_operator_table(dim: int, m: int, lam) -> np.ndarray:
    """The fused operator (dim, nq, nq) indexed [i, l, s]."""
    nq = (m + 1) ** dim
    out = np.empty(dim * nq * nq, dtype=np.float64)
    lm = (_D * 3)(*([float(x) for x in lam] + [0.0] * (3 - len(lam))))
    rc = load().hl_operator_table(int(dim), int(m), lm, out.ctypes.data_as(ctypes.POINTER(_D)))
    if rc != HL_OK:
        raise HLError(rc, hl_last_error(None))
    return out.reshape(dim, nq, nq)


def hl_tc_tables(m: int, lam):
    """The tensor-core split mode's operator digits (3, 6, 16, 136) as BF16 bit patterns
    (uint16) and column exponents (3, 16)."""
    digits = np.zeros(HL_TC_TABLE_ELEMS, dtype=np.uint16)
    expo = np.zeros(HL_TC_EXPO_ELEMS, dtype=np.int32)
    lm = (_D * 2)(*[float(x) for x in lam[:2]])
    rc = load().hl_tc_tables(int(m), lm, ctypes.c_void_p(digits.ctypes.data), ctypes.c_void_p(expo.ctypes.data))
    if rc != HL_OK:
        raise HLError(rc, hl_last_error(None))
    return digits.reshape(3, 6, 16, 136), expo.reshape(3, 16)


def hl_tc_image(dim: int, m: int, lam):
    """The tensor-core kernels' operator images (FP16 bit patterns, uint16) and column
    exponents: dim 2 -> ((2, 14336), (3, 16)); dim 3 -> ((2, 12, 4, 2, 224, 8), (4, 32))."""
    n_img = HL_TC_IMAGE2_ELEMS if dim == 2 else HL_TC_IMAGE3_ELEMS
    n_ex = HL_TC_EXPO_ELEMS if dim == 2 else HL_TC_EXPO3_ELEMS
    image = np.zeros(n_img, dtype=np.uint16)
    expo = np.zeros(n_ex, dtype=np.int32)
    lm = (_D * 3)(*([float(x) for x in lam[:3]] + [0.0] * (3 - len(lam[:3]))))
    rc = load().hl_tc_image(int(dim), int(m), lm, ctypes.c_void_p(image.ctypes.data), n_img,
                            ctypes.c_void_p(expo.ctypes.data), n_ex)
    if rc != HL_OK:
        raise HLError(rc, hl_last_error(None))
    if dim == 2:
        return image.reshape(2, 14336), expo.reshape(3, 16)
    return image.reshape(2, 12, 4, 2, 224, 8), expo.reshape(4, 32)


def hl_step_noalloc(dim: int, m: int, n_cells, dt: float, p_dev, u_dev, n_steps: int, stream=None) -> int:
    """FP64 steps on caller-owned device buffers (device layout) with no device allocation.
    Returns HL_OK or HL_ENONFINITE; raises on other failures.  Both buffers must live on
    the current CUDA device (the library checks this too)."""
    if 1 <= dim <= 3 and len(n_cells) != dim:   # other dims are the C library's to reject
        raise ValueError("n_cells must hold dim entries")
    for t in (p_dev, u_dev):
        if getattr(t, "is_cuda", False):
            import torch
            if t.device.index != torch.cuda.current_device():
                raise ValueError("p_dev and u_dev must be on the current CUDA device")
    nnode = int(np.prod(n_cells))
    nq = (m + 1) ** dim
    nc = (_I64 * len(n_cells))(*[int(x) for x in n_cells])
    raw = getattr(stream, "cuda_stream", stream)
    rc = load().hl_step_noalloc(int(dim), int(m), nc, float(dt), _dev_ptr(p_dev, nnode * nq),
                                _dev_ptr(u_dev, dim * nnode * nq), int(n_steps),
                                ctypes.c_void_p(int(raw) if raw else 0))
    if rc not in (HL_OK, HL_ENONFINITE):
        raise HLError(rc, hl_last_error(None))
    return rc


def hl_op_counts(dim: int, m: int):
    f, a = _D(), _D()
    rc = load().hl_op_counts(int(dim), int(m), ctypes.byref(f), ctypes.byref(a))
    if rc != HL_OK:
        raise HLError(rc, hl_last_error(None))
    return f.value, a.value


def hl_info(h: Handle):
    nn, nq, st = _I64(), _I64(), _I64()
    _check(h, load().hl_info(h.ptr, ctypes.byref(nn), ctypes.byref(nq), ctypes.byref(st)))
    return nn.value, nq.value, st.value


# ----------------------------------------------------------------------------- learned correction
@dataclass
class MLP:
    ptr: ctypes.c_void_p


def _mcheck(m: MLP, rc: int) -> None:
    if rc != HL_OK:
        raise HLError(rc, load().hl_mlp_last_error(m.ptr if m is not None else None).decode(errors="replace"))


def _fptr(t, count: int):
    if t is None:
        return None
    if not getattr(t, "is_cuda", False) or str(t.dtype) != "torch.float32" or not t.is_contiguous() \
            or t.numel() < count:
        raise ValueError("expected a contiguous float32 CUDA tensor of sufficient size")
    return ctypes.c_void_p(t.data_ptr())


def _iptr(t, count: int):
    if t is None:
        return None
    if not getattr(t, "is_cuda", False) or str(t.dtype) != "torch.int32" or not t.is_contiguous() \
            or t.numel() < count:
        raise ValueError("expected a contiguous int32 CUDA tensor of sufficient size")
    return ctypes.c_void_p(t.data_ptr())


def hl_mlp_create(seed: int) -> MLP:
    out = _P()
    rc = load().hl_mlp_create(int(seed), ctypes.byref(out))
    if rc != HL_OK:
        raise HLError(rc, load().hl_mlp_last_error(None).decode(errors="replace"))
    return MLP(out)


def hl_mlp_destroy(m: MLP) -> None:
    if m is not None and m.ptr:
        load().hl_mlp_destroy(m.ptr)
        m.ptr = _P()


def hl_mlp_last_error(m: MLP | None) -> str:
    return load().hl_mlp_last_error(m.ptr if m is not None else None).decode(errors="replace")


def hl_mlp_set_stream(m: MLP, stream) -> None:
    raw = getattr(stream, "cuda_stream", stream)
    _mcheck(m, load().hl_mlp_set_stream(m.ptr, ctypes.c_void_p(int(raw) if raw else 0)))


def hl_mlp_params(m: MLP, set_params=None, want_grads: bool = False):
    """Returns (params, grads or None) as float32 numpy arrays; set_params replaces the weights."""
    p = np.empty(HL_MLP_NPARAMS, dtype=np.float32)
    g = np.empty(HL_MLP_NPARAMS, dtype=np.float32) if want_grads else None
    sp = None
    if set_params is not None:
        sp = np.ascontiguousarray(set_params, dtype=np.float32)
        if sp.size != HL_MLP_NPARAMS:
            raise ValueError("parameter block has the wrong size")
        sp = ctypes.c_void_p(sp.ctypes.data)
    _mcheck(m, load().hl_mlp_params(m.ptr, ctypes.c_void_p(p.ctypes.data), sp,
                                    ctypes.c_void_p(g.ctypes.data) if g is not None else None))
    return p, g


def hl_mlp_forward(m: MLP, X, rows: int, Y) -> None:
    _mcheck(m, load().hl_mlp_forward(m.ptr, _fptr(X, rows * HL_MLP_IN), int(rows), _fptr(Y, rows * HL_MLP_OUT)))


def hl_mlp_loss_grad(m: MLP, X, T, rows: int, want_loss: bool = True):
    loss = _D()
    _mcheck(m, load().hl_mlp_loss_grad(m.ptr, _fptr(X, rows * HL_MLP_IN), _fptr(T, rows * HL_MLP_OUT), int(rows),
                                       ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def hl_mlp_adam_step(m: MLP, lr: float) -> None:
    _mcheck(m, load().hl_mlp_adam_step(m.ptr, ctypes.c_float(lr)))


class _DeviceFloats:
    """A device float array exposed through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                         "strides": None}


def hl_mlp_grad_buffer(m: MLP) -> int:
    """Device address of the network's gradient (HL_MLP_NPARAMS floats, owned by the network)."""
    ptr = ctypes.c_void_p()
    _mcheck(m, load().hl_mlp_grad_buffer(m.ptr, ctypes.byref(ptr)))
    return int(ptr.value)


def hl_mlp_grad_tensor(m: MLP):
    """The network's gradient buffer as a torch tensor sharing its device memory
    (HL_MLP_NPARAMS floats; valid while the network lives): data-parallel training
    reduces it in place between hl_mlp_loss_grad and hl_mlp_adam_step."""
    import torch
    return torch.as_tensor(_DeviceFloats(hl_mlp_grad_buffer(m), HL_MLP_NPARAMS), device="cuda")


def hl_mlp_sample(m: MLP, X_pool, T_pool, rows: int, seed: int, step: int, X, T=None) -> None:
    """Device minibatch draw: X[i] = X_pool[splitmix64 index], likewise T."""
    pool = int(X_pool.shape[0])
    _mcheck(m, load().hl_mlp_sample(m.ptr, _fptr(X_pool, pool * HL_MLP_IN),
                                    None if T_pool is None else _fptr(T_pool, pool * HL_MLP_OUT), pool, int(rows),
                                    int(seed) & (2**64 - 1), int(step) & (2**64 - 1), _fptr(X, rows * HL_MLP_IN),
                                    None if T is None else _fptr(T, rows * HL_MLP_OUT)))


def hl_features(coarse: Handle, nodes, rows: int, feat_scale: float, t_feature: float, X) -> None:
    rc = load().hl_features(coarse.ptr, _iptr(nodes, rows), int(rows), ctypes.c_float(feat_scale),
                            ctypes.c_float(t_feature), _fptr(X, rows * HL_MLP_IN))
    _mcheck(None, rc)


def hl_targets(fine: Handle, ratio: int, coarse: Handle, nodes, rows: int, out_scale: float, T) -> None:
    rc = load().hl_targets(fine.ptr, int(ratio), coarse.ptr, _iptr(nodes, rows), int(rows), float(out_scale),
                           _fptr(T, rows * HL_MLP_OUT))
    _mcheck(None, rc)


def hl_set_correction(h: Handle, m, every_k_steps: int = 1, feat_scale: float = 1.0, t_feature: float = 0.0,
                      out_scale: float = 1.0, max_ratio: float = 1.0) -> None:
    """Apply the network's correction inside hl_step after every k-th step (m=None removes it);
    corrections larger than max_ratio times the last plain step's change are skipped."""
    rc = load().hl_set_correction(h.ptr, m.ptr if m is not None else None, int(every_k_steps),
                                  ctypes.c_float(feat_scale), ctypes.c_float(t_feature), float(out_scale),
                                  float(max_ratio))
    _mcheck(None, rc)


def hl_correction_stats(h: Handle):
    """Returns (applied, skipped) corrections so far."""
    a, sk = _I64(), _I64()
    _mcheck(None, load().hl_correction_stats(h.ptr, ctypes.byref(a), ctypes.byref(sk)))
    return a.value, sk.value


def hl_apply_correction(coarse: Handle, m: MLP, feat_scale: float, t_feature: float, out_scale: float) -> None:
    _mcheck(m, load().hl_apply_correction(coarse.ptr, m.ptr, ctypes.c_float(feat_scale), ctypes.c_float(t_feature),
                                          float(out_scale)))


# ----------------------------------------------------------------------------- modified scheme (1D)
@dataclass
class ModHandle:
    """Handle of the modified Hermite-leapfrog solver (both fields on both grids, 1D)."""
    ptr: ctypes.c_void_p
    m: int
    n: int
    dt: float


def _modcheck(h, rc: int) -> int:
    if rc != HL_OK:
        raise HLError(rc, load().hl_mod_last_error(h.ptr if h is not None else None).decode(errors="replace"))
    return rc


def hl_mod_create(m: int, n_cells: int, dt: float) -> ModHandle:
    out = _P()
    rc = load().hl_mod_create(int(m), int(n_cells), float(dt), ctypes.byref(out))
    if rc != HL_OK:
        raise HLError(rc, load().hl_mod_last_error(None).decode(errors="replace"))
    return ModHandle(out, int(m), int(n_cells), float(dt))


def hl_mod_destroy(h: ModHandle) -> None:
    if h is not None and h.ptr:
        load().hl_mod_destroy(h.ptr)
        h.ptr = _P()


def hl_mod_set_stream(h: ModHandle, stream) -> None:
    raw = getattr(stream, "cuda_stream", stream)
    _modcheck(h, load().hl_mod_set_stream(h.ptr, ctypes.c_void_p(int(raw) if raw else 0)))


def hl_mod_set_initial(h: ModHandle, pp, up, pd, ud) -> None:
    n = h.n * (h.m + 1)
    _modcheck(h, load().hl_mod_set_initial(h.ptr, *[_host_ptr(a, n, False) for a in (pp, up, pd, ud)]))


def hl_mod_step(h: ModHandle, n_steps: int) -> None:
    _modcheck(h, load().hl_mod_step(h.ptr, int(n_steps)))


def hl_mod_get_fields(h: ModHandle, raise_nonfinite: bool = True):
    """Returns (pp, up, pd, ud), each (n, m+1) float64."""
    outs = [np.empty((h.n, h.m + 1), dtype=np.float64) for _ in range(4)]
    rc = load().hl_mod_get_fields(h.ptr, *[_host_ptr(a, a.size, True) for a in outs])
    if rc != HL_OK and (rc != HL_ENONFINITE or raise_nonfinite):
        raise HLError(rc, load().hl_mod_last_error(h.ptr).decode(errors="replace"))
    return tuple(outs)


def hl_mod_info(h: ModHandle):
    st, tp, td = _I64(), _D(), _D()
    _modcheck(h, load().hl_mod_info(h.ptr, ctypes.byref(st), ctypes.byref(tp), ctypes.byref(td)))
    return st.value, tp.value, td.value


def hl_mod_last_error(h: ModHandle | None) -> str:
    return load().hl_mod_last_error(h.ptr if h is not None else None).decode(errors="replace")
