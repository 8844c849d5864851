"""ctypes binding of libvlbm.so: the C ABI of include/vlbm.h, same names.

Argument marshalling only.  Arrays may be torch tensors (CUDA or CPU, pinned
or not) or numpy arrays; their data pointers go to the library, which finds
out itself whether they are device or host memory.  Every computation runs in
the library's CUDA kernels; there is no Python or CPU fallback, and importing
this module fails if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvlbm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python paper_2607_24059_b300/build.py, or __graft_entry__.build())")

lib = ctypes.CDLL(LIB_PATH)

# ---- constants (include/vlbm.h) ------------------------------------------------
VLBM_OK = 0
VLBM_WSTABILITY = 1
VLBM_EINVAL = -1
VLBM_ESTABILITY = -2
VLBM_ENOMEM = -3
VLBM_ECUDA = -4
VLBM_EDIVERGED = -5
VLBM_ETIMEOUT = -6
VLBM_EUNSUPPORTED = -7

VLBM_FP64 = 0
VLBM_FP32 = 1
VLBM_FP16_SHIFTED = 2
VLBM_BF16_SHIFTED = 3
VLBM_FP16_SPLIT = 4
VLBM_BF16_SPLIT = 5

VLBM_DTYPE_F32 = 0
VLBM_DTYPE_F64 = 1

VLBM_STEP_CHECK_FINITE = 1
VLBM_STEP_NO_GRAPH = 2
VLBM_STEP_PERSISTENT = 4
VLBM_STEP_TEST_TIMEOUT = 8

VLBM_NUM_INVARIANTS = 8
VLBM_OPT_KERNEL = 0
VLBM_OPT_SPLIT_LANES = 1
VLBM_OPT_ROUNDING_16 = 2

VLBM_BC_PERIODIC = 0
VLBM_BC_CHANNEL = 1

PRECISIONS = {"fp64": VLBM_FP64, "fp32": VLBM_FP32, "fp16": VLBM_FP16_SHIFTED, "bf16": VLBM_BF16_SHIFTED,
              "fp16split": VLBM_FP16_SPLIT, "bf16split": VLBM_BF16_SPLIT}

EXPORTED = [
    "vlbm_params_default", "vlbm_params_check", "vlbm_create", "vlbm_destroy", "vlbm_set_stream",
    "vlbm_init", "vlbm_step", "vlbm_step_record", "vlbm_macros", "vlbm_invariants", "vlbm_time", "vlbm_state_bytes",
    "vlbm_get_state", "vlbm_set_state", "vlbm_get_populations", "vlbm_launch_count", "vlbm_set_option",
    "vlbm_strerror", "vlbm_last_error", "vlbm_invariants_noalloc", "vlbm_vorticity_sq", "vlbm_set_boundary",
    "vlbm_batch_create", "vlbm_batch_destroy", "vlbm_batch_init", "vlbm_batch_step", "vlbm_batch_macros",
    "vlbm_batch_invariants", "vlbm_batch_set_config", "vlbm_batch_autotune", "vlbm_batch_info",
    "vlbm_batch_last_error", "vlbm_batch_init_states", "vlbm_batch_macros_states", "vlbm_tc_gemm_bf16", "vlbm_sur_conv3x3", "vlbm_sur_conv3x3_wgrad",
    "vlbm_sur_create", "vlbm_sur_destroy", "vlbm_sur_num_params", "vlbm_sur_forward", "vlbm_sur_train_step",
    "vlbm_sur_get_params", "vlbm_sur_get_grads", "vlbm_sur_set_params", "vlbm_sur_status", "vlbm_sur_advance",
    "vlbm_sur_set_scaling", "vlbm_sur_set_train_noise", "vlbm_sur_launch_count", "vlbm_sur_increment",
    "vlbm_field_pool", "vlbm_sur_gather_pairs", "vlbm_field_stats", "vlbm_sur_rollout_check", "vlbm_field_diff_norms",
]


class vlbm_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("precision", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
        ("dx", ctypes.c_double), ("mu", ctypes.c_double), ("nu", ctypes.c_double),
        ("omega", ctypes.c_double * 4), ("alpha", ctypes.c_double * 4),
        ("gamma", ctypes.c_double), ("rho_bar", ctypes.c_double),
        ("strict", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class vlbm_derived(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("alpha", ctypes.c_double * 4), ("viscosity", ctypes.c_double * 4),
        ("mu_min", ctypes.c_double), ("nodes", ctypes.c_int64), ("populations_per_node", ctypes.c_int32),
        ("bytes_per_population", ctypes.c_int32), ("lattice_bytes", ctypes.c_size_t),
    ]


class vlbm_boundary(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("wall_correction", ctypes.c_int32), ("phi_out", ctypes.c_double),
        ("u_in", ctypes.POINTER(ctypes.c_double)),
    ]


_P = ctypes.POINTER(vlbm_params)
_H = ctypes.c_void_p
_V = ctypes.c_void_p

lib.vlbm_params_default.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int32]
lib.vlbm_params_default.restype = None
lib.vlbm_params_check.argtypes = [_P, ctypes.POINTER(vlbm_derived)]
lib.vlbm_create.argtypes = [_P, _V, ctypes.POINTER(_H)]
lib.vlbm_destroy.argtypes = [_H]
lib.vlbm_destroy.restype = None
lib.vlbm_set_stream.argtypes = [_H, _V]
lib.vlbm_init.argtypes = [_H, _V, _V, ctypes.c_int32]
lib.vlbm_step.argtypes = [_H, ctypes.c_int64, ctypes.c_int32]
lib.vlbm_step_record.argtypes = [_H, ctypes.c_int64, ctypes.c_int64, _V]
lib.vlbm_macros.argtypes = [_H, _V, _V, _V, ctypes.c_int32]
lib.vlbm_invariants.argtypes = [_H, _V]
lib.vlbm_vorticity_sq.argtypes = [_H, _V]
lib.vlbm_time.argtypes = [_H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
lib.vlbm_state_bytes.argtypes = [_H]
lib.vlbm_state_bytes.restype = ctypes.c_size_t
lib.vlbm_get_state.argtypes = [_H, _V, ctypes.c_size_t]
lib.vlbm_set_state.argtypes = [_H, _V, ctypes.c_size_t]
lib.vlbm_get_populations.argtypes = [_H, _V, ctypes.c_int32, ctypes.c_int32]
lib.vlbm_launch_count.argtypes = [_H, ctypes.POINTER(ctypes.c_int64)]
lib.vlbm_set_option.argtypes = [_H, ctypes.c_int32, ctypes.c_int64]
lib.vlbm_set_boundary.argtypes = [_H, ctypes.POINTER(vlbm_boundary)]
lib.vlbm_invariants_noalloc.argtypes = [_P, _V, _V, _V]
lib.vlbm_batch_create.argtypes = [_P, ctypes.c_int32, _V, ctypes.POINTER(_H)]
lib.vlbm_batch_destroy.argtypes = [_H]
lib.vlbm_batch_destroy.restype = None
lib.vlbm_batch_init.argtypes = [_H, ctypes.c_int32, _V, _V, ctypes.c_int32]
lib.vlbm_batch_step.argtypes = [_H, ctypes.c_int64, ctypes.c_int32]
lib.vlbm_batch_macros.argtypes = [_H, ctypes.c_int32, _V, _V, _V, ctypes.c_int32]
lib.vlbm_batch_invariants.argtypes = [_H, ctypes.c_int32, _V]
lib.vlbm_batch_set_config.argtypes = [_H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
lib.vlbm_batch_autotune.argtypes = [_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
lib.vlbm_batch_info.argtypes = [_H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int64)]
lib.vlbm_batch_init_states.argtypes = [_H, _V, ctypes.c_int32, _V]
lib.vlbm_batch_macros_states.argtypes = [_H, _V, ctypes.c_int32, _V]
lib.vlbm_batch_last_error.argtypes = [_H]
lib.vlbm_batch_last_error.restype = ctypes.c_char_p
lib.vlbm_tc_gemm_bf16.argtypes = [_V, _V, _V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _V, _V]
lib.vlbm_sur_conv3x3.argtypes = [_V, _V, _V, _V, _V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_int32, _V, _V]
lib.vlbm_sur_conv3x3_wgrad.argtypes = [_V, _V, _V, _V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int32, _V, _V]
lib.vlbm_sur_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_uint64, _V, ctypes.POINTER(_H)]
lib.vlbm_sur_set_scaling.argtypes = [_H, _V, _V]
lib.vlbm_sur_set_train_noise.argtypes = [_H, _V, ctypes.c_uint64]
lib.vlbm_sur_launch_count.argtypes = []
lib.vlbm_sur_launch_count.restype = ctypes.c_int64
lib.vlbm_sur_destroy.argtypes = [_H]
lib.vlbm_sur_destroy.restype = None
lib.vlbm_sur_num_params.argtypes = [_H]
lib.vlbm_sur_num_params.restype = ctypes.c_int64
lib.vlbm_sur_forward.argtypes = [_H, _V, _V, ctypes.c_int32]
lib.vlbm_sur_train_step.argtypes = [_H, _V, _V, ctypes.c_int32, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]
lib.vlbm_sur_get_params.argtypes = [_H, _V]
lib.vlbm_sur_get_grads.argtypes = [_H, _V]
lib.vlbm_sur_set_params.argtypes = [_H, _V]
lib.vlbm_sur_status.argtypes = [_H]
lib.vlbm_sur_advance.argtypes = [_H, _V, _V, ctypes.c_int32]
lib.vlbm_sur_increment.argtypes = [_H, _V, _V, ctypes.c_int32]
lib.vlbm_field_pool.argtypes = [_V, _V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                _V]
lib.vlbm_sur_gather_pairs.argtypes = [_V, _V, _V, _V, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                      _V, _V]
lib.vlbm_field_stats.argtypes = [_V, _V, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _V]
lib.vlbm_sur_rollout_check.argtypes = [_V, _V, _V, _V, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _V, _V, _V]
lib.vlbm_field_diff_norms.argtypes = [_V, _V, _V, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _V]
lib.vlbm_strerror.argtypes = [ctypes.c_int]
lib.vlbm_strerror.restype = ctypes.c_char_p
lib.vlbm_last_error.argtypes = [_H]
lib.vlbm_last_error.restype = ctypes.c_char_p


class VlbmError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {lib.vlbm_strerror(code).decode()} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def _check(code: int, where: str, h=None) -> int:
    if code < 0:
        detail = lib.vlbm_last_error(h).decode() if h else ""
        raise VlbmError(code, where, detail)
    if code > 0:
        warnings.warn(f"{where}: {lib.vlbm_strerror(code).decode()}", RuntimeWarning, stacklevel=3)
    return code


# ---- marshalling helpers ----------------------------------------------------------
def _ptr_dtype(a):
    """(pointer, VLBM_DTYPE) of a contiguous float32/float64 torch tensor or numpy array."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        if a.dtype == np.float64:
            return a.ctypes.data, VLBM_DTYPE_F64
        if a.dtype == np.float32:
            return a.ctypes.data, VLBM_DTYPE_F32
        raise TypeError(f"unsupported dtype {a.dtype}")
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError(f"expected a torch tensor or numpy array, got {type(a)}")
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if a.dtype == torch.float64:
        return a.data_ptr(), VLBM_DTYPE_F64
    if a.dtype == torch.float32:
        return a.data_ptr(), VLBM_DTYPE_F32
    raise TypeError(f"unsupported dtype {a.dtype}")


def current_stream():
    """The torch current CUDA stream handle (0 when CUDA is unavailable)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


# ---- the C ABI, same names ------------------------------------------------------------
def vlbm_params_default(dim, n, dx, nu, precision=VLBM_FP32) -> vlbm_params:
    p = vlbm_params()
    arr = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    lib.vlbm_params_default(ctypes.byref(p), int(dim), arr, float(dx), float(nu), int(precision))
    return p


def vlbm_params_check(p: vlbm_params):
    """Returns (status, vlbm_derived); raises on an error status."""
    d = vlbm_derived()
    rc = lib.vlbm_params_check(ctypes.byref(p), ctypes.byref(d))
    _check(rc, "vlbm_params_check")
    return rc, d


def vlbm_create(p: vlbm_params, stream=None):
    h = _H()
    s = current_stream() if stream is None else stream
    rc = lib.vlbm_create(ctypes.byref(p), _V(s), ctypes.byref(h))
    _check(rc, "vlbm_create")
    return h


def vlbm_destroy(h) -> None:
    lib.vlbm_destroy(h)


def vlbm_set_stream(h, stream) -> None:
    _check(lib.vlbm_set_stream(h, _V(stream)), "vlbm_set_stream", h)


def vlbm_init(h, u, phi=None) -> None:
    up, dt = _ptr_dtype(u)
    pp, dt2 = _ptr_dtype(phi)
    if dt2 is not None and dt2 != dt:
        raise TypeError("u and phi must have the same dtype")
    _check(lib.vlbm_init(h, _V(up), _V(pp), dt), "vlbm_init", h)


def vlbm_step(h, nsteps: int, flags: int = 0) -> None:
    _check(lib.vlbm_step(h, int(nsteps), int(flags)), "vlbm_step", h)


def vlbm_step_record(h, nsteps: int, every: int, history=None):
    """Step with fused invariant records; returns `history` (8 float64 per record)."""
    if history is None:
        history = np.zeros(((int(nsteps) + int(every) - 1) // int(every), VLBM_NUM_INVARIANTS), dtype=np.float64)
    p, dt = _ptr_dtype(history)
    if dt != VLBM_DTYPE_F64:
        raise TypeError("records are float64")
    _check(lib.vlbm_step_record(h, int(nsteps), int(every), _V(p)), "vlbm_step_record", h)
    return history


def vlbm_macros(h, rho=None, u=None, phi=None) -> None:
    dts = {d for d in (_ptr_dtype(a)[1] for a in (rho, u, phi)) if d is not None}
    if len(dts) != 1:
        raise TypeError("give at least one output, all of one dtype")
    _check(lib.vlbm_macros(h, _V(_ptr_dtype(rho)[0]), _V(_ptr_dtype(u)[0]), _V(_ptr_dtype(phi)[0]), dts.pop()),
           "vlbm_macros", h)


def vlbm_invariants(h, out=None):
    """Fills `out` (8 float64, host or device) or returns a numpy array."""
    if out is None:
        out = np.zeros(VLBM_NUM_INVARIANTS, dtype=np.float64)
    p, dt = _ptr_dtype(out)
    if dt != VLBM_DTYPE_F64:
        raise TypeError("invariants are float64")
    _check(lib.vlbm_invariants(h, _V(p)), "vlbm_invariants", h)
    return out


def vlbm_vorticity_sq(h, out=None):
    """Sum over nodes of |curl u|^2 dx^d (centred differences); `out` = 1 float64 (host or
    device), else returns a float."""
    if out is None:
        buf = np.zeros(1, dtype=np.float64)
        _check(lib.vlbm_vorticity_sq(h, _V(buf.ctypes.data)), "vlbm_vorticity_sq", h)
        return float(buf[0])
    p, dt = _ptr_dtype(out)
    if dt != VLBM_DTYPE_F64:
        raise TypeError("the vorticity sum is float64")
    _check(lib.vlbm_vorticity_sq(h, _V(p)), "vlbm_vorticity_sq", h)
    return out


def vlbm_time(h):
    s = ctypes.c_int64()
    t = ctypes.c_double()
    _check(lib.vlbm_time(h, ctypes.byref(s), ctypes.byref(t)), "vlbm_time", h)
    return s.value, t.value


def vlbm_state_bytes(h) -> int:
    return int(lib.vlbm_state_bytes(h))


def vlbm_get_state(h, dst=None):
    if dst is None:
        dst = np.empty(vlbm_state_bytes(h), dtype=np.uint8)
    ptr = dst.ctypes.data if isinstance(dst, np.ndarray) else dst.data_ptr()
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(lib.vlbm_get_state(h, _V(ptr), nbytes), "vlbm_get_state", h)
    return dst


def vlbm_set_state(h, src) -> None:
    ptr = src.ctypes.data if isinstance(src, np.ndarray) else src.data_ptr()
    nbytes = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
    _check(lib.vlbm_set_state(h, _V(ptr), nbytes), "vlbm_set_state", h)


def vlbm_get_populations(h, dst, deviation: bool = False) -> None:
    p, dt = _ptr_dtype(dst)
    _check(lib.vlbm_get_populations(h, _V(p), dt, int(bool(deviation))), "vlbm_get_populations", h)


def vlbm_launch_count(h) -> int:
    c = ctypes.c_int64()
    _check(lib.vlbm_launch_count(h, ctypes.byref(c)), "vlbm_launch_count", h)
    return c.value


def vlbm_set_option(h, key: int, value: int) -> None:
    _check(lib.vlbm_set_option(h, int(key), int(value)), "vlbm_set_option", h)


def vlbm_set_boundary(h, kind: int, u_in=None, phi_out: float = 0.0, wall_correction: bool = False) -> None:
    """kind VLBM_BC_PERIODIC or VLBM_BC_CHANNEL; u_in: the n_y inflow velocities (host, FP64)."""
    b = vlbm_boundary()
    b.kind = int(kind)
    b.wall_correction = 1 if wall_correction else 0
    b.phi_out = float(phi_out)
    keep = None
    if u_in is not None:
        keep = np.ascontiguousarray(u_in, dtype=np.float64)
        b.u_in = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib.vlbm_set_boundary(h, ctypes.byref(b)), "vlbm_set_boundary", h)


def vlbm_invariants_noalloc(p: vlbm_params, lattice, out, stream=None) -> None:
    """Invariants of a caller-owned device lattice; the library allocates nothing.

    lattice: CUDA tensor (or raw device address) holding one population lattice
    in a handle's storage layout; out: 8 float64, device or host.
    """
    lp = lattice if isinstance(lattice, int) else lattice.data_ptr()
    op, dt = _ptr_dtype(out)
    if dt != VLBM_DTYPE_F64:
        raise TypeError("invariants are float64")
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_invariants_noalloc(ctypes.byref(p), _V(lp), _V(op), _V(s)), "vlbm_invariants_noalloc")


# ---- batched problems
def _bcheck(code, where, b):
    if code < 0:
        raise VlbmError(code, where, lib.vlbm_batch_last_error(b).decode() if b else "")
    return code


def vlbm_batch_create(problems, stream=None):
    """problems: sequence of vlbm_params (dim 2, one precision)."""
    arr = (vlbm_params * len(problems))(*problems)
    b = _H()
    s = current_stream() if stream is None else stream
    _bcheck(lib.vlbm_batch_create(arr, len(problems), _V(s), ctypes.byref(b)), "vlbm_batch_create", None)
    return b


def vlbm_batch_destroy(b) -> None:
    lib.vlbm_batch_destroy(b)


def vlbm_batch_init(b, problem: int, u, phi=None) -> None:
    up, dt = _ptr_dtype(u)
    pp, _ = _ptr_dtype(phi)
    _bcheck(lib.vlbm_batch_init(b, int(problem), _V(up), _V(pp), dt), "vlbm_batch_init", b)


def vlbm_batch_step(b, nsteps: int, flags: int = 0) -> None:
    _bcheck(lib.vlbm_batch_step(b, int(nsteps), int(flags)), "vlbm_batch_step", b)


def vlbm_batch_macros(b, problem: int, rho=None, u=None, phi=None) -> None:
    dts = {d for d in (_ptr_dtype(a)[1] for a in (rho, u, phi)) if d is not None}
    if len(dts) != 1:
        raise TypeError("give at least one output, all of one dtype")
    _bcheck(lib.vlbm_batch_macros(b, int(problem), _V(_ptr_dtype(rho)[0]), _V(_ptr_dtype(u)[0]),
                                  _V(_ptr_dtype(phi)[0]), dts.pop()), "vlbm_batch_macros", b)


def vlbm_batch_invariants(b, problem: int, out=None):
    if out is None:
        out = np.zeros(VLBM_NUM_INVARIANTS, dtype=np.float64)
    p, _ = _ptr_dtype(out)
    _bcheck(lib.vlbm_batch_invariants(b, int(problem), _V(p)), "vlbm_batch_invariants", b)
    return out


def vlbm_batch_set_config(b, threads: int, blocks_per_sm: int, lanes: int = 4) -> None:
    _bcheck(lib.vlbm_batch_set_config(b, threads, blocks_per_sm, lanes), "vlbm_batch_set_config", b)


def vlbm_batch_autotune(b, repeats: int = 5):
    """Returns ((threads, blocks_per_sm, lanes), ms_per_step)."""
    cfg = (ctypes.c_int32 * 3)()
    ms = ctypes.c_double()
    _bcheck(lib.vlbm_batch_autotune(b, int(repeats), cfg, ctypes.byref(ms)), "vlbm_batch_autotune", b)
    return tuple(cfg), ms.value


def vlbm_batch_info(b):
    n, s, l = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _bcheck(lib.vlbm_batch_info(b, ctypes.byref(n), ctypes.byref(s), ctypes.byref(l)), "vlbm_batch_info", b)
    return n.value, s.value, l.value


def vlbm_batch_init_states(b, states, mask) -> None:
    """Masked init of equal problems from states (count, C, ny, nx) fp32 and mask (count,) uint8, on the device."""
    _check(lib.vlbm_batch_init_states(b, _V(states.data_ptr()), states.shape[1], _V(mask.data_ptr())),
           "vlbm_batch_init_states")


def vlbm_batch_macros_states(b, states, mask) -> None:
    """Masked read-out of u (and phi) of equal problems into states (count, C, ny, nx) fp32."""
    _check(lib.vlbm_batch_macros_states(b, _V(states.data_ptr()), states.shape[1], _V(mask.data_ptr())),
           "vlbm_batch_macros_states")


def vlbm_batch_last_error(b) -> str:
    return lib.vlbm_batch_last_error(b).decode()


def vlbm_tc_gemm_bf16(A, B, D, err, stream=None) -> None:
    """D = A B^T on tcgen05 tensor cores; CUDA tensors: A (M, K) bf16, B (N, K) bf16, D (M, N) fp32,
    err: one int32 set to 1 if a wait for the tensor core gave up."""
    M, K = A.shape
    N = B.shape[0]
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_tc_gemm_bf16(_V(A.data_ptr()), _V(B.data_ptr()), _V(D.data_ptr()), M, N, K,
                                 _V(err.data_ptr()), _V(s)), "vlbm_tc_gemm_bf16")


def vlbm_sur_conv3x3(X, W, bias, Y, err, act=True, Z=None, stream=None) -> None:
    """Periodic 3x3 convolution on tcgen05: X (B, H, W, cin) bf16, W (cout, 9, cin) bf16, bias (cout,) fp32,
    Y (and Z) (B, H, W, cout) bf16, err one int32 on the device."""
    B, H, Wd, cin = X.shape
    cout = W.shape[0]
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_sur_conv3x3(_V(X.data_ptr()), _V(W.data_ptr()), _V(bias.data_ptr()), _V(Y.data_ptr()),
                                _V(Z.data_ptr() if Z is not None else None), B, H, Wd, cin, cout, int(bool(act)),
                                _V(err.data_ptr()), _V(s)), "vlbm_sur_conv3x3")


def vlbm_sur_conv3x3_wgrad(X, dZ, G, Gb, err, stream=None) -> None:
    """Accumulate weight (G (cout, 9, cin) fp32) and bias (Gb (cout,) fp32) gradients of vlbm_sur_conv3x3
    from X (B, H, W, cin) bf16 and dZ (B, H, W, cout) bf16."""
    B, H, Wd, cin = X.shape
    cout = dZ.shape[3]
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_sur_conv3x3_wgrad(_V(X.data_ptr()), _V(dZ.data_ptr()), _V(G.data_ptr()), _V(Gb.data_ptr()),
                                      B, H, Wd, cin, cout, _V(err.data_ptr()), _V(s)), "vlbm_sur_conv3x3_wgrad")


VLBM_SUR_FEATURE_DIV = 1
VLBM_SUR_FEATURE_CURL = 2


def vlbm_sur_create(H: int, W: int, channels: int, features: int, max_batch: int, seed: int, stream=None):
    h = _H()
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_sur_create(H, W, channels, features, max_batch, seed, _V(s), ctypes.byref(h)), "vlbm_sur_create")
    return h


def _float_array(vals):
    if vals is None:
        return None
    vals = [float(x) for x in vals]
    return (ctypes.c_float * len(vals))(*vals)


def vlbm_sur_set_scaling(h, in_scale=None, out_scale=None) -> None:
    """Per-channel input and output factors (sequences of floats; None = 1)."""
    _check(lib.vlbm_sur_set_scaling(h, _float_array(in_scale), _float_array(out_scale)), "vlbm_sur_set_scaling")


def vlbm_sur_destroy(h) -> None:
    lib.vlbm_sur_destroy(h)


def vlbm_sur_set_train_noise(h, sigma=None, seed: int = 0) -> None:
    """Per-input-channel standard deviation of the training-input noise (None = off)."""
    _check(lib.vlbm_sur_set_train_noise(h, _float_array(sigma), int(seed)), "vlbm_sur_set_train_noise")


def vlbm_sur_launch_count() -> int:
    return int(lib.vlbm_sur_launch_count())


def vlbm_sur_num_params(h) -> int:
    return int(lib.vlbm_sur_num_params(h))


def vlbm_sur_forward(h, u, du, batch: int) -> None:
    _check(lib.vlbm_sur_forward(h, _V(u.data_ptr()), _V(du.data_ptr()), batch), "vlbm_sur_forward")


def vlbm_sur_train_step(h, u, target, batch: int, lr: float, want_loss: bool = True):
    loss = ctypes.c_float(0.0)
    _check(lib.vlbm_sur_train_step(h, _V(u.data_ptr()), _V(target.data_ptr()), batch, lr,
                                   ctypes.byref(loss) if want_loss else None), "vlbm_sur_train_step")
    return float(loss.value) if want_loss else None


def vlbm_sur_get_params(h, dst) -> None:
    _check(lib.vlbm_sur_get_params(h, _V(dst.data_ptr())), "vlbm_sur_get_params")


def vlbm_sur_get_grads(h, dst) -> None:
    _check(lib.vlbm_sur_get_grads(h, _V(dst.data_ptr())), "vlbm_sur_get_grads")


def vlbm_sur_set_params(h, src) -> None:
    _check(lib.vlbm_sur_set_params(h, _V(src.data_ptr())), "vlbm_sur_set_params")


def vlbm_sur_status(h) -> None:
    _check(lib.vlbm_sur_status(h), "vlbm_sur_status")


def vlbm_sur_advance(h, u, u_next, batch: int) -> None:
    _check(lib.vlbm_sur_advance(h, _V(u.data_ptr()), _V(u_next.data_ptr()), batch), "vlbm_sur_advance")


def vlbm_sur_increment(h, u, du, batch: int) -> None:
    _check(lib.vlbm_sur_increment(h, _V(u.data_ptr()), _V(du.data_ptr()), batch), "vlbm_sur_increment")


def vlbm_field_pool(x, out, factor: int, stream=None) -> None:
    """Average-pool x (B, C, H f, W f) fp32 into out (B, C, H, W) fp32 on the device."""
    B, C, H, W = out.shape
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_field_pool(_V(x.data_ptr()), _V(out.data_ptr()), B, C, H, W, factor, _V(s)), "vlbm_field_pool")


def vlbm_sur_gather_pairs(snaps, idx, u, target, inv_scale, stream=None) -> None:
    """u[b] = snaps[idx[b]], target[b][c] = (snaps[idx[b]+1][c] - snaps[idx[b]][c]) * inv_scale[c]
    (device arrays; inv_scale a sequence of C floats or one float for every channel)."""
    B, C, H, W = u.shape
    if isinstance(inv_scale, (int, float)):
        inv_scale = [inv_scale] * C
    if len(inv_scale) != C:
        raise ValueError("one inverse scale per channel")
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_sur_gather_pairs(_V(snaps.data_ptr()), _V(idx.data_ptr()), _V(u.data_ptr()),
                                     _V(target.data_ptr()), C, H, W, B, _float_array(inv_scale), _V(s)),
           "vlbm_sur_gather_pairs")


def vlbm_field_stats(u, out, stream=None) -> None:
    """out (B, 3) fp64 = per-state energy, squared divergence and squared gradient sums of the
    velocity channels 0, 1 of u (B, C, H, W)."""
    B, C, H, W = u.shape
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_field_stats(_V(u.data_ptr()), _V(out.data_ptr()), B, C, H, W, _V(s)), "vlbm_field_stats")


def vlbm_sur_rollout_check(stats, prev, e0, r_max, step_tol, drift_tol, mask, counts, stream=None) -> None:
    """Per-state rollout check on the device: stats, prev (n, 3) fp64; e0, r_max (n,) fp64;
    mask (n,) uint8 out; counts (n + 3,) int64 accumulated (per-state failures, then the failing
    energy-step, energy-drift and divergence tests)."""
    n = stats.shape[0]
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_sur_rollout_check(_V(stats.data_ptr()), _V(prev.data_ptr()), _V(e0.data_ptr()),
                                      _V(r_max.data_ptr()), n, float(step_tol), float(drift_tol),
                                      _V(mask.data_ptr()), _V(counts.data_ptr()), _V(s)), "vlbm_sur_rollout_check")


def vlbm_field_diff_norms(a, b, out, n=None, stream=None) -> None:
    """out (F, 2) fp64 = per-field sum (a - b)^2 and sum b^2 over the first n values (default: all)
    of each field of a, b (F, ...) fp32 on the device."""
    F = a.shape[0]
    ld = a.numel() // F
    s = current_stream() if stream is None else stream
    _check(lib.vlbm_field_diff_norms(_V(a.data_ptr()), _V(b.data_ptr()), _V(out.data_ptr()), F,
                                     ld if n is None else int(n), ld, _V(s)), "vlbm_field_diff_norms")


def vlbm_strerror(code: int) -> str:
    return lib.vlbm_strerror(int(code)).decode()


def vlbm_last_error(h) -> str:
    return lib.vlbm_last_error(h).decode()
