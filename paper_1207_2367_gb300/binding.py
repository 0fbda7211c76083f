"""Thin ctypes binding of libhgpu.so with the C ABI's names (include/hg.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Array arguments may be numpy arrays (host) or torch tensors (host or
CUDA, contiguous, float64 / int32); None passes NULL.  Functions raise HGError
on a non-zero status.  There is no CPU fallback: load() raises if the library
cannot be built or loaded.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

HG_OK, HG_EINVAL, HG_ENOMEM, HG_ECUDA, HG_ESTATE, HG_ETIMEOUT = range(6)
HG_FP64, HG_MIXED = 0, 1
HG_FAULT_NONE, HG_FAULT_ALLOC, HG_FAULT_CUDA = 0, 1, 2
_NAMES = {1: "HG_EINVAL", 2: "HG_ENOMEM", 3: "HG_ECUDA", 4: "HG_ESTATE", 5: "HG_ETIMEOUT"}


class HGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class hg_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("energy_precision", C.c_int32), ("device", C.c_int32),
                ("tpi", C.c_int32), ("jsplit", C.c_int32), ("graph_steps", C.c_int32),
                ("start_mode", C.c_int32), ("profile", C.c_int32),
                ("test_stall_eval", C.c_int32), ("order", C.c_int32),
                ("dt_min", C.c_double), ("dt_max", C.c_double), ("eta_init", C.c_double),
                ("stream", C.c_void_p)]


class hg_state(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in ("mass", "pos", "vel", "acc", "jerk", "snap", "crackle", "t", "dt")] + [
        ("t_sys", C.c_double)]


class hg_stats(C.Structure):
    _fields_ = [("block_steps", C.c_int64), ("interactions", C.c_int64), ("last_m", C.c_int64),
                ("t_sys", C.c_double), ("kernels", C.c_int64)]


class hg_profile(C.Structure):
    _fields_ = [("ms", C.c_double * 5), ("block_steps", C.c_int64)]


class hg_tune_entry(C.Structure):
    _fields_ = [("m", C.c_int64), ("bucket", C.c_int32), ("candidates", C.c_int32), ("model", C.c_int32),
                ("chosen", C.c_int32), ("model_us", C.c_double), ("best_us", C.c_double)]


HG_TUNE_BUCKETS = 32
SECTIONS = ("next", "predict", "evaluate", "reduce", "correct")


STATE_FIELDS = ("mass", "pos", "vel", "acc", "jerk", "snap", "crackle", "t", "dt")

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Build (if needed) and load the CUDA library; raises on failure.  The
    environment variable HG_LIB_VARIANT=checked selects the checked build
    (device bounds checks that report instead of faulting)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.build(checked=os.environ.get("HG_LIB_VARIANT", "") == "checked")
        L = C.CDLL(path)
        P, I64, D, I32P = C.c_void_p, C.c_int64, C.c_double, C.c_void_p
        L.hg_default_opts.argtypes = [C.POINTER(hg_opts)]
        L.hg_default_opts.restype = None
        L.hg_init.argtypes = [C.POINTER(P), I64, P, P, P, D, D, C.POINTER(hg_opts)]
        L.hg_init_batch.argtypes = [C.POINTER(P), C.c_int32, P, I64, P, P, P, D, D, C.POINTER(hg_opts)]
        L.hg_init_batch.restype = C.c_int
        L.hg_next_block.argtypes = [P, C.POINTER(D), I32P, I64, C.POINTER(I64)]
        L.hg_predict.argtypes = [P, D]
        L.hg_evaluate.argtypes = [P, I32P, I64, P, P, P]
        L.hg_correct.argtypes = [P, I32P, I64]
        L.hg_step.argtypes = [P, I64]
        L.hg_advance.argtypes = [P, D, C.POINTER(I64)]
        L.hg_energy.argtypes = [P, C.POINTER(D), C.POINTER(D)]
        L.hg_get_state.argtypes = [P, C.POINTER(hg_state)]
        L.hg_set_state.argtypes = [P, C.POINTER(hg_state)]
        L.hg_get_stats.argtypes = [P, C.POINTER(hg_stats)]
        L.hg_get_profile.argtypes = [P, C.POINTER(hg_profile), C.c_int]
        L.hg_size.argtypes = [P]
        L.hg_size.restype = I64
        L.hg_last_error.argtypes = [P]
        L.hg_last_error.restype = C.c_char_p
        L.hg_init_error.argtypes = []
        L.hg_init_error.restype = C.c_char_p
        L.hg_free.argtypes = [P]
        L.hg_free.restype = None
        L.hg_evaluate_static.argtypes = [I64, P, P, P, P, D, C.c_int32, I32P, I64, P, P, P, P]
        L.hg_evaluate_static.restype = C.c_int
        L.hg_peak_flops.argtypes = [C.c_int32, C.c_int32, P, C.POINTER(D), C.POINTER(D)]
        L.hg_peak_flops.restype = C.c_int
        L.hg_angular_momentum.argtypes = [P, C.POINTER(D)]
        L.hg_bind_device.argtypes = [P, C.c_void_p, C.c_int]
        L.hg_tune.argtypes = [P, I64, C.c_int32, C.POINTER(hg_tune_entry), C.c_int32, C.POINTER(C.c_int32)]
        L.hg_time_evaluate.argtypes = [P, I32P, I64, C.c_int32, C.POINTER(D)]
        L.hg_condition_scale.argtypes = [P, P, I64]
        L.hg_build_checked.argtypes = []
        L.hg_build_checked.restype = C.c_int
        L.hg_test_corrupt_list.argtypes = [P, I64, C.c_int32]
        L.hg_test_corrupt_list.restype = C.c_int
        L.hg_inject_fault.argtypes = [C.c_int32, I64]
        L.hg_inject_fault.restype = C.c_int
        L.hg_get_tuning.argtypes = [P, C.POINTER(C.c_int16)]
        L.hg_set_tuning.argtypes = [P, C.POINTER(C.c_int16)]
        for name in ("hg_init", "hg_next_block", "hg_predict", "hg_evaluate", "hg_correct", "hg_step",
                     "hg_advance", "hg_energy", "hg_get_state", "hg_set_state", "hg_get_stats", "hg_get_profile",
                     "hg_tune", "hg_time_evaluate", "hg_condition_scale", "hg_get_tuning", "hg_set_tuning", "hg_angular_momentum", "hg_bind_device"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _ptr(a, dtype=np.float64):
    """Raw address of a numpy array or torch tensor (contiguous, dtype checked); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        want = torch.float64 if dtype == np.float64 else torch.int32
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, rc):
    if rc != HG_OK:
        raise HGError(rc, load().hg_last_error(ctx).decode())


def hg_default_opts(**kw) -> hg_opts:
    o = hg_opts()
    load().hg_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "stream":
            v = getattr(v, "cuda_stream", v)
        setattr(o, k, v)
    return o


def hg_init(mass, pos, vel, eps, eta, opts: hg_opts | None = None):
    """Returns a context handle (int)."""
    n = int(mass.shape[0])
    ctx = C.c_void_p()
    rc = load().hg_init(C.byref(ctx), n, _ptr(mass), _ptr(pos), _ptr(vel), float(eps), float(eta),
                        C.byref(opts) if opts is not None else None)
    if rc != HG_OK:
        raise HGError(rc, load().hg_init_error().decode())
    return ctx.value


def hg_init_batch(offsets, mass, pos, vel, eps, eta, opts: hg_opts | None = None):
    """Context of independent clusters; offsets: int64 [n_clusters + 1]."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = int(mass.shape[0])
    ctx = C.c_void_p()
    rc = load().hg_init_batch(C.byref(ctx), int(offsets.shape[0] - 1), offsets.ctypes.data, n, _ptr(mass),
                              _ptr(pos), _ptr(vel), float(eps), float(eta),
                              C.byref(opts) if opts is not None else None)
    if rc != HG_OK:
        raise HGError(rc, load().hg_init_error().decode())
    return ctx.value


def hg_next_block(ctx, idx=None):
    """(t_next, m); fills idx (capacity len(idx)) when given."""
    t = C.c_double()
    m = C.c_int64()
    cap = 0 if idx is None else int(idx.shape[0])
    _check(ctx, load().hg_next_block(ctx, C.byref(t), _ptr(idx, np.int32), cap, C.byref(m)))
    return t.value, m.value


def hg_predict(ctx, t):
    _check(ctx, load().hg_predict(ctx, float(t)))


def hg_evaluate(ctx, idx, m, acc=None, jerk=None, snap=None):
    _check(ctx, load().hg_evaluate(ctx, _ptr(idx, np.int32), int(m), _ptr(acc), _ptr(jerk), _ptr(snap)))


def hg_condition_scale(ctx, m, out=None):
    """sum_j m_j / (r_ij^2 + eps^2) of the last mixed evaluation's m particles."""
    out = np.empty(int(m)) if out is None else out
    _check(ctx, load().hg_condition_scale(ctx, _ptr(out), int(m)))
    return out


def hg_correct(ctx, idx, m):
    _check(ctx, load().hg_correct(ctx, _ptr(idx, np.int32), int(m)))


def hg_step(ctx, n_steps):
    _check(ctx, load().hg_step(ctx, int(n_steps)))


def hg_advance(ctx, t_end):
    k = C.c_int64()
    _check(ctx, load().hg_advance(ctx, float(t_end), C.byref(k)))
    return k.value


def hg_energy(ctx):
    K, W = C.c_double(), C.c_double()
    _check(ctx, load().hg_energy(ctx, C.byref(K), C.byref(W)))
    return K.value, W.value


def hg_angular_momentum(ctx):
    L = (C.c_double * 3)()
    _check(ctx, load().hg_angular_momentum(ctx, L))
    return np.array(list(L))


def hg_bind_device(ctx, arrays: dict | None, copy_in: bool = True):
    """Bind CUDA float64 tensors (keys of STATE_FIELDS) as the context's state;
    None unbinds.  Keep the tensors alive while bound."""
    if arrays is None:
        _check(ctx, load().hg_bind_device(ctx, None, 0))
        return
    s = hg_state(**{f: _ptr(arrays[f]) for f in STATE_FIELDS}, t_sys=0.0)
    _check(ctx, load().hg_bind_device(ctx, C.byref(s), int(bool(copy_in))))


def hg_get_state(ctx, out: dict):
    """Fills the arrays of out (keys of STATE_FIELDS; missing keys are skipped); returns t_sys."""
    st = hg_state()
    for f in STATE_FIELDS:
        setattr(st, f, _ptr(out.get(f)))
    _check(ctx, load().hg_get_state(ctx, C.byref(st)))
    return st.t_sys


def hg_set_state(ctx, state: dict, t_sys: float):
    st = hg_state()
    for f in STATE_FIELDS:
        setattr(st, f, _ptr(state[f]))
    st.t_sys = float(t_sys)
    _check(ctx, load().hg_set_state(ctx, C.byref(st)))


def hg_get_stats(ctx):
    s = hg_stats()
    _check(ctx, load().hg_get_stats(ctx, C.byref(s)))
    return {"block_steps": s.block_steps, "interactions": s.interactions, "last_m": s.last_m, "t_sys": s.t_sys,
            "kernels": s.kernels}


def hg_get_profile(ctx, reset=False):
    p = hg_profile()
    _check(ctx, load().hg_get_profile(ctx, C.byref(p), int(bool(reset))))
    return {"ms": dict(zip(SECTIONS, list(p.ms))), "block_steps": p.block_steps}


def hg_tune(ctx, m_max=0, reps=0):
    """Time the evaluation plans per block-size bucket; returns one dict per bucket measured."""
    rep = (hg_tune_entry * HG_TUNE_BUCKETS)()
    n = C.c_int32(0)
    _check(ctx, load().hg_tune(ctx, int(m_max), int(reps), rep, HG_TUNE_BUCKETS, C.byref(n)))
    keys = [f for f, _ in hg_tune_entry._fields_]
    return [{k: getattr(rep[q], k) for k in keys} for q in range(n.value)]


def hg_time_evaluate(ctx, idx, m, reps=0):
    """Mean device time (us) of evaluating the listed particles with the context's plan."""
    us = C.c_double()
    _check(ctx, load().hg_time_evaluate(ctx, _ptr(idx, np.int32), int(m), int(reps), C.byref(us)))
    return us.value


def hg_get_tuning(ctx):
    t = np.empty(HG_TUNE_BUCKETS, dtype=np.int16)
    _check(ctx, load().hg_get_tuning(ctx, t.ctypes.data_as(C.POINTER(C.c_int16))))
    return t


def hg_set_tuning(ctx, table):
    t = np.ascontiguousarray(table, dtype=np.int16)
    if t.shape != (HG_TUNE_BUCKETS,):
        raise ValueError(f"the table holds {HG_TUNE_BUCKETS} values")
    _check(ctx, load().hg_set_tuning(ctx, t.ctypes.data_as(C.POINTER(C.c_int16))))


def hg_evaluate_static(mass, pos, vel, acc_pred, eps, precision, idx, m, acc, jerk, snap, stream=None):
    """Context-free evaluation that allocates nothing (device arrays only, n <= 16384)."""
    s = getattr(stream, "cuda_stream", stream)
    rc = load().hg_evaluate_static(int(mass.shape[0]), _ptr(mass), _ptr(pos), _ptr(vel), _ptr(acc_pred),
                                   float(eps), int(precision), _ptr(idx, np.int32), int(m), _ptr(acc),
                                   _ptr(jerk), _ptr(snap), s)
    if rc != HG_OK:
        raise HGError(rc, load().hg_init_error().decode())


PEAK_FORMS = {"f32": 0, "f32x2": 1, "f64": 2}


def hg_peak_flops(form, device=0, stream=None):
    """Measured FMA rate of the CUDA cores (form "f32", "f32x2" or "f64"):
    (TFLOP/s, duration of the timed launch in ms)."""
    s = getattr(stream, "cuda_stream", stream)
    tf, ms = C.c_double(), C.c_double()
    rc = load().hg_peak_flops(PEAK_FORMS[form], int(device), s, C.byref(tf), C.byref(ms))
    if rc != HG_OK:
        raise HGError(rc, load().hg_init_error().decode())
    return tf.value, ms.value


def hg_inject_fault(kind, nth=0):
    """Testing: make the nth library allocation (HG_FAULT_ALLOC) or checked CUDA
    call (HG_FAULT_CUDA) fail; HG_FAULT_NONE disarms."""
    rc = load().hg_inject_fault(int(kind), int(nth))
    if rc != HG_OK:
        raise HGError(rc, "bad fault kind or count")


def hg_build_checked():
    """True when the loaded library is the checked build."""
    return bool(load().hg_build_checked())


def hg_test_corrupt_list(ctx, pos, value):
    """Testing (checked build only): write value into entry pos of the current block list."""
    _check(ctx, load().hg_test_corrupt_list(ctx, int(pos), int(value)))


def hg_size(ctx):
    return load().hg_size(ctx)


def hg_last_error(ctx):
    return load().hg_last_error(ctx).decode()


def hg_free(ctx):
    if ctx:
        load().hg_free(ctx)


def new_state(n: int, like=None):
    """Host (numpy) or, with like=a torch device, CUDA arrays for hg_get_state."""
    shapes = {f: ((n,) if f in ("mass", "t", "dt") else (n, 3)) for f in STATE_FIELDS}
    if like is None:
        return {f: np.empty(s) for f, s in shapes.items()}
    import torch
    return {f: torch.empty(s, dtype=torch.float64, device=like) for f, s in shapes.items()}
