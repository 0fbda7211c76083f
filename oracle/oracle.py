"""ctypes access to hg_oracle.c (plain single-threaded FP64 C).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the benchmark).
The library is compiled from source with gcc on first use, with FP contraction
off so that x86 and Arm hosts produce identical results.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.c_int64

FIELDS = {"mass": 0, "pos": 1, "vel": 2, "acc": 3, "jerk": 4, "snap": 5, "crackle": 6, "t": 7, "dt": 8}


def build(force: bool = False) -> str:
    """Compile liboracle.so if it is missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                        "-shared", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # HG_ORACLE_LIB: a separately built copy (the planted-mistake test
            # points the pins at a deliberately broken build this way).
            L = C.CDLL(os.environ.get("HG_ORACLE_LIB") or build())
            L.or_predict.argtypes = [_I64] + [_D] * 7 + [C.c_double] + [_D] * 3
            L.or_eval.argtypes = [_I64, _D, _D, _D, _D, C.c_double, _I64, _I32, _D, _D, _D]
            L.or_eval_absum.argtypes = [_I64, _D, _D, _D, _D, C.c_double, _I64, _I32, _D]
            L.or_correct.argtypes = [C.c_double] + [_D] * 10
            L.or_interp.argtypes = [C.c_double] + [_D] * 9
            L.or_criterion.argtypes = [C.c_double, C.c_int, _D]
            L.or_criterion.restype = C.c_double
            L.or_block_dt.argtypes = [C.c_double] * 5
            L.or_block_dt.restype = C.c_double
            L.or_block_dt_init.argtypes = [C.c_double] * 3
            L.or_block_dt_init.restype = C.c_double
            L.or_next_block.argtypes = [_I64, _D, _D, _D, _I32]
            L.or_next_block.restype = _I64
            L.or_energy.argtypes = [_I64, _D, _D, _D, C.c_double, _D, _D]
            L.or_angular_momentum.argtypes = [_I64, _D, _D, _D, _D]
            L.or_angular_momentum.restype = None
            L.or_sys_angular_momentum.argtypes = [C.c_void_p, C.c_double, _D]
            L.or_sys_angular_momentum.restype = None
            L.or_sys_create.argtypes = [_I64, _D, _D, _D] + [C.c_double] * 5
            L.or_sys_create_order.argtypes = [_I64, _D, _D, _D] + [C.c_double] * 5 + [C.c_int]
            L.or_sys_create_order.restype = C.c_void_p
            L.or_sys_set_order.argtypes = [C.c_void_p, C.c_int]
            L.or_sys_set_order.restype = None
            L.or_correct4.argtypes = [C.c_double] + [_D] * 8
            L.or_correct4.restype = None
            L.or_interp4.argtypes = [C.c_double] + [_D] * 6
            L.or_interp4.restype = None
            L.or_sys_create.restype = C.c_void_p
            L.or_sys_alloc.argtypes = [_I64] + [C.c_double] * 5
            L.or_sys_alloc.restype = C.c_void_p
            L.or_sys_free.argtypes = [C.c_void_p]
            L.or_sys_step.argtypes = [C.c_void_p, _D]
            L.or_sys_step.restype = _I64
            L.or_sys_advance.argtypes = [C.c_void_p, C.c_double]
            L.or_sys_advance.restype = _I64
            L.or_sys_energy.argtypes = [C.c_void_p, C.c_double, _D, _D]
            L.or_sys_predict_eval.argtypes = [C.c_void_p, C.c_double, _I64, _I32, _D, _D, _D]
            L.or_sys_predict_absum.argtypes = [C.c_void_p, C.c_double, _I64, _I32, _D]
            L.or_sys_get.argtypes = [C.c_void_p, C.c_int, _D]
            L.or_sys_set.argtypes = [C.c_void_p, C.c_int, _D]
            L.or_sys_time.argtypes = [C.c_void_p]
            L.or_sys_time.restype = C.c_double
            L.or_sys_set_time.argtypes = [C.c_void_p, C.c_double]
            L.or_sys_steps.argtypes = [C.c_void_p]
            L.or_sys_steps.restype = _I64
            L.or_sys_interactions.argtypes = [C.c_void_p]
            L.or_sys_interactions.restype = _I64
            _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def predict(x, v, a, j, s, c, t, t_to):
    """Predicted positions, velocities and accelerations of every particle at t_to."""
    x, v, a, j, s, c = (_f64(q, (-1, 3)) for q in (x, v, a, j, s, c))
    t = _f64(t)
    n = x.shape[0]
    xp, vp, ap = (np.empty((n, 3)) for _ in range(3))
    lib().or_predict(n, _d(x), _d(v), _d(a), _d(j), _d(s), _d(c), _d(t), float(t_to), _d(xp), _d(vp), _d(ap))
    return xp, vp, ap


def evaluate(mass, xp, vp, ap, eps, idx=None):
    """acc, jerk, snap of the listed particles against all others (direct sum)."""
    mass = _f64(mass)
    xp, vp, ap = (_f64(q, (-1, 3)) for q in (xp, vp, ap))
    n = mass.shape[0]
    idx = np.arange(n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    m = idx.shape[0]
    acc, jerk, snap = (np.empty((m, 3)) for _ in range(3))
    lib().or_eval(n, _d(mass), _d(xp), _d(vp), _d(ap), float(eps), m, idx.ctypes.data_as(_I32),
                  _d(acc), _d(jerk), _d(snap))
    return acc, jerk, snap


def eval_absum(mass, xp, vp, ap, eps, idx=None):
    """Per listed particle: sums over j of |a_ij|, |j_ij|, |s_ij| (columns 0, 1, 2)."""
    mass = _f64(mass)
    xp, vp, ap = (_f64(q, (-1, 3)) for q in (xp, vp, ap))
    n = mass.shape[0]
    idx = np.arange(n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty((idx.shape[0], 3))
    lib().or_eval_absum(n, _d(mass), _d(xp), _d(vp), _d(ap), float(eps), idx.shape[0],
                        idx.ctypes.data_as(_I32), _d(out))
    return out


def correct(h, x0, v0, a0, j0, s0, a1, j1, s1):
    """Corrected position and velocity of one particle after a step h."""
    args = [_f64(q, (3,)) for q in (x0, v0, a0, j0, s0, a1, j1, s1)]
    x1, v1 = np.empty(3), np.empty(3)
    lib().or_correct(float(h), *[_d(q) for q in args], _d(x1), _d(v1))
    return x1, v1


def correct4(h, x0, v0, a0, j0, a1, j1):
    """4th-order Hermite corrector: (x1, v1)."""
    args = [_f64(q, (3,)) for q in (x0, v0, a0, j0, a1, j1)]
    x1, v1 = np.empty(3), np.empty(3)
    lib().or_correct4(float(h), *[_d(q) for q in args], _d(x1), _d(v1))
    return x1, v1


def interp4(h, a0, j0, a1, j1):
    """snap and crackle at the end of a step from the cubic Hermite interpolant."""
    args = [_f64(q, (3,)) for q in (a0, j0, a1, j1)]
    s1, c1 = np.empty(3), np.empty(3)
    lib().or_interp4(float(h), *[_d(q) for q in args], _d(s1), _d(c1))
    return s1, c1


def interp(h, a0, j0, s0, a1, j1, s1):
    """crackle, pop and 5th derivative at the end of a step from the Hermite interpolant."""
    args = [_f64(q, (3,)) for q in (a0, j0, s0, a1, j1, s1)]
    c1, p1, q1 = np.empty(3), np.empty(3), np.empty(3)
    lib().or_interp(float(h), *[_d(q) for q in args], _d(c1), _d(p1), _d(q1))
    return c1, p1, q1


def criterion(eta, p, derivs):
    """Generalized Aarseth step from a^(0) .. a^(p-1) (p 3-vectors)."""
    d = _f64(derivs, (-1,))
    assert d.shape[0] == 3 * p
    return lib().or_criterion(float(eta), int(p), _d(d))


def block_dt(crit, dt_old, t_new, dt_min, dt_max):
    return lib().or_block_dt(float(crit), float(dt_old), float(t_new), float(dt_min), float(dt_max))


def block_dt_init(crit, dt_min, dt_max):
    return lib().or_block_dt_init(float(crit), float(dt_min), float(dt_max))


def next_block(t, dt):
    t, dt = _f64(t), _f64(dt)
    idx = np.empty(t.shape[0], dtype=np.int32)
    tn = C.c_double()
    m = lib().or_next_block(t.shape[0], _d(t), _d(dt), C.byref(tn), idx.ctypes.data_as(_I32))
    return tn.value, idx[:m].copy()


def energy(mass, x, v, eps):
    """(kinetic, potential) with the softened pair potential."""
    mass = _f64(mass)
    x, v = _f64(x, (-1, 3)), _f64(v, (-1, 3))
    K, W = C.c_double(), C.c_double()
    lib().or_energy(mass.shape[0], _d(mass), _d(x), _d(v), float(eps), C.byref(K), C.byref(W))
    return K.value, W.value


def angular_momentum(mass, x, v):
    """Total angular momentum sum_i m_i r_i x v_i (3-vector)."""
    mass = _f64(mass)
    x, v = _f64(x, (-1, 3)), _f64(v, (-1, 3))
    L = np.empty(3)
    lib().or_angular_momentum(mass.shape[0], _d(mass), _d(x), _d(v), _d(L))
    return L


class System:
    """The oracle integrator (start-up evaluation included unless state= is given)."""

    def __init__(self, mass, pos, vel, eps, eta, eta_init=0.01, dt_min=2.0 ** -25, dt_max=2.0 ** -3,
                 state=None, order=6):
        L = lib()
        mass = _f64(mass)
        self.n = mass.shape[0]
        if order not in (4, 6):
            raise ValueError("order must be 4 or 6")
        if state is None:
            pos, vel = _f64(pos, (-1, 3)), _f64(vel, (-1, 3))
            self._p = L.or_sys_create_order(self.n, _d(mass), _d(pos), _d(vel), float(eps), float(eta),
                                            float(eta_init), float(dt_min), float(dt_max), int(order))
        else:
            self._p = L.or_sys_alloc(self.n, float(eps), float(eta), float(eta_init), float(dt_min),
                                     float(dt_max))
            if self._p:
                L.or_sys_set_order(self._p, int(order))
        if not self._p:
            raise MemoryError("oracle allocation failed")
        if state is not None:
            self.set_state(state)

    def __del__(self):
        p = getattr(self, "_p", None)
        if p:
            lib().or_sys_free(p)
            self._p = None

    def step(self):
        t = C.c_double()
        m = lib().or_sys_step(self._p, C.byref(t))
        return m, t.value

    def advance(self, t_end):
        return lib().or_sys_advance(self._p, float(t_end))

    def energy(self, t=None):
        K, W = C.c_double(), C.c_double()
        lib().or_sys_energy(self._p, float(self.t_sys if t is None else t), C.byref(K), C.byref(W))
        return K.value, W.value

    def angular_momentum(self, t=None):
        L = np.empty(3)
        lib().or_sys_angular_momentum(self._p, float(self.t_sys if t is None else t), _d(L))
        return L

    def predict_eval(self, t, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        m = idx.shape[0]
        acc, jerk, snap = (np.empty((m, 3)) for _ in range(3))
        lib().or_sys_predict_eval(self._p, float(t), m, idx.ctypes.data_as(_I32), _d(acc), _d(jerk), _d(snap))
        return acc, jerk, snap

    def predict_absum(self, t, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        out = np.empty((idx.shape[0], 3))
        lib().or_sys_predict_absum(self._p, float(t), idx.shape[0], idx.ctypes.data_as(_I32), _d(out))
        return out

    def get(self, field):
        shape = (self.n,) if field in ("mass", "t", "dt") else (self.n, 3)
        out = np.empty(shape)
        lib().or_sys_get(self._p, FIELDS[field], _d(out))
        return out

    def set(self, field, value):
        shape = (self.n,) if field in ("mass", "t", "dt") else (self.n, 3)
        lib().or_sys_set(self._p, FIELDS[field], _d(_f64(value, shape)))

    def get_state(self):
        st = {f: self.get(f) for f in FIELDS}
        st["t_sys"] = self.t_sys
        return st

    def set_state(self, st):
        for f in FIELDS:
            self.set(f, st[f])
        lib().or_sys_set_time(self._p, float(st.get("t_sys", 0.0)))

    @property
    def t_sys(self):
        return lib().or_sys_time(self._p)

    @property
    def steps(self):
        return lib().or_sys_steps(self._p)

    @property
    def interactions(self):
        return lib().or_sys_interactions(self._p)
