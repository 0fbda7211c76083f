"""Helpers of the GPU parity tests: oracle-made states injected into the CUDA path.

Inputs always flow oracle -> GPU (never the reverse): the oracle's state is
built from seeded inputs, then copied into a CUDA context with hg_set_state.
"""
import numpy as np

import oracle
from paper_1207_2367_gb300 import inputs

DT_MAX = 1.0 / 16
DT_MIN = 2.0 ** -25


def rel_rows(x, ref):
    """Per-particle relative error ||x_i - ref_i|| / ||ref_i||."""
    x, ref = np.asarray(x).reshape(-1, 3), np.asarray(ref).reshape(-1, 3)
    den = np.linalg.norm(ref, axis=1)
    den = np.where(den > 0, den, 1.0)
    return np.linalg.norm(x - ref, axis=1) / den


def oracle_system(n, seed, eps, steps=0, imf="equal", eta=0.45, eta_init=0.01, dt_max=DT_MAX):
    p = inputs.plummer(n, seed, imf)
    s = oracle.System(p.mass, p.pos, p.vel, eps, eta, eta_init, DT_MIN, dt_max)
    for _ in range(steps):
        s.step()
    return s


def gpu_context(hg, sys_, precision, eps, eta=0.45, eta_init=0.01, dt_max=DT_MAX, **opt):
    """A CUDA context holding the oracle system's current state."""
    st = sys_.get_state()
    o = hg.hg_default_opts(precision=precision, dt_min=DT_MIN, dt_max=dt_max, eta_init=eta_init, start_mode=1, **opt)
    ctx = hg.hg_init(st["mass"], st["pos"], st["vel"], eps, eta, o)
    hg.hg_set_state(ctx, {f: st[f] for f in hg.STATE_FIELDS}, st["t_sys"])
    return ctx


def gpu_state(hg, ctx, n):
    out = hg.new_state(n)
    t = hg.hg_get_state(ctx, out)
    return out, t


def gpu_eval(hg, ctx, idx, t):
    m = len(idx)
    acc, jerk, snap = (np.empty((m, 3)) for _ in range(3))
    hg.hg_predict(ctx, t)
    hg.hg_evaluate(ctx, np.ascontiguousarray(idx, dtype=np.int32), m, acc, jerk, snap)
    return acc, jerk, snap
