"""The mixed path's noise floor for the step criterion.

FP32 rounding of the pair terms leaves an error in a_i of order 1e-7 of
sum_j |a_ij|, which is far above 1e-7 |a_i| where the pull of the rest of the
system nearly cancels (a particle near the centre).  The corrector scales its
noise floor with the evaluation's noise scale sum_j m_j / r_ij^2 >= sum_j |a_ij|:
a fourth-order residual A = a1 - a0 - j0 h - s0 h^2/2 below 3e-6 of that scale
may not shrink the step (the derivatives interpolated from it are noise), a
residual well above it does.
"""
import numpy as np
import pytest

import oracle
from paper_1207_2367_gb300 import inputs
from gpu_util import DT_MAX, DT_MIN, gpu_context, gpu_state

pytestmark = pytest.mark.gpu

NOISE_REL = 3e-6


def _noise_scale(mass, pos, i, eps):
    """sum_j m_j / (|r_ij|^2 + eps^2) and |a_i| (FP64, j != i)."""
    r = pos - pos[i]
    r2 = (r * r).sum(1) + eps * eps
    w = mass / r2
    w[i] = 0.0
    a = ((mass / r2 ** 1.5)[:, None] * r)
    a[i] = 0.0
    return float(w.sum()), float(np.linalg.norm(a.sum(0)))


@pytest.mark.parametrize("factor, shrinks", [(0.3, False), (10.0, True)])
def test_planted_residual_against_noise_scale(hg, factor, shrinks):
    """Every particle at t = 0 with dt = 2^-14 (one block of all N).  P, the
    particle among the 64 most central with the largest sum_j m_j/r_ij^2 / |a_i|
    (~70), gets a0 offset by factor * 3e-6 * scale along a0; its own residual at
    this step is ~1e-7, far below.  The oracle (FP64, no noise floor) shrinks
    P's step for both offsets.  The mixed path keeps it for the offset below its
    floor (the former floor, 3e-6 |a1|, would have shrunk it) and shrinks it for
    the one above."""
    n, eps, h = 4096, 1e-3, 2.0 ** -14
    p = inputs.plummer(n, 1)
    sysm = oracle.System(p.mass, p.pos, p.vel, eps, 0.45, 0.01, DT_MIN, DT_MAX)
    st = sysm.get_state()
    r_c = np.linalg.norm(st["pos"], axis=1)
    ratio = {}
    for i in np.argsort(r_c)[:64]:                  # near the centre: the pull cancels
        scale, amag = _noise_scale(st["mass"], st["pos"], i, eps)
        ratio[int(i)] = scale / amag
    P = max(ratio, key=ratio.get)
    scale, amag = _noise_scale(st["mass"], st["pos"], P, eps)
    assert scale > 10.0 * amag, (scale, amag)       # the former floor (|a1|) is >10x lower
    planted = factor * NOISE_REL * scale
    assert planted > 3.0 * NOISE_REL * amag         # above the former floor in both cases

    st["t"][:] = 0.0
    st["dt"][:] = h
    st["acc"][P] = st["acc"][P] * (1.0 + planted / np.linalg.norm(st["acc"][P]))
    ref = oracle.System(p.mass, p.pos, p.vel, eps, 0.45, 0.01, DT_MIN, DT_MAX)
    ref.set_state(st)
    ref.step()
    assert ref.get("dt")[P] < h                     # FP64 criterion: the residual is resolved
    ctx = gpu_context(hg, sysm, 1, eps, eta=0.45)
    try:
        hg.hg_set_state(ctx, {f: st[f] for f in hg.STATE_FIELDS}, 0.0)
        idx = np.empty(n, dtype=np.int32)
        t, m = hg.hg_next_block(ctx, idx)
        assert t == h and m == n
        hg.hg_predict(ctx, t)
        hg.hg_evaluate(ctx, None, m)
        hg.hg_correct(ctx, None, m)
        got, _ = gpu_state(hg, ctx, n)
        if shrinks:
            assert got["dt"][P] < h, got["dt"][P]
        else:
            assert got["dt"][P] >= h, got["dt"][P]
    finally:
        hg.hg_free(ctx)


def test_no_step_collapse_near_the_centre(hg):
    """N = 2^20 Salpeter (seed 3), eps = 1e-4, mixed: a particle near the centre
    (sum_j |a_ij| ~ 600 |a_i|) has an FP32 evaluation error of 1e-6 to 4e-6 of
    |a_i|.  With the floor at 3e-6 |a1| its step fell to dt_min = 2^-25 within 10
    block steps and 64 block steps reached only t = 1.1e-4; the FP64 path reaches
    t = 6.8e-4.  With the noise-scale floor no step falls below 2^-22."""
    n, eps = 1 << 20, 1e-4
    p = inputs.plummer(n, 3, imf="salpeter")
    o = hg.hg_default_opts(precision=hg.HG_MIXED, dt_min=DT_MIN, dt_max=DT_MAX)
    ctx = hg.hg_init(p.mass, p.pos, p.vel, eps, 0.45, o)
    try:
        low = np.inf
        for _ in range(8):
            hg.hg_step(ctx, 8)
            st = hg.new_state(n)
            hg.hg_get_state(ctx, st)
            low = min(low, float(st["dt"].min()))
        t = hg.hg_get_stats(ctx)["t_sys"]
        assert low >= 2.0 ** -22, low
        assert t > 4e-4, t
    finally:
        hg.hg_free(ctx)
