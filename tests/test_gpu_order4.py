"""The 4th-order Hermite variant (hg_opts.order = 4, the paper's criterion with
p = 4) against the oracle's 4th-order integrator."""
import math

import numpy as np
import pytest

import oracle
from paper_1207_2367_gb300 import inputs
from gpu_util import DT_MAX, DT_MIN, gpu_context, gpu_state, rel_rows
from test_gpu_parity import TOL, check_eval

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_order4_block_steps_with_injection_match_oracle(hg, precision):
    """Each block step from the oracle's current state: same block, corrected
    state, snap and crackle kept zero, and (FP64) the same new steps."""
    n, eps = 1024, 1e-3
    p = inputs.plummer(n, 1)
    sysm = oracle.System(p.mass, p.pos, p.vel, eps, 0.3, 0.01, DT_MIN, DT_MAX, order=4)
    assert np.all(sysm.get("snap") == 0)
    ctx = gpu_context(hg, sysm, precision, eps, eta=0.3, order=4)
    dt_mismatch = active = 0
    try:
        for _ in range(40):
            st = sysm.get_state()
            hg.hg_set_state(ctx, {f: st[f] for f in hg.STATE_FIELDS}, st["t_sys"])
            idx = np.empty(n, dtype=np.int32)
            tn, m = hg.hg_next_block(ctx, idx)
            tn_ref, idx_ref = oracle.next_block(st["t"], st["dt"])
            assert tn == tn_ref and m == len(idx_ref)
            np.testing.assert_array_equal(idx[:m], idx_ref)
            acc, jerk, snap = (np.empty((m, 3)) for _ in range(3))
            hg.hg_predict(ctx, tn)
            hg.hg_evaluate(ctx, None, m, acc, jerk, snap)
            ref = sysm.predict_eval(tn, idx_ref)
            check_eval((acc, jerk, snap), ref, precision, sysm.predict_absum(tn, idx_ref) if precision else None)
            hg.hg_correct(ctx, None, m)
            sysm.step()
            got, t_sys = gpu_state(hg, ctx, n)
            assert t_sys == tn
            ids = idx_ref
            for f, tol in (("pos", 1e-13 if precision == 0 else 1e-9), ("vel", 1e-12 if precision == 0 else 1e-7)):
                assert rel_rows(got[f][ids], sysm.get(f)[ids]).max() < tol, f
            for f, tol in (("acc", TOL[precision][0]), ("jerk", TOL[precision][1])):
                g, r = got[f][ids], sysm.get(f)[ids]
                err = rel_rows(g, r).max() if precision == 0 else np.linalg.norm(g - r) / np.linalg.norm(r)
                assert err < tol, (f, err)   # mixed: normwise, as for the evaluation itself
            assert np.all(got["snap"][ids] == 0) and np.all(got["crackle"][ids] == 0)
            np.testing.assert_array_equal(got["t"], sysm.get("t"))
            dt_mismatch += int(np.sum(got["dt"][ids] != sysm.get("dt")[ids]))
            active += m
        assert dt_mismatch <= (0 if precision == 0 else max(1, active // 200)), (dt_mismatch, active)
    finally:
        hg.hg_free(ctx)


def test_order4_integration_matches_oracle(hg):
    """N = 1024 Plummer to t = 0.25 with graph-replayed block steps: the oracle's
    step count and energy error, every particle at t_end."""
    n, eps, eta = 1024, 1e-3, 0.15
    p = inputs.plummer(n, 1)
    ref = oracle.System(p.mass, p.pos, p.vel, eps, eta, 0.01, DT_MIN, DT_MAX, order=4)
    E0 = sum(ref.energy())
    ref.advance(0.25)
    dE_ref = abs(sum(ref.energy()) - E0) / abs(E0)
    o = hg.hg_default_opts(precision=0, dt_min=DT_MIN, dt_max=DT_MAX, order=4)
    ctx = hg.hg_init(p.mass, p.pos, p.vel, eps, eta, o)
    try:
        steps = hg.hg_advance(ctx, 0.25)
        got, t_sys = gpu_state(hg, ctx, n)
        assert t_sys == 0.25 and np.all(got["t"] == 0.25)
        assert abs(steps - ref.steps) <= max(2, ref.steps // 50), (steps, ref.steps)
        dE = abs(sum(hg.hg_energy(ctx)) - E0) / abs(E0)
        assert dE < 10 * dE_ref + 1e-11, (dE, dE_ref)
        assert rel_rows(got["pos"], ref.get("pos")).max() < 1e-6
        assert np.all(got["snap"] == 0) and np.all(got["crackle"] == 0)
    finally:
        hg.hg_free(ctx)


def test_order4_kepler_converges_at_fourth_order(hg):
    """Two bodies, eps = 0, e = 0.5 to t = 8 on the GPU: error ratio ~16 per
    halving of eta, against the closed-form orbit."""
    p = inputs.kepler_pair()
    M = 8.0
    E = M
    for _ in range(60):
        E -= (E - 0.5 * math.sin(E) - M) / (1 - 0.5 * math.cos(E))
    exact = np.array([math.cos(E) - 0.5, math.sqrt(0.75) * math.sin(E), 0.0])
    errs = []
    for eta in (0.04, 0.02, 0.01):
        o = hg.hg_default_opts(precision=0, dt_min=DT_MIN, dt_max=1.0, eta_init=eta / 45, order=4)
        ctx = hg.hg_init(p.mass, p.pos, p.vel, 0.0, eta, o)
        try:
            hg.hg_advance(ctx, 8.0)
            got, _ = gpu_state(hg, ctx, 2)
            errs.append(np.linalg.norm(got["pos"][1] - got["pos"][0] - exact))
        finally:
            hg.hg_free(ctx)
    assert errs[-1] < 1e-7
    for e1, e2 in zip(errs, errs[1:]):
        assert 10.0 < e1 / e2 < 25.0, errs


def test_order_option_is_checked(hg):
    p = inputs.plummer(16, 1)
    with pytest.raises(hg.HGError):
        hg.hg_init(p.mass, p.pos, p.vel, 1e-3, 0.45, hg.hg_default_opts(order=5))
    o = hg.hg_default_opts(order=0)   # 0 means the default, 6
    ctx = hg.hg_init(p.mass, p.pos, p.vel, 1e-3, 0.45, o)
    hg.hg_free(ctx)
