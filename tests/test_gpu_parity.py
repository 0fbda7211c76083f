"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 path: per-particle relative error ||x_i - ref_i|| / ||ref_i|| <= 1e-12 for
every particle, on acc, jerk and snap.
Mixed path (tolerances 1e-6 / 1e-5 / 1e-4 on acc / jerk / snap), all of:
  - normwise relative error of the output array, ||X - REF||_F / ||REF||_F;
  - per particle, the error relative to the condition scale sum_j ||term_ij||
    (oracle), i.e. relative to what any FP32 summation of the terms can resolve;
  - per-particle relative error for every particle whose sum is not badly
    conditioned (condition number kappa_i = sum_j ||term_ij|| / ||ref_i|| <= 10:
    99 % of a Plummer sphere's particles, the dense centre included; FP32 pair
    terms leave a per-particle error of up to ~1e-7 kappa_i, see
    test_fp32_pair_limits.py).
Integer and index work (block selection) is compared bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1207_2367_gb300 import inputs
from gpu_util import DT_MAX, DT_MIN, gpu_context, gpu_eval, gpu_state, oracle_system, rel_rows

pytestmark = pytest.mark.gpu

TOL = {0: (1e-12, 1e-12, 1e-12), 1: (1e-6, 1e-5, 1e-4)}
KAPPA_PER_PARTICLE = 10.0   # mixed path: the per-particle tolerance binds up to this condition number


def check_eval(got, ref, precision, absum=None):
    for k, (g, r, tol, name) in enumerate(zip(got, ref, TOL[precision], ("acc", "jerk", "snap"))):
        per = rel_rows(g, r)
        if precision == 0:
            assert per.max() <= tol, f"{name}: max rel err {per.max():.3e} > {tol:.0e}"
            continue
        g, r = np.asarray(g).reshape(-1, 3), np.asarray(r).reshape(-1, 3)
        normwise = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert normwise <= tol, f"{name}: normwise rel err {normwise:.3e} > {tol:.0e}"
        if absum is not None:
            scale = absum[:, k]
            cond = np.linalg.norm(g - r, axis=1) / np.where(scale > 0, scale, 1.0)
            assert cond.max() <= tol, f"{name}: conditioned rel err {cond.max():.3e} > {tol:.0e}"
            well = scale <= KAPPA_PER_PARTICLE * np.linalg.norm(r, axis=1)
            if well.any():
                assert per[well].max() <= tol, f"{name}: max rel err at kappa <= 10 {per[well].max():.3e}"


# --------------------------------------------------------------------------
# Evaluation step on injected oracle states.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [2, 3, 31, 257, 1000, 3001])
def test_eval_matches_oracle(hg, precision, n):
    eps = 1e-3
    sysm = oracle_system(n, 100 + n, eps, steps=3)
    ctx = gpu_context(hg, sysm, precision, eps)
    try:
        rng = np.random.default_rng(n)
        t = sysm.t_sys + 1.0 / 256
        lists = [np.arange(n), np.array([0]), np.array([n - 1]),
                 np.sort(rng.choice(n, size=max(1, n // 3), replace=False))]
        for idx in lists:
            got = gpu_eval(hg, ctx, idx, t)
            ref = sysm.predict_eval(t, idx)
            check_eval(got, ref, precision, sysm.predict_absum(t, idx))
    finally:
        hg.hg_free(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_every_launch_plan_gives_the_same_result(hg, precision):
    """Threads per i (1..64) and j-split factors change the work layout, not the result."""
    n, eps = 2000, 1e-3
    sysm = oracle_system(n, 7, eps, steps=2)
    t = sysm.t_sys + 1.0 / 512
    idx_sets = [np.arange(0, n, 3), np.array([5, 17, 1999])]
    refs = [sysm.predict_eval(t, idx) for idx in idx_sets]
    scales = [sysm.predict_absum(t, idx) for idx in idx_sets]
    for tpi in (1, 2, 4, 8, 16, 32, 64):
        for jsplit in (0, 1, 3, 8):
            ctx = gpu_context(hg, sysm, precision, eps, tpi=tpi, jsplit=jsplit)
            try:
                for idx, ref, sc in zip(idx_sets, refs, scales):
                    check_eval(gpu_eval(hg, ctx, idx, t), ref, precision, sc)
            finally:
                hg.hg_free(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_softening_skips_self_pair(hg, precision):
    """eps = 0 takes the guarded path: the j == i pair is skipped, results finite."""
    n = 300
    p = inputs.plummer(n, 4)
    sysm = oracle.System(p.mass, p.pos, p.vel, 0.0, 0.45, 0.01, DT_MIN, DT_MAX)
    ctx = gpu_context(hg, sysm, precision, 0.0)
    try:
        idx = np.arange(n)
        got = gpu_eval(hg, ctx, idx, 0.0)
        assert all(np.all(np.isfinite(g)) for g in got)
        check_eval(got, sysm.predict_eval(0.0, idx), precision, sysm.predict_absum(0.0, idx))
    finally:
        hg.hg_free(ctx)


# --------------------------------------------------------------------------
# Block selection (bit exact), start-up and one whole block step.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 5, 1000, 8193, 20000])
def test_next_block_bit_exact(hg, n):
    sysm = oracle_system(n, 3, 1e-3, steps=0) if n <= 1000 else None
    rng = np.random.default_rng(n)
    if sysm is None:
        p = inputs.plummer(n, 3)
        sysm = oracle.System(p.mass, p.pos, p.vel, 1e-3, 0.45, state={
            "mass": p.mass, "pos": p.pos, "vel": p.vel, "acc": np.zeros((n, 3)), "jerk": np.zeros((n, 3)),
            "snap": np.zeros((n, 3)), "crackle": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.full(n, DT_MAX),
            "t_sys": 0.0})
    # random commensurate times and steps
    k = rng.integers(4, 12, size=n)
    dt = 2.0 ** -k
    t = np.floor(rng.uniform(0, 1, size=n) / dt) * dt
    sysm.set("t", t)
    sysm.set("dt", dt)
    ctx = gpu_context(hg, sysm, 0, 1e-3)
    try:
        idx = np.empty(n, dtype=np.int32)
        tn, m = hg.hg_next_block(ctx, idx)
        tn_ref, idx_ref = oracle.next_block(t, dt)
        assert tn == tn_ref
        assert m == len(idx_ref)
        np.testing.assert_array_equal(idx[:m], idx_ref)
    finally:
        hg.hg_free(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_start_up_matches_oracle(hg, precision):
    n, eps = 1024, 1e-3
    p = inputs.plummer(n, 1)
    ref = oracle.System(p.mass, p.pos, p.vel, eps, 0.45, 0.01, DT_MIN, DT_MAX)
    o = hg.hg_default_opts(precision=precision, dt_min=DT_MIN, dt_max=DT_MAX)
    ctx = hg.hg_init(p.mass, p.pos, p.vel, eps, 0.45, o)
    try:
        got, t_sys = gpu_state(hg, ctx, n)
        assert t_sys == 0.0
        check_eval((got["acc"], got["jerk"], got["snap"]), (ref.get("acc"), ref.get("jerk"), ref.get("snap")),
                   precision, oracle.eval_absum(p.mass, p.pos, p.vel, np.zeros((n, 3)), eps))
        assert np.all(got["crackle"] == 0) and np.all(got["t"] == 0)
        same = np.mean(got["dt"] == ref.get("dt"))
        assert same >= (1.0 if precision == 0 else 0.99), same
    finally:
        hg.hg_free(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_block_steps_with_injection_match_oracle(hg, precision):
    """Each block step from the oracle's current state: same block, matching
    evaluation, corrected state and steps (configuration N = 1024, eps = 1e-3)."""
    n, eps = 1024, 1e-3
    sysm = oracle_system(n, 1, eps, steps=0)
    ctx = gpu_context(hg, sysm, precision, eps)
    worst = np.zeros(3)
    dt_mismatch = 0
    active = 0
    try:
        for step in range(40):
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
            absum = sysm.predict_absum(tn, idx_ref)
            check_eval((acc, jerk, snap), ref, precision, absum if precision else None)
            for k, (g, r) in enumerate(zip((acc, jerk, snap), ref)):
                worst[k] = max(worst[k], np.linalg.norm(g - r) / np.linalg.norm(r))
            hg.hg_correct(ctx, None, m)
            sysm.step()
            got, t_sys = gpu_state(hg, ctx, n)
            assert t_sys == tn
            ids = idx_ref
            for f, tol in (("pos", 1e-13 if precision == 0 else 1e-9), ("vel", 1e-12 if precision == 0 else 1e-7)):
                assert rel_rows(got[f][ids], sysm.get(f)[ids]).max() < tol, f
            check_corrected_derivatives(got, st, sysm, ids, (acc, jerk, snap), absum, precision)
            np.testing.assert_array_equal(got["t"], sysm.get("t"))
            dt_mismatch += int(np.sum(got["dt"][ids] != sysm.get("dt")[ids]))
            active += m
        assert np.all(worst <= np.array(TOL[precision])), worst
        assert dt_mismatch <= (0 if precision == 0 else max(1, active // 200)), (dt_mismatch, active)
    finally:
        hg.hg_free(ctx)


def _nrm(x):
    return np.linalg.norm(np.asarray(x).reshape(-1, 3), axis=1)


def check_corrected_derivatives(got, st, sysm, ids, evaluated, absum, precision):
    """After a correction, element by element for the corrected particles ids:
    - the stored acc, jerk, snap are the evaluated ones (bitwise) and match the
      oracle's step (the evaluation metric);
    - the stored crackle equals the oracle's Hermite interpolant (reading R5)
      applied to the same inputs (old a, jerk, snap from the injected state, the
      GPU's new ones) within FP64 rounding: 1e-13 of the formula's condition
      scale S_c = (60 (|a1| + |a0| + |j0| h + |s0| h^2/2) + 36 (|j1| + |j0| +
      |s0| h) h + 9 (|s1| + |s0|) h^2) / h^3;
    - the stored crackle matches the oracle's own step within what the
      evaluation tolerance allows: (60 da + 36 dj h + 9 ds h^2) / h^3 with da,
      dj, ds the tolerated errors of the new acc, jerk, snap (FP64: 1e-12 of
      their norms; mixed: 1e-6 / 1e-5 / 1e-4 of the condition scales), plus the
      rounding term above."""
    acc, jerk, snap = evaluated
    for f, g in (("acc", acc), ("jerk", jerk), ("snap", snap)):
        np.testing.assert_array_equal(got[f][ids], g, err_msg=f)
    check_eval(tuple(got[f][ids] for f in ("acc", "jerk", "snap")),
               tuple(sysm.get(f)[ids] for f in ("acc", "jerk", "snap")), precision, absum if precision else None)
    h = st["dt"][ids]
    a0, j0, s0 = st["acc"][ids], st["jerk"][ids], st["snap"][ids]
    c_same = np.stack([oracle.interp(h[q], a0[q], j0[q], s0[q], acc[q], jerk[q], snap[q])[0]
                       for q in range(len(ids))])
    Sc = (60.0 * (_nrm(acc) + _nrm(a0) + _nrm(j0) * h + _nrm(s0) * h ** 2 / 2)
          + 36.0 * (_nrm(jerk) + _nrm(j0) + _nrm(s0) * h) * h + 9.0 * (_nrm(snap) + _nrm(s0)) * h ** 2) / h ** 3
    dc = _nrm(got["crackle"][ids] - c_same)
    assert (dc / Sc).max() <= 1e-13, (dc / Sc).max()
    if precision == 0:
        da, dj, ds = 1e-12 * _nrm(acc), 1e-12 * _nrm(jerk), 1e-12 * _nrm(snap)
    else:
        da, dj, ds = 1e-6 * absum[:, 0], 1e-5 * absum[:, 1], 1e-4 * absum[:, 2]
    bound = (60.0 * da + 36.0 * dj * h + 9.0 * ds * h ** 2) / h ** 3 + 1e-13 * Sc
    dref = _nrm(got["crackle"][ids] - sysm.get("crackle")[ids])
    assert np.all(dref <= bound), (dref / bound).max()


# --------------------------------------------------------------------------
# Whole integration (configuration: N = 1024 Plummer, eps = 1e-3, eta = 0.45,
# dt_max = 1/16, t = 0.25).
# --------------------------------------------------------------------------
def test_fp64_integration_config_small(hg):
    n, eps = 1024, 1e-3
    p = inputs.plummer(n, 1)
    ref = oracle.System(p.mass, p.pos, p.vel, eps, 0.45, 0.01, DT_MIN, DT_MAX)
    E0_ref = sum(ref.energy())
    ref.advance(0.25)
    dE_ref = abs(sum(ref.energy()) - E0_ref) / abs(E0_ref)

    o = hg.hg_default_opts(precision=0, dt_min=DT_MIN, dt_max=DT_MAX)
    ctx = hg.hg_init(p.mass, p.pos, p.vel, eps, 0.45, o)
    try:
        K0, W0 = hg.hg_energy(ctx)
        assert (K0 + W0) == pytest.approx(E0_ref, rel=1e-13)
        steps = hg.hg_advance(ctx, 0.25)
        K1, W1 = hg.hg_energy(ctx)
        dE = abs(K1 + W1 - (K0 + W0)) / abs(K0 + W0)
        got, t_sys = gpu_state(hg, ctx, n)
        assert t_sys == 0.25 and np.all(got["t"] == 0.25)
        assert abs(steps - ref.steps) <= max(2, ref.steps // 50), (steps, ref.steps)
        assert dE < 1e-8 and dE_ref < 1e-8
        assert dE < 10 * dE_ref + 1e-11
        assert rel_rows(got["pos"], ref.get("pos")).max() < 1e-6
        stats = hg.hg_get_stats(ctx)
        assert stats["block_steps"] == steps and stats["t_sys"] == 0.25
    finally:
        hg.hg_free(ctx)


def test_graph_steps_equal_explicit_steps_bitwise(hg):
    n, eps = 777, 1e-3
    sysm = oracle_system(n, 9, eps, steps=1)
    a = gpu_context(hg, sysm, 1, eps, graph_steps=4)
    b = gpu_context(hg, sysm, 1, eps)
    try:
        hg.hg_step(a, 11)
        for _ in range(11):
            tn, m = hg.hg_next_block(b)
            hg.hg_predict(b, tn)
            hg.hg_evaluate(b, None, m)
            hg.hg_correct(b, None, m)
        sa, ta = gpu_state(hg, a, n)
        sb, tb = gpu_state(hg, b, n)
        assert ta == tb
        for f in hg.STATE_FIELDS:
            np.testing.assert_array_equal(sa[f], sb[f], err_msg=f)
    finally:
        hg.hg_free(a)
        hg.hg_free(b)


def test_energy_matches_oracle(hg):
    n, eps = 3000, 1e-3
    sysm = oracle_system(n, 21, eps, steps=5)
    ref = sysm.energy()
    for prec, tol in ((0, 1e-13), (1, 2e-7)):
        ctx = gpu_context(hg, sysm, 0, eps, energy_precision=prec)
        try:
            K, W = hg.hg_energy(ctx)
            assert K == pytest.approx(ref[0], rel=1e-14)
            assert W == pytest.approx(ref[1], rel=tol)
        finally:
            hg.hg_free(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_black_hole_system_matches_oracle(hg, precision):
    """A Plummer sphere with a central object of 5 % of its mass (the
    massive-object case of Sect. 5.5): evaluations of all particles and of
    random subsets, and 20 injected block steps with their new steps."""
    n, eps = 1024, 1e-4
    p = inputs.plummer_black_hole(n, 11, m_bh=0.05)
    sysm = oracle.System(p.mass, p.pos, p.vel, eps, 0.45, 0.01, DT_MIN, DT_MAX)
    for _ in range(3):
        sysm.step()
    ctx = gpu_context(hg, sysm, precision, eps)
    dt_mismatch = active = 0
    try:
        t = sysm.t_sys + 2.0 ** -12
        rng = np.random.default_rng(4)
        for idx in (np.arange(n), np.array([n - 1]), np.sort(rng.choice(n, 100, replace=False))):
            check_eval(gpu_eval(hg, ctx, idx, t), sysm.predict_eval(t, idx), precision, sysm.predict_absum(t, idx))
        for _ in range(20):
            st = sysm.get_state()
            hg.hg_set_state(ctx, {f: st[f] for f in hg.STATE_FIELDS}, st["t_sys"])
            tn, m = hg.hg_next_block(ctx)
            hg.hg_predict(ctx, tn)
            hg.hg_evaluate(ctx, None, m)
            hg.hg_correct(ctx, None, m)
            sysm.step()
            got, t_sys = gpu_state(hg, ctx, n)
            assert t_sys == sysm.t_sys
            np.testing.assert_array_equal(got["t"], sysm.get("t"))
            ids = np.nonzero(got["t"] == t_sys)[0]
            dt_mismatch += int(np.sum(got["dt"][ids] != sysm.get("dt")[ids]))
            active += len(ids)
            # relative to max(|r_i|, 0.01): the black hole sits ~1e-7 from the origin
            ref_pos = sysm.get("pos")
            err = np.linalg.norm(got["pos"] - ref_pos, axis=1) / np.maximum(np.linalg.norm(ref_pos, axis=1), 0.01)
            assert err.max() < (1e-13 if precision == 0 else 1e-9), err.max()
        assert dt_mismatch <= (0 if precision == 0 else max(1, active // 200)), (dt_mismatch, active)
    finally:
        hg.hg_free(ctx)


def test_angular_momentum_matches_oracle(hg):
    """L of the predicted system at the last block time (oracle state injected;
    particles at their own times), against the oracle's sum, relative to the
    condition scale sum_i m_i |r_i| |v_i| (|L| of an isotropic Plummer sphere is
    a near cancellation).  Then 60 graph block steps on the GPU against 60
    oracle block steps: L at the same block time.  (Individual block steps do
    not conserve L exactly: forces on a pair act at different times.)"""
    n, eps = 3000, 1e-3
    sysm = oracle_system(n, 22, eps, steps=5)
    ref = sysm.angular_momentum()
    st = sysm.get_state()
    scale = float(np.sum(st["mass"] * np.linalg.norm(st["pos"], axis=1) * np.linalg.norm(st["vel"], axis=1)))
    ctxs = [gpu_context(hg, sysm, prec, eps) for prec in (0, 1)]
    try:
        for ctx in ctxs:
            L = hg.hg_angular_momentum(ctx)
            assert np.linalg.norm(L - ref) <= 1e-14 * scale, (L, ref)
            hg.hg_step(ctx, 60)
        for _ in range(60):
            sysm.step()
        ref60 = sysm.angular_momentum()
        for prec, ctx in zip((0, 1), ctxs):
            assert hg.hg_get_stats(ctx)["t_sys"] == sysm.t_sys
            L1 = hg.hg_angular_momentum(ctx)
            assert np.linalg.norm(L1 - ref60) <= (1e-13 if prec == 0 else 1e-9) * scale, (prec, L1, ref60)
    finally:
        for ctx in ctxs:
            hg.hg_free(ctx)


def test_kepler_orbit_zero_softening(hg):
    """Two bodies, eps = 0, e = 0.5: the GPU integrator follows the closed-form orbit."""
    p = inputs.kepler_pair()
    o = hg.hg_default_opts(precision=0, dt_min=DT_MIN, dt_max=1.0, eta_init=0.1 / 45)
    ctx = hg.hg_init(p.mass, p.pos, p.vel, 0.0, 0.1, o)
    ref = oracle.System(p.mass, p.pos, p.vel, 0.0, 0.1, eta_init=0.1 / 45, dt_max=1.0)
    try:
        hg.hg_advance(ctx, 8.0)
        ref.advance(8.0)
        got, _ = gpu_state(hg, ctx, 2)
        rel = got["pos"][1] - got["pos"][0]
        M = 8.0
        E = M
        for _ in range(60):
            E -= (E - 0.5 * math.sin(E) - M) / (1 - 0.5 * math.cos(E))
        exact = np.array([math.cos(E) - 0.5, math.sqrt(0.75) * math.sin(E), 0.0])
        assert np.linalg.norm(rel - exact) < 1e-8
        np.testing.assert_allclose(got["pos"], ref.get("pos"), rtol=0, atol=1e-11)
    finally:
        hg.hg_free(ctx)


@pytest.mark.parametrize("precision,order", [(0, 6), (1, 6), (0, 4), (1, 4)])
def test_single_particle(hg, precision, order):
    """Degenerate system: no forces, the criterion has a zero denominator
    (infinite step, clamped to dt_max), free motion is exact; an empty
    evaluation and correction (m = 0) are accepted."""
    o = hg.hg_default_opts(dt_max=DT_MAX, precision=precision, order=order)
    ctx = hg.hg_init(np.array([1.0]), np.zeros((1, 3)), np.array([[0.5, 0.0, 0.0]]), 1e-3, 0.45, o)
    try:
        got, _ = gpu_state(hg, ctx, 1)
        assert np.all(got["acc"] == 0) and got["dt"][0] == DT_MAX
        hg.hg_advance(ctx, 0.5)
        got, t = gpu_state(hg, ctx, 1)
        assert t == 0.5 and got["pos"][0, 0] == pytest.approx(0.25, rel=1e-15)
        assert got["dt"][0] == DT_MAX and np.all(got["acc"] == 0)
        hg.hg_predict(ctx, 0.5)
        hg.hg_evaluate(ctx, np.empty(0, dtype=np.int32), 0)
        hg.hg_correct(ctx, None, 0)
        assert gpu_state(hg, ctx, 1)[1] == 0.5
    finally:
        hg.hg_free(ctx)


# --------------------------------------------------------------------------
# Errors are reported, never silently accepted; the state is left unchanged.
# --------------------------------------------------------------------------
def test_error_paths(hg):
    n = 64
    sysm = oracle_system(n, 5, 1e-3, steps=1)
    ctx = gpu_context(hg, sysm, 0, 1e-3)
    try:
        before, _ = gpu_state(hg, ctx, n)
        with pytest.raises(hg.HGError) as e:
            hg.hg_evaluate(ctx, np.array([0, 1], dtype=np.int32), 2)
        assert e.value.code == hg.HG_ESTATE
        hg.hg_predict(ctx, sysm.t_sys)
        for bad in ([1, 0], [0, 0], [-1, 2], [0, n]):
            with pytest.raises(hg.HGError) as e:
                hg.hg_evaluate(ctx, np.array(bad, dtype=np.int32), len(bad))
            assert e.value.code == hg.HG_EINVAL
        with pytest.raises(hg.HGError) as e:
            hg.hg_correct(ctx, None, 2)
        assert e.value.code == hg.HG_ESTATE
        # a particle that is not due at the prediction time
        st = sysm.get_state()
        not_due = int(np.argmax(st["t"] + st["dt"] != sysm.t_sys + 1.0))
        t_wrong = st["t"][not_due] + st["dt"][not_due] + 1.0
        hg.hg_predict(ctx, t_wrong)
        hg.hg_evaluate(ctx, np.array([not_due], dtype=np.int32), 1)
        with pytest.raises(hg.HGError) as e:
            hg.hg_correct(ctx, None, 1)
        assert e.value.code == hg.HG_ESTATE
        small = np.empty(0, dtype=np.int32)
        tn, m = hg.hg_next_block(ctx)
        if m > 0:
            with pytest.raises(hg.HGError) as e:
                hg.hg_next_block(ctx, small)
            assert e.value.code == hg.HG_EINVAL
        bad = {f: st[f].copy() for f in hg.STATE_FIELDS}
        bad["dt"][3] = 0.03
        with pytest.raises(hg.HGError) as e:
            hg.hg_set_state(ctx, bad, st["t_sys"])
        assert e.value.code == hg.HG_EINVAL
        after, _ = gpu_state(hg, ctx, n)
        for f in hg.STATE_FIELDS:
            np.testing.assert_array_equal(before[f], after[f], err_msg=f)
    finally:
        hg.hg_free(ctx)
    with pytest.raises(hg.HGError) as e:
        hg.hg_init(np.array([1.0, -1.0]), np.zeros((2, 3)), np.zeros((2, 3)), 1e-3, 0.45)
    assert e.value.code == hg.HG_EINVAL
    with pytest.raises(hg.HGError):
        hg.hg_init(np.array([1.0]), np.zeros((1, 3)), np.zeros((1, 3)), -1.0, 0.45)
    with pytest.raises(hg.HGError):
        hg.hg_init(np.array([1.0]), np.zeros((1, 3)), np.zeros((1, 3)), 1e-3, 0.45,
                   hg.hg_default_opts(dt_max=0.1))


def test_device_pointers_and_torch_stream(hg):
    import torch
    n, eps = 500, 1e-3
    sysm = oracle_system(n, 13, eps, steps=2)
    stream = torch.cuda.Stream()
    ctx = gpu_context(hg, sysm, 1, eps, stream=stream)
    try:
        idx = torch.arange(0, n, 7, dtype=torch.int32, device="cuda")
        m = idx.numel()
        out = [torch.empty((m, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
        t = sysm.t_sys + 1.0 / 128
        hg.hg_predict(ctx, t)
        hg.hg_evaluate(ctx, idx, m, *out)
        stream.synchronize()
        ref = sysm.predict_eval(t, idx.cpu().numpy())
        check_eval([o.cpu().numpy() for o in out], ref, 1, sysm.predict_absum(t, idx.cpu().numpy()))
    finally:
        hg.hg_free(ctx)


def test_condition_scale_of_the_mixed_evaluation(hg):
    """hg_condition_scale returns, per evaluated particle, sum_{j != i} m_j /
    (r_ij^2 + eps^2) over the predicted data (the definition, summed here in
    numpy from the oracle's prediction), which bounds the oracle's sum_j |a_ij|
    from above; FP64 contexts do not form it."""
    n, eps = 3001, 1e-3
    sysm = oracle_system(n, 24, eps, steps=2)
    t = sysm.t_sys + 1.0 / 512
    idx = np.arange(5, n, 11)
    st = sysm.get_state()
    xp, _, _ = oracle.predict(st["pos"], st["vel"], st["acc"], st["jerk"], st["snap"], st["crackle"], st["t"], t)
    ctx = gpu_context(hg, sysm, 1, eps)
    try:
        gpu_eval(hg, ctx, idx, t)
        sc = hg.hg_condition_scale(ctx, len(idx))
        with pytest.raises(hg.HGError) as e:
            hg.hg_condition_scale(ctx, len(idx) - 1)
        assert e.value.code == hg.HG_EINVAL
    finally:
        hg.hg_free(ctx)
    for q, i in enumerate(idx):
        d2 = np.sum((xp - xp[i]) ** 2, axis=1) + eps * eps
        mask = np.arange(n) != i
        ref = np.sum(st["mass"][mask] / d2[mask])
        assert abs(sc[q] - ref) <= 1e-5 * ref, (q, sc[q], ref)
    absum = sysm.predict_absum(t, idx)[:, 0]
    assert np.all(sc >= absum * (1 - 1e-5))
    ctx = gpu_context(hg, sysm, 0, eps)
    try:
        gpu_eval(hg, ctx, idx, t)
        with pytest.raises(hg.HGError) as e:
            hg.hg_condition_scale(ctx, len(idx))
        assert e.value.code == hg.HG_ESTATE
    finally:
        hg.hg_free(ctx)
