"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: derivatives
of the force along prescribed trajectories (mpmath, 40 digits), the closed-form
Kepler orbit, Newton's third law, exactness on polynomials, hand-computed step
values, the analytic Plummer energy and 6th-order convergence.
"""
import json
import math
import os

import mpmath as mp
import numpy as np
import pytest

import oracle
from paper_1207_2367_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(12345)


def rel(x, ref):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(ref)) / np.linalg.norm(ref))


# --------------------------------------------------------------------------
# Evaluation step (Sect. 3 item 2): jerk and snap are the 1st and 2nd time
# derivatives of the softened acceleration along the trajectories.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_eval_matches_mpmath_derivatives_of_acceleration(eps):
    mp.mp.dps = 40
    n = 4
    c0 = rng.normal(size=(n, 3)) * 1.5
    c1 = rng.normal(size=(n, 3))
    c2 = rng.normal(size=(n, 3))
    c3 = rng.normal(size=(n, 3))
    mass = rng.uniform(0.2, 1.0, size=n)
    t0 = mp.mpf("0.37")

    def pos(k, d, t):
        return (mp.mpf(c0[k, d]) + mp.mpf(c1[k, d]) * t + mp.mpf(c2[k, d]) * t ** 2 / 2
                + mp.mpf(c3[k, d]) * t ** 3 / 6)

    def acc(i, d, t):
        tot = mp.mpf(0)
        for j in range(n):
            if j == i:
                continue
            r = [pos(j, e, t) - pos(i, e, t) for e in range(3)]
            r2 = sum(x * x for x in r) + mp.mpf(eps) ** 2
            tot += mp.mpf(mass[j]) * r[d] / r2 ** mp.mpf(1.5)
        return tot

    tf = float(t0)
    xp = c0 + c1 * tf + c2 * tf ** 2 / 2 + c3 * tf ** 3 / 6
    vp = c1 + c2 * tf + c3 * tf ** 2 / 2
    ap = c2 + c3 * tf
    A, J, S = oracle.evaluate(mass, xp, vp, ap, eps)
    for i in range(n):
        a_ref = [float(acc(i, d, t0)) for d in range(3)]
        j_ref = [float(mp.diff(lambda t: acc(i, d, t), t0, 1)) for d in range(3)]
        s_ref = [float(mp.diff(lambda t: acc(i, d, t), t0, 2)) for d in range(3)]
        assert rel(A[i], a_ref) < 1e-13
        assert rel(J[i], j_ref) < 1e-12
        assert rel(S[i], s_ref) < 1e-12


def _kepler(t, e=0.5, a=1.0, mt=1.0, prec=None):
    """Relative position of a Kepler orbit started at pericentre (closed form)."""
    M = mp.sqrt(mt / a ** 3) * t
    E = M
    for _ in range(60):
        E = E - (E - e * mp.sin(E) - M) / (1 - e * mp.cos(E))
    return [a * (mp.cos(E) - e), a * mp.sqrt(1 - e * e) * mp.sin(E), mp.mpf(0)]


def test_eval_matches_kepler_closed_form():
    """Two bodies on an e = 0.5 orbit: acc, jerk, snap of body 2 equal the 2nd, 3rd
    and 4th time derivatives of its closed-form position (eps = 0)."""
    mp.mp.dps = 40
    e, m1, m2 = mp.mpf("0.5"), mp.mpf("0.3"), mp.mpf("0.7")
    mt = m1 + m2
    t0 = mp.mpf("1.1")

    def body2(d, t):
        return m1 / mt * _kepler(t, e, 1, mt)[d]

    def body1(d, t):
        return -m2 / mt * _kepler(t, e, 1, mt)[d]

    xp = np.array([[float(body1(d, t0)) for d in range(3)], [float(body2(d, t0)) for d in range(3)]])
    vp = np.array([[float(mp.diff(lambda t: body1(d, t), t0, 1)) for d in range(3)],
                   [float(mp.diff(lambda t: body2(d, t), t0, 1)) for d in range(3)]])
    ap = np.array([[float(mp.diff(lambda t: body1(d, t), t0, 2)) for d in range(3)],
                   [float(mp.diff(lambda t: body2(d, t), t0, 2)) for d in range(3)]])
    A, J, S = oracle.evaluate(np.array([float(m1), float(m2)]), xp, vp, ap, 0.0)
    for k, body in enumerate((body1, body2)):
        for order, got in ((2, A), (3, J), (4, S)):
            ref = [float(mp.diff(lambda t: body(d, t), t0, order)) for d in range(2)] + [0.0]
            assert rel(got[k], ref) < 1e-12, (k, order)


def test_newton_third_law_all_active():
    p = inputs.plummer(96, 7, imf="salpeter")
    ap = rng.normal(size=(96, 3))
    A, J, S = oracle.evaluate(p.mass, p.pos, p.vel, ap, 1e-3)
    for q in (A, J, S):
        tot = (p.mass[:, None] * q).sum(axis=0)
        scale = (p.mass[:, None] * np.abs(q)).sum()
        assert np.abs(tot).max() < 1e-14 * scale


def test_condition_scale_equals_norm_when_terms_are_aligned():
    """sum_j |a_ij| equals |a_i| when every pair term points the same way (particle
    at the end of a line of others), and exceeds it otherwise (triangle inequality)."""
    m = np.array([0.5, 0.25, 0.25])
    x = np.array([[0.0, 0, 0], [1.0, 0, 0], [3.0, 0, 0]])
    v = np.array([[0.0, 0, 0], [0.0, 0.5, 0], [0.0, -0.25, 0]])
    a = np.zeros((3, 3))
    A, J, S = oracle.evaluate(m, x, v, a, 0.0)
    sc = oracle.eval_absum(m, x, v, a, 0.0)
    assert sc[0, 0] == pytest.approx(np.linalg.norm(A[0]), rel=1e-15)
    assert sc[0, 0] == pytest.approx(0.25 / 1.0 + 0.25 / 9.0, rel=1e-15)
    assert sc[1, 0] == pytest.approx(0.5 / 1.0 + 0.25 / 4.0, rel=1e-15)   # opposite terms
    assert sc[1, 0] > np.linalg.norm(A[1])
    assert np.all(sc[:, 1] >= np.linalg.norm(J, axis=1) * (1 - 1e-15))
    assert np.all(sc[:, 2] >= np.linalg.norm(S, axis=1) * (1 - 1e-15))


@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_condition_scale_columns_equal_mpmath_pair_derivatives(eps):
    """The condition scale (acc, jerk and snap columns) sums over j of the norms of
    each pair's acceleration m_j r_ij / (r_ij^2 + eps^2)^(3/2) and of its 1st and
    2nd time derivatives along prescribed cubic trajectories (mpmath, 40 digits):
    the pair terms whose sums are acc, jerk and snap."""
    mp.mp.dps = 40
    n = 4
    c0 = rng.normal(size=(n, 3)) * 1.5
    c1 = rng.normal(size=(n, 3))
    c2 = rng.normal(size=(n, 3))
    c3 = rng.normal(size=(n, 3))
    mass = rng.uniform(0.2, 1.0, size=n)
    t0 = mp.mpf("0.29")

    def pos(k, d, t):
        return (mp.mpf(c0[k, d]) + mp.mpf(c1[k, d]) * t + mp.mpf(c2[k, d]) * t ** 2 / 2
                + mp.mpf(c3[k, d]) * t ** 3 / 6)

    def pair_acc(i, j, d, t):
        r = [pos(j, e, t) - pos(i, e, t) for e in range(3)]
        r2 = sum(x * x for x in r) + mp.mpf(eps) ** 2
        return mp.mpf(mass[j]) * r[d] / r2 ** mp.mpf(1.5)

    tf = float(t0)
    xp = c0 + c1 * tf + c2 * tf ** 2 / 2 + c3 * tf ** 3 / 6
    vp = c1 + c2 * tf + c3 * tf ** 2 / 2
    ap = c2 + c3 * tf
    sc = oracle.eval_absum(mass, xp, vp, ap, eps)
    for i in range(n):
        ref = np.zeros(3)
        for j in range(n):
            if j == i:
                continue
            for col, order in ((0, 0), (1, 1), (2, 2)):
                vec = [mp.diff(lambda t: pair_acc(i, j, d, t), t0, order) if order else pair_acc(i, j, d, t0)
                       for d in range(3)]
                ref[col] += float(mp.sqrt(sum(x * x for x in vec)))
        for col in range(3):
            assert abs(sc[i, col] - ref[col]) <= 1e-12 * ref[col], (i, col, sc[i, col], ref[col])


def test_eval_subset_equals_full_rows_and_skips_self():
    p = inputs.plummer(50, 3)
    ap = rng.normal(size=(50, 3))
    full = oracle.evaluate(p.mass, p.pos, p.vel, ap, 0.0)
    idx = np.array([0, 7, 49], dtype=np.int32)
    sub = oracle.evaluate(p.mass, p.pos, p.vel, ap, 0.0, idx)
    for f, s in zip(full, sub):
        np.testing.assert_array_equal(f[idx], s)
        assert np.all(np.isfinite(s))


# --------------------------------------------------------------------------
# Predictor, corrector and interpolation on polynomial motion.
# --------------------------------------------------------------------------
def _poly(coef, t, der=0):
    """Sum_k coef[k] t^k / k!, differentiated der times; coef [deg+1, 3]."""
    out = np.zeros(3)
    for k in range(der, coef.shape[0]):
        out += coef[k] * t ** (k - der) / math.factorial(k - der)
    return out


def test_predictor_exact_for_quintic_motion():
    coef = rng.normal(size=(6, 3))
    t0, t1 = 0.25, 0.3125
    d = [_poly(coef, t0, k)[None] for k in range(6)]
    xp, vp, ap = oracle.predict(*d, np.array([t0]), t1)
    for got, k in ((xp, 0), (vp, 1), (ap, 2)):
        assert rel(got[0], _poly(coef, t1, k)) < 1e-14


def test_predictor_truncates_after_crackle():
    coef = np.zeros((7, 3))
    coef[6] = [1.0, 2.0, 3.0]                # only x^(6) nonzero: pop is not in the predictor
    xp, vp, ap = oracle.predict(*[np.zeros((1, 3))] * 6, np.array([0.0]), 0.5)
    assert np.all(xp == 0) and np.all(vp == 0) and np.all(ap == 0)


@pytest.mark.parametrize("deg_x,exact_v,exact_x", [(6, True, True), (7, True, False)])
def test_corrector_exactness(deg_x, exact_v, exact_x):
    """v_corr is exact when a(t) has degree <= 5, r_corr when x(t) has degree <= 6."""
    coef = rng.normal(size=(deg_x + 1, 3))
    h = 0.375
    x0, v0, a0, j0, s0 = (_poly(coef, 0.0, k) for k in range(5))
    a1, j1, s1 = (_poly(coef, h, k) for k in (2, 3, 4))
    x1, v1 = oracle.correct(h, x0, v0, a0, j0, s0, a1, j1, s1)
    ev, ex = rel(v1, _poly(coef, h, 1)), rel(x1, _poly(coef, h, 0))
    assert (ev < 1e-13) == exact_v, ev
    assert (ex < 1e-13) == exact_x, ex


def test_interpolation_exact_for_quintic_acceleration():
    ca = rng.normal(size=(6, 3))       # a(t) = sum ca[k] t^k/k!, degree 5
    h = 0.125
    a0, j0, s0 = (_poly(ca, 0.0, k) for k in range(3))
    a1, j1, s1 = (_poly(ca, h, k) for k in range(3))
    c1, p1, q1 = oracle.interp(h, a0, j0, s0, a1, j1, s1)
    assert rel(c1, _poly(ca, h, 3)) < 1e-10
    assert rel(p1, _poly(ca, h, 4)) < 1e-9
    assert rel(q1, _poly(ca, h, 5)) < 1e-8


@pytest.mark.parametrize("deg_x,exact_v,exact_x", [(4, True, True), (5, True, False), (6, False, False)])
def test_corrector4_exactness(deg_x, exact_v, exact_x):
    """4th-order corrector (two-point Hermite quadrature, exact for cubic
    integrands): v exact when a(t) has degree <= 3, x when x(t) has degree <= 4."""
    coef = rng.normal(size=(deg_x + 1, 3))
    h = 0.375
    x0, v0, a0, j0 = (_poly(coef, 0.0, k) for k in range(4))
    a1, j1 = (_poly(coef, h, k) for k in (2, 3))
    x1, v1 = oracle.correct4(h, x0, v0, a0, j0, a1, j1)
    ev, ex = rel(v1, _poly(coef, h, 1)), rel(x1, _poly(coef, h, 0))
    assert (ev < 1e-13) == exact_v, ev
    assert (ex < 1e-13) == exact_x, ex


def test_interpolation4_exact_for_cubic_acceleration():
    ca = rng.normal(size=(4, 3))       # a(t) = sum ca[k] t^k/k!, degree 3
    h = 0.125
    a0, j0 = (_poly(ca, 0.0, k) for k in range(2))
    a1, j1 = (_poly(ca, h, k) for k in range(2))
    s1, c1 = oracle.interp4(h, a0, j0, a1, j1)
    assert rel(s1, _poly(ca, h, 2)) < 1e-11
    assert rel(c1, _poly(ca, h, 3)) < 1e-10


def test_kepler_integration_fourth_order():
    """The p = 4 scheme converges at 4th order on the Kepler orbit (error ratio
    2^4 = 16 per halving of eta) and follows the closed form."""
    mp.mp.dps = 30
    p = inputs.kepler_pair()
    T = 8.0
    ref = np.array([float(x) for x in _kepler(mp.mpf(T))])
    errs = []
    for eta in (0.04, 0.02, 0.01):
        s = oracle.System(p.mass, p.pos, p.vel, 0.0, eta, eta_init=eta / 45, dt_max=1.0, order=4)
        s.advance(T)
        x = s.get("pos")
        errs.append(np.linalg.norm((x[1] - x[0]) - ref))
        assert np.all(s.get("snap") == 0) and np.all(s.get("crackle") == 0)
    assert errs[-1] < 1e-7
    for e1, e2 in zip(errs, errs[1:]):
        assert 10.0 < e1 / e2 < 25.0, errs      # 2^4 = 16


def test_energy_conservation_plummer_1024_fourth_order():
    p = inputs.plummer(1024, 1)
    s = oracle.System(p.mass, p.pos, p.vel, 1e-3, 0.15, 0.01, 2.0 ** -25, 1.0 / 16, order=4)
    E0 = sum(s.energy())
    s.advance(0.125)
    assert np.all(s.get("t") == 0.125)
    assert abs((sum(s.energy()) - E0) / E0) < 3e-8


# --------------------------------------------------------------------------
# Time steps and block selection (hand-computed golden cases).
# --------------------------------------------------------------------------
def test_criterion_golden():
    g = json.load(open(os.path.join(GOLDEN, "aarseth_criterion.json")))
    d = np.array(g["derivs"], dtype=float)
    for case in g["cases"]:
        p = case["p"]
        got = oracle.criterion(case["eta"], p, d[:p])
        assert got == pytest.approx(eval(case["expected"]), rel=1e-15), case["by_hand"]


def test_block_dt_golden():
    g = json.load(open(os.path.join(GOLDEN, "block_steps.json")))
    for c in g["block_dt"]:
        crit = math.inf if c["crit"] == "inf" else c["crit"]
        got = oracle.block_dt(crit, c["dt_old"], c["t_new"], c["dt_min"], c["dt_max"])
        assert got == c["expected"], c["why"]
    for c in g["block_dt_init"]:
        assert oracle.block_dt_init(c["crit"], c["dt_min"], c["dt_max"]) == c["expected"]
    nb = g["next_block"]
    tn, idx = oracle.next_block(np.array(nb["t"]), np.array(nb["dt"]))
    assert tn == nb["expected_t_next"]
    assert idx.tolist() == nb["expected_idx"]


def test_block_invariants_along_integration():
    p = inputs.plummer(128, 11)
    s = oracle.System(p.mass, p.pos, p.vel, 1e-3, 0.45, 0.01, 2.0 ** -25, 1.0 / 16)
    for _ in range(60):
        m, tn = s.step()
        assert m >= 1
        t, dt = s.get("t"), s.get("dt")
        assert np.all(np.fmod(t, dt) == 0.0)
        e = np.log2(dt)
        assert np.all(e == np.round(e)) and dt.max() <= 1.0 / 16 and dt.min() >= 2.0 ** -25
        assert np.all(t + dt > tn)
        assert np.all(t <= tn)


# --------------------------------------------------------------------------
# Energy (Sect. 2 softened potential; Sect. 5.1 error measure).
# --------------------------------------------------------------------------
def test_energy_two_body_by_hand():
    m = np.array([0.25, 0.75])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    K, W = oracle.energy(m, x, v, 0.0)
    assert K == pytest.approx(0.5 * 0.25 * 1.0 + 0.5 * 0.75 * 4.0, rel=1e-15)
    assert W == pytest.approx(-0.25 * 0.75 / 5.0, rel=1e-15)
    K, W = oracle.energy(m, x, v, 12.0)       # sqrt(25 + 144) = 13
    assert W == pytest.approx(-0.25 * 0.75 / 13.0, rel=1e-15)


def test_energy_plummer_henon_units():
    """Henon units: W = -1/2 and K = 1/4 analytically; sampling noise ~ N^-1/2."""
    p = inputs.plummer(4096, 5)
    K, W = oracle.energy(p.mass, p.pos, p.vel, 0.0)
    assert W == pytest.approx(-0.5, rel=0.06)
    assert K == pytest.approx(0.25, rel=0.06)


def test_energy_conservation_plummer_1024():
    p = inputs.plummer(1024, 1)
    s = oracle.System(p.mass, p.pos, p.vel, 1e-3, 0.45, 0.01, 2.0 ** -25, 1.0 / 16)
    E0 = sum(s.energy())
    s.advance(0.25)
    assert s.t_sys == 0.25
    assert np.all(s.get("t") == 0.25)
    E1 = sum(s.energy())
    assert abs((E1 - E0) / E0) < 1e-8


# --------------------------------------------------------------------------
# Angular momentum (Sect. 5.1 conservation check): hand value, the rigid-body
# identity L = I omega, and the Kepler orbit's closed form and conservation.
# --------------------------------------------------------------------------
def test_angular_momentum_two_body_by_hand():
    m = np.array([0.25, 0.75])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    # 0.75 * (3, 4, 0) x (0, 2, 0) = 0.75 * (0, 0, 6)
    np.testing.assert_allclose(oracle.angular_momentum(m, x, v), [0.0, 0.0, 4.5], rtol=0, atol=1e-15)


def test_angular_momentum_rigid_rotation_is_inertia_times_omega():
    p = inputs.plummer(500, 7)
    omega = np.array([0.3, -1.1, 0.7])
    v = np.cross(omega, p.pos)                 # rigid rotation about the origin
    r2 = np.einsum("ij,ij->i", p.pos, p.pos)
    inertia = np.einsum("i,jk->jk", p.mass * r2, np.eye(3)) - np.einsum("i,ij,ik->jk", p.mass, p.pos, p.pos)
    np.testing.assert_allclose(oracle.angular_momentum(p.mass, p.pos, v), inertia @ omega, rtol=1e-13)


def test_angular_momentum_kepler_closed_form_and_conservation():
    e, a = 0.5, 1.0
    p = inputs.kepler_pair(e=e, a=a)
    mu = p.mass[0] * p.mass[1] / p.mass.sum()
    L0 = oracle.angular_momentum(p.mass, p.pos, p.vel)
    np.testing.assert_allclose(L0, [0.0, 0.0, mu * math.sqrt(p.mass.sum() * a * (1 - e * e))], rtol=1e-14)
    s = oracle.System(p.mass, p.pos, p.vel, 0.0, 0.1, eta_init=0.1 / 45, dt_max=1.0)
    s.advance(8.0)
    assert np.linalg.norm(s.angular_momentum() - L0) / np.linalg.norm(L0) < 1e-10


# --------------------------------------------------------------------------
# Whole integrator: Kepler orbit, 6th-order convergence.
# --------------------------------------------------------------------------
def test_kepler_integration_sixth_order():
    mp.mp.dps = 30
    p = inputs.kepler_pair()
    T = 8.0
    ref = np.array([float(x) for x in _kepler(mp.mpf(T))])
    errs = []
    for eta in (0.2, 0.1, 0.05):
        s = oracle.System(p.mass, p.pos, p.vel, 0.0, eta, eta_init=eta / 45, dt_max=1.0)
        s.advance(T)
        x = s.get("pos")
        errs.append(np.linalg.norm((x[1] - x[0]) - ref))
    assert errs[-1] < 1e-9
    for e1, e2 in zip(errs, errs[1:]):
        assert 40.0 < e1 / e2 < 100.0, errs      # 2^6 = 64
