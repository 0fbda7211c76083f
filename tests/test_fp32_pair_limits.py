"""What FP32 pair arithmetic can resolve: the reason for the mixed path's metric.

The mixed evaluation forms every pair term of Sect. 3 item 2 in FP32 (position
differences in double-single).  Each term then carries a relative rounding
error of a few 1e-8 no matter how well it is summed, so a particle whose
acceleration is a near cancellation of its pair terms (condition number
kappa = sum_j |a_ij| / |a_i| >> 1) has a per-particle relative error of order
1e-8 kappa.  These tests emulate the FP32 pair terms in numpy (every operation
rounded to float32, the reciprocal square root correctly rounded, the terms
summed exactly) and compare with the FP64 oracle:
  - a constructed near cancellation (kappa ~ 1e4) misses 1e-6 per particle by
    orders of magnitude, while its error stays below 1e-6 of the condition
    scale sum_j |a_ij|;
  - on a Plummer sphere of N = 3001 the normwise error and the error against
    the condition scale stay below 1e-6, and the per-particle error follows
    kappa.
So per-particle 1e-6 is not a property any FP32 pair arithmetic has; the
parity tests of the mixed path bound the normwise error and the error relative
to the condition scale instead, plus the per-particle error of particles with
kappa <= 10 (99 % of a Plummer sphere's particles), where FP32 pair terms do
meet it.
"""
import numpy as np

import oracle
from paper_1207_2367_gb300 import inputs

f32 = np.float32


def _fma(a, b, c):
    """float32 fused multiply-add: the product of two floats is exact in float64."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def fp32_acc_terms(mass, x, eps, i):
    """Pair accelerations m_j r_ij / (r_ij^2 + eps^2)^(3/2) of particle i, j != i,
    with every operation rounded to float32 as the mixed kernel does: double-single
    position differences, r^2 by FMAs, 1/sqrt correctly rounded, q = m / r^3."""
    xh = x.astype(f32)
    xl = (x - xh.astype(np.float64)).astype(f32)
    keep = np.arange(x.shape[0]) != i
    d = ((xh[keep] - xh[i]) + (xl[keep] - xl[i])).astype(f32)          # [n-1, 3], each op rounded
    r2 = _fma(d[:, 2], d[:, 2], _fma(d[:, 1], d[:, 1], _fma(d[:, 0], d[:, 0], np.full(d.shape[0], eps * eps, f32))))
    y = (1.0 / np.sqrt(r2.astype(np.float64))).astype(f32)
    q = ((mass[keep].astype(f32) * (y * y)) * y).astype(f32)
    return (q[:, None] * d).astype(f32)


def exact_sum(terms):
    """Sum of float32 terms in float64: exact to far below the float32 rounding."""
    return terms.astype(np.float64).sum(axis=0)


def test_near_cancellation_defeats_per_particle_tolerance():
    # Particle 0 between two equal masses at almost mirror positions: the pulls
    # cancel to about 3e-5 of each.
    x1 = np.array([0.73151, 0.12113, -0.04337])
    x = np.stack([np.zeros(3), x1, -x1 * (1.0 + 1e-5)])
    mass = np.array([0.1, 0.5, 0.5])
    eps = 1e-4
    ref = oracle.evaluate(mass, x, np.zeros_like(x), np.zeros_like(x), eps, np.array([0]))[0][0]
    scale = oracle.eval_absum(mass, x, np.zeros_like(x), np.zeros_like(x), eps, np.array([0]))[0, 0]
    got = exact_sum(fp32_acc_terms(mass, x, eps, 0))
    err = np.linalg.norm(got - ref)
    kappa = scale / np.linalg.norm(ref)
    assert kappa > 1e4
    assert err / np.linalg.norm(ref) > 1e-4          # per-particle 1e-6 missed by orders of magnitude
    assert err / scale < 1e-6                        # the condition-scaled bound holds


def test_plummer_errors_follow_the_condition_number():
    n, eps = 3001, 1e-3
    p = inputs.plummer(n, 103)
    z = np.zeros((n, 3))
    ref = oracle.evaluate(p.mass, p.pos, z, z, eps)[0]
    scale = oracle.eval_absum(p.mass, p.pos, z, z, eps)[:, 0]
    got = np.stack([exact_sum(fp32_acc_terms(p.mass, p.pos, eps, i)) for i in range(n)])
    err = np.linalg.norm(got - ref, axis=1)
    refn = np.linalg.norm(ref, axis=1)
    per = err / refn
    kappa = scale / refn
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6     # normwise
    assert (err / scale).max() < 1e-6                                  # against the condition scale
    # The worst particles are the ill-conditioned ones: the per-particle error
    # divided by kappa is a few float32 roundings at most, and the largest
    # per-particle errors belong to particles with kappa well above the median.
    assert (per / kappa).max() < 1e-6
    # Up to kappa = 10 the per-particle tolerance itself holds, and such
    # particles are nearly all of the sphere, its centre included.
    assert per[kappa <= 10.0].max() < 1e-6
    assert (kappa <= 10.0).mean() > 0.98
    centre = np.argsort(np.linalg.norm(p.pos, axis=1))[: n // 20]
    assert (kappa[centre] <= 10.0).mean() > 0.9
    worst = np.argsort(per)[-10:]
    assert np.median(kappa[worst]) > 3.0 * np.median(kappa)
