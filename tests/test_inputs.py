"""Seeded input generators: splitmix64 reference values and workload statistics."""
import math

import numpy as np

from paper_1207_2367_gb300 import inputs


def test_splitmix64_reference_sequence():
    # First outputs of splitmix64 seeded with 1234567 (Vigna's reference implementation).
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert [int(x) for x in inputs.splitmix64_sequence(1234567, 5)] == ref


def test_uniform_range_and_independence_of_streams():
    u = inputs.uniform(3, np.arange(100000), 0)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    v = inputs.uniform(3, np.arange(100000), 1)
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.01


def test_plummer_deterministic_and_centred():
    a = inputs.plummer(2000, 9)
    b = inputs.plummer(2000, 9)
    np.testing.assert_array_equal(a.pos, b.pos)
    np.testing.assert_array_equal(a.vel, b.vel)
    assert abs(a.mass.sum() - 1.0) < 1e-14
    assert np.abs((a.mass[:, None] * a.pos).sum(0)).max() < 1e-14
    assert np.abs((a.mass[:, None] * a.vel).sum(0)).max() < 1e-14
    # a subset of the same seed is the prefix's own draws: streams are per particle
    c = inputs.plummer(1000, 9, henon=False)
    assert c.pos.shape == (1000, 3)


def test_plummer_radial_profile():
    """Median radius of a b = 1 Plummer sphere: X = 1/2 gives r = (2^(2/3) - 1)^(-1/2)."""
    p = inputs.plummer(200000, 2, henon=False)
    r = np.linalg.norm(p.pos, axis=1)
    r_half = 1.0 / math.sqrt((0.5 / 0.999) ** (-2.0 / 3.0) - 1.0)   # median of X in (0, 0.999]
    assert abs(np.median(r) - r_half) / r_half < 0.01


def test_salpeter_range_and_slope():
    m = inputs.salpeter_masses(200000, 3)
    assert abs(m.sum() - 1.0) < 1e-12
    raw = m / m.min()
    assert raw.max() <= 1000.0 * 1.0001
    # fraction of stars above 1 Msun for dN/dm ~ m^-2.35 on [0.1, 100]
    p = -1.35
    frac = (100 ** p - 1.0) / (100 ** p - 0.1 ** p)
    # masses are normalised; recover the solar unit from the smallest draw (~0.1)
    m_unit = m / (m.min() / 0.1)
    assert abs((m_unit > 1.0).mean() - frac) < 0.005


def test_cluster_batch_sizes():
    sizes = inputs.cluster_sizes(512, 4)
    assert sizes.min() >= 256 and sizes.max() <= 16384
    assert 2500 < sizes.mean() < 5500


def test_plummer_black_hole():
    p = inputs.plummer_black_hole(1001, 3, m_bh=0.02)
    assert p.mass.shape == (1001,) and p.mass[-1] == 0.02
    assert abs(p.mass[:-1].sum() - 1.0) < 1e-14
    mt = p.mass.sum()
    assert np.abs((p.mass[:, None] * p.pos).sum(0) / mt).max() < 1e-15
    assert np.abs((p.mass[:, None] * p.vel).sum(0) / mt).max() < 1e-15
    # the stars are the plain Plummer sphere of n - 1, shifted by the centre of mass
    s = inputs.plummer(1000, 3)
    np.testing.assert_allclose(p.pos[:-1] - p.pos[-1], s.pos, atol=1e-15)
