"""The integer FP64 <-> FP32 conversions of the mixed path (hg_internal.cuh),
compiled for the host by a small probe (tests/host/conv_probe.cpp), against
IEEE-754 conversions (numpy): d2f rounds to nearest with ties to even, flushes
results below the smallest normal float (2^-126) to a zero of the same sign,
overflows to an infinity of the same sign, keeps infinities and turns NaN into
NaN; f2d widens exactly (subnormal floats, which the FP32 arithmetic flushes,
to zero) and keeps infinities and NaN."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("conv") / "conv_probe")
    subprocess.run(["g++", "-std=c++17", "-O1", "-x", "c++", "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1207_2367_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "conv_probe.cpp"), "-o", exe], check=True)

    def run(kind, bits):
        text = "".join(f"{kind} {int(b):x}\n" for b in bits)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
        return np.array([int(x, 16) for x in out.split()], dtype=np.uint64)
    return run


def _d2f_reference(x):
    with np.errstate(over="ignore"):
        r = x.astype(np.float32)
    tiny = np.abs(x) < np.float64(2.0 ** -126)
    return np.where(tiny, np.where(np.signbit(x), np.float32(-0.0), np.float32(0.0)), r)


def test_d2f_matches_ieee_rounding(probe):
    rng = np.random.default_rng(7)
    edge = np.array([0.0, -0.0, 1.0, -1.0, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 1 + 2.0 ** -24 + 2.0 ** -50,
                     np.finfo(np.float32).max, -np.finfo(np.float32).max,
                     float(np.finfo(np.float32).max) * (1 + 2.0 ** -25), float(np.finfo(np.float32).max) * (1 + 2.0 ** -23),
                     2.0 ** 128, -2.0 ** 128, 1e39, -1e300, np.finfo(np.float64).max, np.inf, -np.inf,
                     2.0 ** -126, -2.0 ** -126, 2.0 ** -127, 1e-40, 5e-324, 1e18, 3.0e38])
    rnd = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-40, 40, size=2000),
                          rng.uniform(-1, 1, size=1000)])
    x = np.concatenate([edge, rnd])
    got = probe("d", x.view(np.uint64)).astype(np.uint32).view(np.float32)
    ref = _d2f_reference(x)
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
    nan = probe("d", np.array([np.nan, -np.nan]).view(np.uint64)).astype(np.uint32).view(np.float32)
    assert np.all(np.isnan(nan))


def test_f2d_widens_exactly(probe):
    rng = np.random.default_rng(8)
    f = np.concatenate([np.array([0.0, -0.0, 1.0, np.finfo(np.float32).max, np.finfo(np.float32).tiny, np.inf,
                                  -np.inf, 1e-40, -1e-42], dtype=np.float32),
                        (rng.normal(size=2000) * 10.0 ** rng.integers(-37, 38, size=2000)).astype(np.float32)])
    got = probe("f", f.view(np.uint32)).view(np.float64)
    ref = f.astype(np.float64)
    ref = np.where(np.abs(f) < np.finfo(np.float32).tiny, np.copysign(0.0, ref), ref)
    np.testing.assert_array_equal(got.view(np.uint64), ref.view(np.uint64))
    nan = probe("f", np.array([np.nan], dtype=np.float32).view(np.uint32)).view(np.float64)
    assert np.isnan(nan[0])
