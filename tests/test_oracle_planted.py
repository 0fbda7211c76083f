"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a scratch copy of oracle/hg_oracle.c (a dropped
term, a wrong coefficient, sign or index, a missing softening, a wrong power),
builds it separately and runs tests/test_oracle_pins.py against that build in a
subprocess: at least one pin must fail.  The unmodified copy must pass.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hg_oracle.c")

# (what the mistake is, text in the oracle, its replacement)
PLANTED = [
    ("snap loses its -3 beta a term", "- 3.0 * beta * aij;", ";"),
    ("6 alpha read as 3 alpha", "- 6.0 * alpha * jij", "- 3.0 * alpha * jij"),
    ("sign of the jerk's alpha term", "double jij = mass[j] * v[k] / r3 - 3.0", "double jij = mass[j] * v[k] / r3 + 3.0"),
    ("corrector h^2/10 read as h^2/12", "h * h / 10.0 * (j1[k] - j0[k])", "h * h / 12.0 * (j1[k] - j0[k])"),
    ("interpolation coefficient of crackle", "- 36.0 * J + 9.0 * S", "- 32.0 * J + 9.0 * S"),
    ("softening missing in alpha", "double alpha = dot3(r, v) / r2;", "double alpha = dot3(r, v) / (r2 - eps * eps);"),
    ("a_ij not differenced", "a[k] = ap[3 * j + k] - ap[3 * i + k];", "a[k] = ap[3 * j + k];"),
    ("predictor crackle term h^5/24", "c[q] * h5 / 120.0;", "c[q] * h5 / 24.0;"),
    ("potential counted half", "W -= mass[i] * mass[j]", "W -= 0.5 * mass[i] * mass[j]"),
    ("criterion exponent 1/2 for p = 6", "return eta * cbrt(ratio);", "return eta * sqrt(ratio);"),
    ("4th-order corrector h^2/12 read as h^2/10", "+ h * h / 12.0 * (j0[k] - j1[k]);", "+ h * h / 10.0 * (j0[k] - j1[k]);"),
    ("4th-order interpolation: crackle coefficient", "double c = (12.0 * (a0[k] - a1[k])", "double c = (10.0 * (a0[k] - a1[k])"),
    ("angular momentum component sign", "Lz += mass[i] * (r[0] * u[1] - r[1] * u[0]);",
     "Lz += mass[i] * (r[1] * u[0] - r[0] * u[1]);"),
    ("condition scale: snap term loses -3 beta A",
     "S[k] = mass[j] * a[k] / r3 - 6.0 * alpha * J[k] - 3.0 * beta * A[k];",
     "S[k] = mass[j] * a[k] / r3 - 6.0 * alpha * J[k];"),
    ("condition scale: sign of the jerk's alpha term", "J[k] = mass[j] * v[k] / r3 - 3.0 * alpha * A[k];",
     "J[k] = mass[j] * v[k] / r3 + 3.0 * alpha * A[k];"),
    ("condition scale: jerk and snap columns swapped", "out[3 * q + 1] = sj;\n        out[3 * q + 2] = ss;",
     "out[3 * q + 1] = ss;\n        out[3 * q + 2] = sj;"),
]


def _run_pins(tmp_path, text):
    src = tmp_path / "hg_oracle.c"
    src.write_text(text)
    so = tmp_path / "liboracle.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", str(src),
                    "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, HG_ORACLE_LIB=str(so))
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def original():
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    return open(SRC).read()


def test_unmodified_copy_passes(original, tmp_path):
    r = _run_pins(tmp_path, original)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("what,old,new", PLANTED, ids=[p[0] for p in PLANTED])
def test_planted_mistake_is_caught(original, tmp_path, what, old, new):
    assert old in original, f"the text to alter is not in the oracle: {old!r}"
    r = _run_pins(tmp_path, original.replace(old, new, 1))   # first occurrence: or_eval
    assert r.returncode != 0, f"no pin caught: {what}"
