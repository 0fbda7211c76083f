"""The checked build (-DHG_CHECKED): device bounds checks that report.

In the checked library every active-list entry, j-tile range and partial-sum
row the evaluation, reduction and correction kernels use is checked; a value
out of range is not used and the next synchronizing call returns HG_ECUDA, so
an indexing bug shows as an error instead of a memory fault (compute-sanitizer
is closed on this machine).  The GPU parity and batch suites run again in a fresh
process on that library and must pass there (no check fires on correct runs);
a list entry planted out of range through the testing hook is caught.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1207_2367_gb300 import inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suites_pass_on_the_checked_build():
    env = dict(os.environ, HG_LIB_VARIANT="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_parity.py", "tests/test_gpu_batch.py",
                        "tests/test_gpu_checked.py::test_planted_bad_index_is_reported"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout


def test_planted_bad_index_is_reported(hg):
    n = 2000
    p = inputs.plummer(n, 34)
    ctx = hg.hg_init(p.mass, p.pos, p.vel, 1e-3, 0.45, hg.hg_default_opts(precision=hg.HG_MIXED, dt_max=1.0 / 16))
    try:
        tn, m = hg.hg_next_block(ctx)
        assert m > 0
        hg.hg_predict(ctx, tn)
        if not hg.hg_build_checked():
            with pytest.raises(hg.HGError) as e:          # the normal build refuses the hook
                hg.hg_test_corrupt_list(ctx, 0, n + 7)
            assert e.value.code == hg.HG_EINVAL
            acc = np.empty((m, 3))
            hg.hg_evaluate(ctx, None, m, acc)               # and its list is intact
            assert np.all(np.isfinite(acc))
            return
        hg.hg_test_corrupt_list(ctx, 0, n + 7)
        with pytest.raises(hg.HGError) as e:
            hg.hg_evaluate(ctx, None, m)
        assert e.value.code == hg.HG_ECUDA and "bounds" in str(e.value)
    finally:
        hg.hg_free(ctx)
    ctx = hg.hg_init(p.mass, p.pos, p.vel, 1e-3, 0.45, hg.hg_default_opts(precision=hg.HG_MIXED, dt_max=1.0 / 16))
    hg.hg_step(ctx, 3)                                      # the GPU stays usable
    assert hg.hg_get_stats(ctx)["block_steps"] == 3
    hg.hg_free(ctx)
