"""The fused block-step kernel: one cooperative launch runs all the block steps
of a graph (selection and prediction, evaluation, j-split reduction,
correction with the next block time), the passes separated by grid-wide
barriers instead of kernel boundaries.  It runs the same device code with the
same launch plans as the separate kernels, so every state it produces is
bitwise the separate kernels' -- and, through them, the explicit calls' and the
oracle's within the parity metric."""
import numpy as np
import pytest

from gpu_util import DT_MAX, gpu_context, gpu_state, oracle_system

pytestmark = pytest.mark.gpu


def _pair(hg, sysm, precision, eps, **opt):
    return [gpu_context(hg, sysm, precision, eps, fused_steps=f, **opt) for f in (1, -1)]


def _same_state(hg, a, b, n):
    sa, ta = gpu_state(hg, a, n)
    sb, tb = gpu_state(hg, b, n)
    assert ta == tb
    for f in hg.STATE_FIELDS:
        np.testing.assert_array_equal(sa[f], sb[f], err_msg=f)
    qa, qb = hg.hg_get_stats(a), hg.hg_get_stats(b)
    for k in ("block_steps", "interactions", "last_m", "t_sys"):
        assert qa[k] == qb[k], k


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [777, 5000])
def test_fused_steps_equal_separate_kernels_bitwise(hg, precision, n):
    eps = 1e-3
    sysm = oracle_system(n, 50 + n, eps, steps=1)
    a, b = _pair(hg, sysm, precision, eps, graph_steps=8)
    try:
        hg.hg_step(a, 37)          # 4 graphs of 8 steps and 5 graphs of 1
        hg.hg_step(b, 37)
        _same_state(hg, a, b, n)
        assert hg.hg_get_stats(a)["kernels"] < hg.hg_get_stats(b)["kernels"]   # one launch per graph
    finally:
        hg.hg_free(a)
        hg.hg_free(b)


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_advance_stops_at_t_end(hg, precision):
    n, eps = 2000, 1e-3
    sysm = oracle_system(n, 51, eps, steps=0)
    a, b = _pair(hg, sysm, precision, eps)
    try:
        ka = hg.hg_advance(a, 1.0 / 32)
        kb = hg.hg_advance(b, 1.0 / 32)
        assert ka == kb > 0
        _same_state(hg, a, b, n)
        st, t = gpu_state(hg, a, n)
        assert t == 1.0 / 32 and np.all(st["t"] == 1.0 / 32)
    finally:
        hg.hg_free(a)
        hg.hg_free(b)


def test_fused_zero_softening_and_fourth_order(hg):
    """eps = 0 (the guarded evaluation that skips the own pair) and the p = 4
    scheme through the fused kernel."""
    n = 600
    sysm = oracle_system(n, 52, 0.0, steps=0)
    for opt in ({"order": 6}, {"order": 4}):
        a, b = _pair(hg, sysm, 1, 0.0, **opt)
        try:
            hg.hg_step(a, 20)
            hg.hg_step(b, 20)
            _same_state(hg, a, b, n)
        finally:
            hg.hg_free(a)
            hg.hg_free(b)


def test_fused_option_checks(hg):
    from paper_1207_2367_gb300 import inputs
    p = inputs.plummer(64, 53)
    for bad in (dict(fused_steps=1, profile=1), dict(fused_steps=2)):
        with pytest.raises(hg.HGError) as e:
            hg.hg_init(p.mass, p.pos, p.vel, 1e-3, 0.45, hg.hg_default_opts(dt_max=DT_MAX, **bad))
        assert e.value.code == hg.HG_EINVAL
