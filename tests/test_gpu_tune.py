"""Autotuning of the evaluation plan (hg_tune / hg_get_tuning / hg_set_tuning).

Tuning changes only how the work is spread over the GPU, never what is
computed: every tuned or forced table must give the oracle's results within the
path's tolerance, leave the integration state untouched, and drive the graph-
replayed block steps (which read the table on the device).
"""
import numpy as np
import pytest

from gpu_util import DT_MAX, DT_MIN, gpu_context, gpu_eval, gpu_state, oracle_system, rel_rows
from test_gpu_batch import _clusters
from test_gpu_parity import check_eval

pytestmark = pytest.mark.gpu

EPS = 1e-3


def _lists(n, rng):
    out = [np.arange(n)]
    for m in (1, 2, 3, 7, 40, 129, 600):
        if m < n:
            out.append(np.sort(rng.choice(n, m, replace=False)))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_tune_report_and_state_unchanged(hg, precision):
    n = 3001
    sysm = oracle_system(n, 71, EPS, steps=2)
    ctx = gpu_context(hg, sysm, precision, EPS)
    try:
        before, t0 = gpu_state(hg, ctx, n)
        rep = hg.hg_tune(ctx, m_max=1024)
        assert [e["bucket"] for e in rep] == list(range(11))
        table = hg.hg_get_tuning(ctx)
        for e in rep:
            assert e["m"] == (1 if e["bucket"] == 0 else min(1024, 3 << (e["bucket"] - 1)))
            assert e["candidates"] >= 2 and e["model_us"] > 0 and 0 < e["best_us"] <= e["model_us"]
            assert table[e["bucket"]] == e["chosen"]
            if e["chosen"] >= 0:
                assert e["best_us"] < 0.97 * e["model_us"]
        assert np.all(table[11:] == -1)
        after, t1 = gpu_state(hg, ctx, n)
        assert t1 == t0
        for f in hg.STATE_FIELDS:
            np.testing.assert_array_equal(after[f], before[f])
        # evaluations with the tuned table still match the oracle
        t = sysm.t_sys + 1.0 / 256
        for idx in _lists(n, np.random.default_rng(3)):
            got = gpu_eval(hg, ctx, idx, t)
            ref = sysm.predict_eval(t, idx.astype(np.int32))
            check_eval(got, ref, precision, sysm.predict_absum(t, idx.astype(np.int32)))
    finally:
        hg.hg_free(ctx)


@pytest.mark.parametrize("code", [0, 33, 70, 131, 165, 194])
def test_forced_table_matches_oracle_fp64(hg, code):
    """Every bucket forced to one plan (tpi 1..64, various j-splits): FP64 parity."""
    n = 1000
    sysm = oracle_system(n, 72, EPS, steps=2)
    ctx = gpu_context(hg, sysm, 0, EPS)
    try:
        hg.hg_set_tuning(ctx, np.full(hg.HG_TUNE_BUCKETS, code, dtype=np.int16))
        assert np.all(hg.hg_get_tuning(ctx) == code)
        t = sysm.t_sys + 1.0 / 128
        for idx in _lists(n, np.random.default_rng(code)):
            got = gpu_eval(hg, ctx, idx, t)
            check_eval(got, sysm.predict_eval(t, idx.astype(np.int32)), 0)
    finally:
        hg.hg_free(ctx)


def test_graph_steps_follow_the_table(hg):
    """Graph-replayed block steps with a forced table equal the explicit calls
    with the same table (bitwise: same plans, same summation order), and stay
    within rounding of the untuned run."""
    n = 1024
    sysm = oracle_system(n, 73, EPS, steps=1)
    table = np.full(hg.HG_TUNE_BUCKETS, 4 * 32 + 2, dtype=np.int16)   # tpi 16, 3 tiles per chunk
    a = gpu_context(hg, sysm, 0, EPS)
    b = gpu_context(hg, sysm, 0, EPS)
    u = gpu_context(hg, sysm, 0, EPS)
    try:
        def explicit_step():
            t, m = hg.hg_next_block(b)
            hg.hg_predict(b, t)
            hg.hg_evaluate(b, None, m)
            hg.hg_correct(b, None, m)

        hg.hg_step(a, 1)              # graphs captured before the table is set ...
        explicit_step()
        hg.hg_set_tuning(a, table)    # ... must be rebuilt with it
        hg.hg_set_tuning(b, table)
        hg.hg_step(a, 19)
        hg.hg_step(u, 20)
        for _ in range(19):
            explicit_step()
        sa, ta = gpu_state(hg, a, n)
        sb, tb = gpu_state(hg, b, n)
        su, tu = gpu_state(hg, u, n)
        assert ta == tb == tu
        for f in hg.STATE_FIELDS:
            np.testing.assert_array_equal(sa[f], sb[f], err_msg=f)
        assert rel_rows(sa["pos"], su["pos"]).max() < 1e-12
    finally:
        for c in (a, b, u):
            hg.hg_free(c)


def test_batch_tuning(hg):
    """Cluster contexts: every batch code gives each cluster its oracle result
    (FP64), hg_tune stores only batch codes, and plan indices are rejected."""
    import oracle
    parts, off, mass, pos, vel = _clusters()
    ctx = hg.hg_init_batch(off, mass, pos, vel, EPS, 0.45,
                           hg.hg_default_opts(precision=0, dt_min=DT_MIN, dt_max=DT_MAX))
    systems = [oracle.System(p.mass, p.pos, p.vel, EPS, 0.45, 0.01, DT_MIN, DT_MAX) for p in parts]
    try:
        with pytest.raises(hg.HGError):
            hg.hg_set_tuning(ctx, np.full(hg.HG_TUNE_BUCKETS, 100, dtype=np.int16))
        rep = hg.hg_tune(ctx)
        assert rep and all(e["model"] == 9 for e in rep)
        table = hg.hg_get_tuning(ctx)
        assert all(v == -1 or ((v & 7) <= 6 and (v >> 3) <= 2) for v in table)
        rng = np.random.default_rng(5)
        idx = np.sort(rng.choice(off[-1], 700, replace=False)).astype(np.int32)
        for code in (0, 6, 8 + 3, 16 + 6, 16):
            hg.hg_set_tuning(ctx, np.full(hg.HG_TUNE_BUCKETS, code, dtype=np.int16))
            t = 1.0 / 1024
            acc, jerk, snap = gpu_eval(hg, ctx, idx, t)
            for c, s in enumerate(systems):
                sel = (idx >= off[c]) & (idx < off[c + 1])
                if not sel.any() or s.n == 1:
                    continue
                ref = s.predict_eval(t, (idx[sel] - off[c]).astype(np.int32))
                check_eval([acc[sel], jerk[sel], snap[sel]], ref, 0)
    finally:
        hg.hg_free(ctx)


def test_tune_rejects_bad_arguments(hg):
    sysm = oracle_system(64, 74, EPS)
    ctx = gpu_context(hg, sysm, 1, EPS)
    try:
        with pytest.raises(hg.HGError):
            hg.hg_tune(ctx, reps=-1)
        for bad in (224, -2, 5000):   # plans [0, 224)
            with pytest.raises(hg.HGError):
                hg.hg_set_tuning(ctx, np.full(hg.HG_TUNE_BUCKETS, bad, dtype=np.int16))
        assert np.all(hg.hg_get_tuning(ctx) == -1)
    finally:
        hg.hg_free(ctx)
    ctx = gpu_context(hg, sysm, 0, EPS)
    try:
        with pytest.raises(hg.HGError):   # FP64: one kernel, plans [0, 224)
            hg.hg_set_tuning(ctx, np.full(hg.HG_TUNE_BUCKETS, 224, dtype=np.int16))
    finally:
        hg.hg_free(ctx)


@pytest.mark.parametrize("code", [0, 33, 70, 131, 165, 194])
def test_forced_table_matches_oracle_mixed(hg, code):
    """The mixed kernel under forced plans (threads per i-particle 1 to 64,
    short and long j-chunks): the mixed tolerances against the oracle."""
    n = 1000
    sysm = oracle_system(n, 75, EPS, steps=2)
    ctx = gpu_context(hg, sysm, 1, EPS)
    try:
        hg.hg_set_tuning(ctx, np.full(hg.HG_TUNE_BUCKETS, code, dtype=np.int16))
        t = sysm.t_sys + 1.0 / 128
        for idx in _lists(n, np.random.default_rng(code)):
            got = gpu_eval(hg, ctx, idx, t)
            i32 = idx.astype(np.int32)
            check_eval(got, sysm.predict_eval(t, i32), 1, sysm.predict_absum(t, i32))
    finally:
        hg.hg_free(ctx)
