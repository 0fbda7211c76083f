"""Independent clusters in one context (hg_init_batch).

Clusters are centred on the same point, so any interaction leaking between
clusters would change the results by orders of magnitude.  Each cluster is
checked against its own oracle system; the batched integration is checked
against separate contexts, one per cluster.
"""
import numpy as np
import pytest

import oracle
from paper_1207_2367_gb300 import inputs
from gpu_util import DT_MAX, DT_MIN, gpu_state, rel_rows
from test_gpu_parity import check_eval

pytestmark = pytest.mark.gpu

SIZES = [37, 300, 1, 1000, 513, 2]


def _clusters(sizes=SIZES, seed0=1000):
    parts = [inputs.plummer(s, seed0 + c) for c, s in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    cat = lambda f: np.ascontiguousarray(np.concatenate([getattr(p, f) for p in parts]))
    return parts, offsets, cat("mass"), cat("pos"), cat("vel")


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_evaluation_matches_each_cluster_oracle(hg, precision):
    eps = 1e-3
    parts, off, mass, pos, vel = _clusters()
    systems = [oracle.System(p.mass, p.pos, p.vel, eps, 0.45, 0.01, DT_MIN, DT_MAX) for p in parts]
    for s in systems:
        for _ in range(2):
            if s.n > 1:
                s.step()
    # inject the oracle states (each cluster at its own times) into one batch context
    sts = [s.get_state() for s in systems]
    state = {f: np.ascontiguousarray(np.concatenate([st[f] for st in sts])) for f in hg.STATE_FIELDS}
    ctx = hg.hg_init_batch(off, mass, pos, vel, eps, 0.45,
                           hg.hg_default_opts(precision=precision, dt_min=DT_MIN, dt_max=DT_MAX, start_mode=1))
    try:
        hg.hg_set_state(ctx, state, 0.0)
        t = max(s.t_sys for s in systems) + 1.0 / 512
        rng = np.random.default_rng(precision)
        for idx in (np.arange(off[-1]), np.sort(rng.choice(off[-1], 400, replace=False))):
            idx = idx.astype(np.int32)
            m = len(idx)
            got = [np.empty((m, 3)) for _ in range(3)]
            hg.hg_predict(ctx, t)
            hg.hg_evaluate(ctx, idx, m, *got)
            ref = [np.empty((m, 3)) for _ in range(3)]
            scale = np.empty((m, 3))
            for c, s in enumerate(systems):
                sel = (idx >= off[c]) & (idx < off[c + 1])
                if not sel.any():
                    continue
                local = (idx[sel] - off[c]).astype(np.int32)
                for k, r in enumerate(s.predict_eval(t, local)):
                    ref[k][sel] = r
                scale[sel] = s.predict_absum(t, local)
            single = np.isin(idx, off[:-1][np.diff(off) == 1])   # one-particle clusters feel nothing
            for g in got:
                assert np.all(g[single] == 0.0)
            keep = ~single
            check_eval([g[keep] for g in got], [r[keep] for r in ref], precision, scale[keep])
    finally:
        hg.hg_free(ctx)


def test_batch_start_up_matches_oracle(hg):
    eps = 1e-3
    parts, off, mass, pos, vel = _clusters()
    ctx = hg.hg_init_batch(off, mass, pos, vel, eps, 0.45,
                           hg.hg_default_opts(precision=hg.HG_FP64, dt_min=DT_MIN, dt_max=DT_MAX))
    try:
        got, t = gpu_state(hg, ctx, int(off[-1]))
        assert t == 0.0
        for c, p in enumerate(parts):
            s = oracle.System(p.mass, p.pos, p.vel, eps, 0.45, 0.01, DT_MIN, DT_MAX)
            sl = slice(off[c], off[c + 1])
            if p.n > 1:
                for f in ("acc", "jerk", "snap"):
                    assert rel_rows(got[f][sl], s.get(f)).max() <= 1e-12, (c, f)
            np.testing.assert_array_equal(got["dt"][sl], s.get("dt"))
    finally:
        hg.hg_free(ctx)


def test_batch_integration_equals_separate_contexts(hg):
    """FP64: the batched global block steps give each cluster the same
    trajectory, steps and energy as its own context."""
    eps = 1e-3
    sizes = [200, 57, 640, 333]
    parts, off, mass, pos, vel = _clusters(sizes, 2000)
    opts = dict(precision=hg.HG_FP64, dt_min=DT_MIN, dt_max=DT_MAX)
    b = hg.hg_init_batch(off, mass, pos, vel, eps, 0.45, hg.hg_default_opts(**opts))
    ctxs = [hg.hg_init(p.mass, p.pos, p.vel, eps, 0.45, hg.hg_default_opts(**opts)) for p in parts]
    try:
        hg.hg_advance(b, 1.0 / 16)
        gb, tb = gpu_state(hg, b, int(off[-1]))
        assert tb == 1.0 / 16
        Kb, Wb = hg.hg_energy(b)
        K = W = inter = 0.0
        for c, (p, cx) in enumerate(zip(parts, ctxs)):
            hg.hg_advance(cx, 1.0 / 16)
            gs, _ = gpu_state(hg, cx, p.n)
            sl = slice(off[c], off[c + 1])
            assert rel_rows(gb["pos"][sl], gs["pos"]).max() < 1e-10, c
            assert np.mean(gb["dt"][sl] == gs["dt"]) >= 0.99, c
            k, w = hg.hg_energy(cx)
            K, W = K + k, W + w
            inter += hg.hg_get_stats(cx)["interactions"]
        assert Kb == pytest.approx(K, rel=1e-12)
        assert Wb == pytest.approx(W, rel=1e-12)
        # pair evaluations are counted per cluster (sum of m_c N_c), not m N
        assert hg.hg_get_stats(b)["interactions"] == pytest.approx(inter, rel=0.01)
    finally:
        hg.hg_free(b)
        for cx in ctxs:
            hg.hg_free(cx)
