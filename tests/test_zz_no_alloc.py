"""The evaluation entry point that allocates no memory (hg_evaluate_static).

Callers that may not allocate device memory (their host framework owns all of
it, or fixed its budget at start-up) use hg_evaluate_static, which keeps its
scratch in one fixed array inside the library.  Its results must agree with the
context-based hg_evaluate on the same predicted data, within the parity
tolerances, on consecutive calls: the shared scratch keeps the previous call's
contents, so the second call uses a different system size and list.
"""
import numpy as np
import pytest

from paper_1207_2367_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: (1e-12, 1e-12, 1e-12), 1: (1e-6, 1e-5, 1e-4)}


def _system(hg, n, seed, precision, eps):
    """A context whose state sits at t = 0 with arbitrary derivatives, so that the
    prediction to t = 0 is exactly the state itself."""
    p = inputs.plummer(n, seed)
    rng = np.random.default_rng(seed)
    st = {"mass": p.mass, "pos": p.pos, "vel": p.vel, "acc": rng.normal(size=(n, 3)),
          "jerk": rng.normal(size=(n, 3)), "snap": rng.normal(size=(n, 3)), "crackle": rng.normal(size=(n, 3)),
          "t": np.zeros(n), "dt": np.full(n, 1.0 / 16)}
    ctx = hg.hg_init(p.mass, p.pos, p.vel, eps, 0.45,
                     hg.hg_default_opts(precision=precision, dt_max=1.0 / 16, start_mode=1))
    hg.hg_set_state(ctx, st, 0.0)
    hg.hg_predict(ctx, 0.0)
    return ctx, st


def _compare(got, ref, precision):
    for g, r, tol in zip(got, ref, TOL[precision]):
        if precision == 0:
            err = (np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)).max()
        else:
            err = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert err <= tol, (err, tol)


@pytest.mark.parametrize("precision", [0, 1])
def test_static_entry_matches_context_entry_twice(hg, precision):
    import torch
    eps = 1e-3
    for call, (n, seed, stride) in enumerate(((3001, 31, 3), (1500, 32, 7))):
        ctx, st = _system(hg, n, seed, precision, eps)
        try:
            idx = np.arange(call, n, stride, dtype=np.int32)
            m = idx.shape[0]
            ref = [np.empty((m, 3)) for _ in range(3)]
            hg.hg_evaluate(ctx, idx, m, *ref)
        finally:
            hg.hg_free(ctx)
        dev = {k: torch.tensor(st[k], device="cuda") for k in ("mass", "pos", "vel", "acc")}
        idx_d = torch.tensor(idx, device="cuda")
        out = [torch.full((m, 3), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
        hg.hg_evaluate_static(dev["mass"], dev["pos"], dev["vel"], dev["acc"], eps, precision, idx_d, m, *out)
        _compare([o.cpu().numpy() for o in out], ref, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_static_entry_at_its_limits(hg, precision):
    """The largest system the fixed array holds (n = 16384: the full record area)
    with one active particle (the largest j-split, b * m at its cap), 16, and all
    of them (m = n); and eps = 0 (the guarded path that skips the own pair)."""
    import torch
    n = 16384
    for eps, lists in ((1e-3, (np.array([n // 2]), np.arange(5, n, n // 16)[:16], np.arange(n))),
                       (0.0, (np.arange(0, n, 5),))):
        ctx, st = _system(hg, n, 40, precision, eps)
        dev = {k: torch.tensor(st[k], device="cuda") for k in ("mass", "pos", "vel", "acc")}
        try:
            for idx in lists:
                idx = np.ascontiguousarray(idx, dtype=np.int32)
                m = idx.shape[0]
                ref = [np.empty((m, 3)) for _ in range(3)]
                hg.hg_evaluate(ctx, idx, m, *ref)
                out = [torch.full((m, 3), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
                hg.hg_evaluate_static(dev["mass"], dev["pos"], dev["vel"], dev["acc"], eps, precision,
                                      torch.tensor(idx, device="cuda"), m, *out)
                _compare([o.cpu().numpy() for o in out], ref, precision)
        finally:
            hg.hg_free(ctx)


def test_static_entry_allocates_nothing_after_set_up(hg):
    """A call with m = 0 loads the fixed array; after one full call, a second
    call leaves the device's free memory exactly as it was (cudaMemGetInfo)."""
    import torch
    n, m, eps = 4096, 1024, 1e-3
    ctx, st = _system(hg, n, 41, 1, eps)
    hg.hg_free(ctx)
    dev = {k: torch.tensor(st[k], device="cuda") for k in ("mass", "pos", "vel", "acc")}
    idx = torch.arange(0, n, n // m, dtype=torch.int32, device="cuda")
    out = [torch.empty((m, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    args = (dev["mass"], dev["pos"], dev["vel"], dev["acc"], eps, 1, idx)
    hg.hg_evaluate_static(*args, 0, *out)        # set-up only
    hg.hg_evaluate_static(*args, m, *out)
    first = [o.clone() for o in out]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    hg.hg_evaluate_static(*args, m, *out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for a, b in zip(first, out):
        assert torch.equal(a, b)


def test_static_entry_rejects_what_it_cannot_hold(hg):
    import torch
    n = 16385
    z = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    mass = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    idx = torch.arange(4, dtype=torch.int32, device="cuda")
    out = [torch.empty((4, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(hg.HGError) as e:
        hg.hg_evaluate_static(mass, z, z, z, 1e-3, 1, idx, 4, *out)
    assert e.value.code == hg.HG_EINVAL and "16384" in str(e.value)
    n = 64
    z = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    mass = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HGError) as e:       # not increasing
        hg.hg_evaluate_static(mass, z, z, z, 1e-3, 1, torch.tensor([3, 1], dtype=torch.int32, device="cuda"), 2,
                              *[o[:2] for o in out])
    assert e.value.code == hg.HG_EINVAL
    with pytest.raises(hg.HGError) as e:       # host memory
        hg.hg_evaluate_static(mass.cpu(), z, z, z, 1e-3, 1, idx, 4, *out)
    assert e.value.code == hg.HG_EINVAL
