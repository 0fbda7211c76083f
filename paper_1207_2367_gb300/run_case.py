"""Run one seeded synthetic case: start-up plus a number of block steps.

    python -m paper_1207_2367_gb300.run_case --n 131072 --imf equal --precision mixed --steps 0

Builds a Plummer sphere (Henon units), creates a context (the start-up
evaluation has every particle active), replays --steps block steps from CUDA
graphs and prints the device counters; --eval-m then times evaluations (evaluation
and j-split reduction kernels) of that many particles.  Used for profiling single
kernels.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=65536)
    ap.add_argument("--imf", choices=["equal", "salpeter"], default="equal")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--eta", type=float, default=0.45)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--dt-max", type=float, default=1.0 / 16)
    ap.add_argument("--eval-m", type=int, default=0,
                    help="then time evaluations of m particles spread over the system (hg_time_evaluate)")
    ap.add_argument("--eval-reps", type=int, default=20)
    a = ap.parse_args(argv)

    from . import binding as hg
    from . import inputs

    hg.load()
    p = inputs.plummer(a.n, a.seed, imf=a.imf)
    prec = hg.HG_MIXED if a.precision == "mixed" else hg.HG_FP64
    t0 = time.perf_counter()
    ctx = hg.hg_init(p.mass, p.pos, p.vel, a.eps, a.eta, hg.hg_default_opts(precision=prec, dt_max=a.dt_max))
    try:
        t_init = time.perf_counter() - t0
        t0 = time.perf_counter()
        if a.steps:
            hg.hg_step(ctx, a.steps)
        stats = hg.hg_get_stats(ctx)
        stats.update(n=a.n, init_s=t_init, steps_s=time.perf_counter() - t0)
        if a.eval_m:
            import numpy as np
            lst = np.unique(np.linspace(0, a.n - 1, a.eval_m).astype(np.int32))
            hg.hg_predict(ctx, stats["t_sys"])
            stats.update(eval_m=int(lst.shape[0]),
                         eval_us=hg.hg_time_evaluate(ctx, lst, lst.shape[0], a.eval_reps))
        print(json.dumps(stats))
    finally:
        hg.hg_free(ctx)


if __name__ == "__main__":
    main()
