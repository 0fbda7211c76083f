"""Plain FP64 CPU oracle of the HiGPUs 6th-order Hermite block-timestep method.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg.  The CUDA product path never imports it.
"""
from .oracle import (  # noqa: F401
    build, lib, predict, evaluate, eval_absum, correct, correct4, interp, interp4, criterion, block_dt, block_dt_init,
    next_block, energy, angular_momentum, System,
)
