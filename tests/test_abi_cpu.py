"""The C ABI library builds, loads without a GPU and exports every declared call."""
import ctypes
import os
import re

from paper_1207_2367_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hg_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hg_init", "hg_next_block", "hg_predict", "hg_evaluate", "hg_correct", "hg_step",
                     "hg_energy", "hg_get_state", "hg_set_state", "hg_free", "hg_last_error"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_opts_without_gpu():
    from paper_1207_2367_gb300 import binding
    o = binding.hg_default_opts()
    assert o.dt_min == 2.0 ** -25 and o.dt_max == 0.125 and o.eta_init == 0.01
    assert o.precision == binding.HG_FP64 and o.graph_steps == 8 and o.start_mode == 0 and o.profile == 0
    assert o.test_stall_eval == 0 and o.order == 6
    assert ctypes.sizeof(binding.hg_opts) == 10 * 4 + 3 * 8 + 8
