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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of hg_opts, hg_state, hg_stats, hg_profile and
    hg_tune_entry have the C structs' sizes and field offsets (a C probe
    compiled against include/hg.h prints them)."""
    import shutil
    import subprocess
    import pytest
    from paper_1207_2367_gb300 import binding
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    structs = {"hg_opts": binding.hg_opts, "hg_state": binding.hg_state, "hg_stats": binding.hg_stats,
               "hg_profile": binding.hg_profile, "hg_tune_entry": binding.hg_tune_entry}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        name, field, value = line.split()
        cls = structs[name]
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == int(value), (name, field, got, value)
