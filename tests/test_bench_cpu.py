"""Host logic of bench.py that needs no GPU: the paper's block-size groups of the
cost attribution (Sect. 5.5).  The text's group bounds overlap at 1k, 10k and
100k; the reading used is A [1, 20], B [21, 100], C [101, 1000], D [1001, 10^4],
E [10^4 + 1, 10^5], F above."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_groups_partition_the_block_sizes():
    edges = {1: "A", 20: "A", 21: "B", 100: "B", 101: "C", 1000: "C", 1001: "D", 10000: "D",
             10001: "E", 100000: "E", 100001: "F", 1 << 23: "F"}
    for m, g in edges.items():
        assert bench.paper_group(m) == g, m
    ranges = sorted(bench.PAPER_GROUPS.values())
    assert ranges[0][0] == 1
    for (lo0, hi0), (lo1, hi1) in zip(ranges, ranges[1:]):
        assert lo1 == hi0 + 1          # contiguous, no overlap
        assert lo1 <= hi1


def test_relative_error_statistics():
    import numpy as np
    ref = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 2.0]])
    got = ref + np.array([[0.0, 0.0, 5e-7], [0.0, 0.0, 2e-6]])
    st = bench._rel_stats(got, ref)
    assert abs(st["max"] - 1e-6) < 1e-15            # particle 2: 2e-6 / 2
    assert abs(st["median"] - 0.5 * (1e-7 + 1e-6)) < 1e-15
    assert abs(st["normwise"] - np.sqrt(5e-7 ** 2 + 2e-6 ** 2) / np.sqrt(25.0 + 4.0)) < 1e-15


def test_clock_samples_and_throttle_reasons():
    lines = [
        "0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1010.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n",   # unreadable sample: skipped
        "garbage\n",
    ]
    out = bench.parse_clock_samples(lines)
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    hot = bench.parse_clock_samples(["0, 1500, 2070, 1400, 0x48, Active, Active, Not Active, Not Active\n"])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.parse_clock_samples([])["reasons"] == ["no samples"]


def test_kappa_statistics():
    import numpy as np
    ref = np.array([[1.0, 0.0, 0.0], [0.0, 1e-3, 0.0]])
    got = ref + np.array([[1e-7, 0.0, 0.0], [0.0, 1e-8, 0.0]])
    scale = np.array([2.0, 1.0])
    st = bench._kappa_stats(got, ref, scale)
    assert abs(st["worst_particle_rel_err"] - 1e-5) < 1e-15        # particle 2: 1e-8 / 1e-3
    assert abs(st["worst_particle_kappa"] - 1e3) < 1e-9             # 1.0 / 1e-3
    assert abs(st["max_err_over_scale"] - 5e-8) < 1e-15            # particle 1: 1e-7 / 2


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host, no GPU): one JSON line
    with the metric, a positive rate, the configuration and the keys the
    reference arm carries (cpu_baseline describing the run, e2e with no copies)."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n", "65536"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == "interactions/s" and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0 and line["config"]["n"] == 65536
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "interactions/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
