"""Host logic of the evaluation planner with a tuning table (no GPU).

The planner header is compiled for the host with a small probe program
(tests/host/plan_probe.cpp) that reads "m value" queries and prints the bucket,
the cost model's plan, the plan with the value stored in m's bucket and the
batch knobs that value decodes to.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

TPS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16,
       20, 24, 32, 40, 48, 64, 96, 128, 192, 256, 384, 512, 1024, 2048, 4096, 8192]


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_probe")
    subprocess.run(["g++", "-std=c++17", "-O1", "-x", "c++", "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1207_2367_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "plan_probe.cpp"), "-o", exe], check=True)

    def run(queries, npad=65536):
        text = "".join(f"{m} {v}\n" for m, v in queries)
        out = subprocess.run([exe, str(npad)], input=text, capture_output=True, text=True, check=True).stdout
        keys = ("bucket", "model_tpi", "model_tps", "tpi", "tps", "b", "w_log", "tpi_shift", "variant", "ti",
                "model_variant", "n_points", "p0", "p1", "p2")
        return [dict(zip(keys, map(int, line.split()))) for line in out.splitlines()]
    return run


def test_buckets_are_floor_log2(probe):
    ms = [1, 2, 3, 4, 7, 8, 1000, 1023, 1024, 65535, 65536]
    got = probe([(m, -1) for m in ms], npad=65536)
    assert [g["bucket"] for g in got] == [m.bit_length() - 1 for m in ms]


def test_untuned_value_keeps_the_cost_model(probe):
    for g in probe([(m, -1) for m in (1, 5, 100, 5000, 65536)]):
        assert (g["tpi"], g["tps"]) == (g["model_tpi"], g["model_tps"])
        assert (g["w_log"], g["tpi_shift"]) == (1, 0)


@pytest.mark.parametrize("c", [0, 5, 33, 70, 100, 150, 200, 223])
def test_tuned_candidate_decodes_to_its_plan(probe, c):
    ntiles = 65536 // 256
    tps = TPS[c % 32]
    if tps > ntiles:
        pytest.skip("candidate not admissible at this size")
    g = probe([(64, c)])[0]
    assert g["variant"] == 0
    assert g["tpi"] == 1 << (c // 32)
    assert g["ti"] == 128 // g["tpi"]
    assert g["tps"] == tps
    assert g["b"] == -(-ntiles // tps)


def test_inadmissible_tuned_value_falls_back_to_the_model(probe):
    # tps 8192 > 256 tiles, and values outside [0, 224): both fall back.
    for v in (31, 224, 224 + 33, 5000):
        g = probe([(100, v)])[0]
        assert (g["tpi"], g["tps"]) == (g["model_tpi"], g["model_tps"])


def test_batch_codes_decode(probe):
    for w in range(7):
        for s in (-1, 0, 1):
            g = probe([(300, w + 8 * (s + 1))])[0]
            assert (g["w_log"], g["tpi_shift"]) == (w, s)
    for bad in (7, 15, 24, 40):   # w > 6 or s > 1: the untuned knobs
        g = probe([(300, bad)])[0]
        assert (g["w_log"], g["tpi_shift"]) == (1, 0)


def test_tuning_points_span_each_bucket(probe):
    """The autotuner times a bucket's plans at 5/4, 3/2 and 7/4 of 2^k (a plan
    stored for the bucket must hold for every m in it, and its wave count jumps
    with m); the first two buckets at their own sizes; all clamped to the
    largest tuned size."""
    big = 1 << 20
    for k in range(2, 20):
        g = probe([((1 << (k + 1)) - 1, -1)], npad=big)[0]   # m = top of bucket k: no clamping
        assert g["bucket"] == k
        assert (g["n_points"], g["p0"], g["p1"], g["p2"]) == (3, 5 << k >> 2, 3 << k >> 1, 7 << k >> 2)
        assert all((1 << k) <= p < (1 << (k + 1)) for p in (g["p0"], g["p1"], g["p2"]))
    g0, g1 = probe([(1, -1), (3, -1)])
    assert (g0["n_points"], g0["p0"]) == (1, 1)
    assert (g1["n_points"], g1["p0"], g1["p1"]) == (2, 2, 3)
    # m = 2: bucket 1 clamped to 2, a single size; m = 5 (bucket 2 = [4, 7]): 5, then 6 and 7 clamp to 5
    g2, g5 = probe([(2, -1), (5, -1)])
    assert (g2["n_points"], g2["p0"]) == (1, 2)
    assert (g5["n_points"], g5["p0"]) == (1, 5)
    g6 = probe([(6, -1)])[0]
    assert (g6["n_points"], g6["p0"], g6["p1"]) == (2, 5, 6)
