"""Host logic of bench.py that needs no GPU: which committed oracle golden checks a timed result,
the algorithmic-byte model and the DRAM-traffic lookup gated by the kernel sources' hash."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_the_headline_pulse_has_a_full_length_golden():
    W, w = bench.workload("xxz_L20_N400_m20")

    class Args:
        grad = "centered"
        workload = "xxz_L20_N400_m20"

    with open(os.path.join(ROOT, "tests", "golden", "oracle_xxz_L20_N400_m20.json")) as fh:
        gd = json.load(fh)
    err = bench.err_vs_oracle(Args, w, gd["F_centered"], gd["grad_centered"])
    assert err is not None and err["F"] == 0.0 and err["grad"] == 0.0


def test_the_l24_chain_is_checked_on_its_shorter_golden():
    # the L = 24 workload has no 400-slice golden: the 12-slice one of the same workload is used
    found = bench.short_pulse_golden("xxz_L24_N400_m24_ckpt20", "centered")
    assert found is not None
    path, gd = found
    assert os.path.basename(path) == "oracle_xxz_L24_N12_m24.json"
    assert gd["N"] == 12 and gd["workload"] == "xxz_L24_N400_m24_ckpt20"
    assert bench.short_pulse_golden("xxz_L24_N400_m24_ckpt20", "exact") is None
    assert bench.short_pulse_golden("no_such_workload", "centered") is None


def test_algorithmic_bytes_of_the_headline_launch():
    # P = N (2 (4m - 1) + 1) + 2 vector passes of D complex64 amplitudes (8 bytes)
    _, w = bench.workload("xxz_L20_N400_m20")
    assert bench.alg_bytes(w, "c64") == (400 * (2 * (4 * 20 - 1) + 1) + 2) * (1 << 20) * 8


def test_traffic_is_reported_only_for_the_captured_sources():
    key = "kg_eval_kernel<float2>@xxz_L20_N400_m20"
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
        ent = json.load(fh)[key]
    t = bench.ncu_traffic(key)
    if ent["source_hash"] == bench.kernel_source_hash():
        assert t == float(ent["dram_bytes_per_launch_full"])
    else:
        assert t is None
    assert bench.ncu_traffic("no_such_kernel@nowhere") is None
