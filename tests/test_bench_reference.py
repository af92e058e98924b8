"""The bench's reference arm (the FP64 oracle on the host) produces a line
with a positive rate; runs on the CPU."""
import argparse
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("_hsc_bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_times_at_least_one_band():
    bench = _bench()
    args = argparse.Namespace(steps=1, warmup=0, k=6)
    res = bench.run_reference(args, 0, 1)
    assert res["impl"] == "reference" and res["value"] > 0 and res["ms_per_step"] > 0
    assert res["cpu_baseline"]["value"] == res["value"] and res["e2e"]["h2d_bytes_per_step"] == 0
    assert bench.run_reference(args, 1, 2) is None  # other ranks do no work
