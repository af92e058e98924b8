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


def test_oracle_leg_clamps_its_band_to_the_row_limit():
    # a band never runs past the rows asked for (or the frame's 1080 rows)
    bench = _bench()
    rate, rows, secs = bench.oracle_rate(0.0, 6, max_rows=20)
    assert rows == 20 and rate > 0 and secs > 0


def test_row_groups_and_host_info():
    import pytest
    bench = _bench()
    every = bench.wanted_rows(argparse.Namespace(rows_only=""))
    assert {"core", "precision", "small", "batch", "chains", "upsample", "pathtrace", "sweep", "serve"} == every
    assert bench.wanted_rows(argparse.Namespace(rows_only="small, serve")) == {"small", "serve"}
    with pytest.raises(SystemExit):
        bench.wanted_rows(argparse.Namespace(rows_only="nope"))
    h = bench.host_cpu_info()
    assert h["cpu_count"] >= 1 and h["oracle_threads"] == 1
