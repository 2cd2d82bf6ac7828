"""The benchmark's JSON contract on the CPU: the reference arm (the oracle timed on the
host cores) prints one line with the keys the driver reads, and the clock sampler counts
only the samples of the timed region and flags throttling."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_complete_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "grid64", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "grid64"


def test_clock_sampler_counts_the_timed_region_only():
    import bench

    c = bench.ClockSampler(0)
    warm = "0, 1400, 2070, 300.0, 0x1, Not Active, Active, Not Active, Not Active"
    timed = ["0, 2070, 2070, 550.0, 0x0, Not Active, Not Active, Not Active, Active",
             "0, 2065, 2070, 560.5, 0x0, Not Active, Not Active, Not Active, Not Active"]
    c.lines = [warm, warm]
    c.mark()
    c.lines += timed

    class P:  # a finished sampling process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = P()
    r = c.stop()
    assert r["samples"] == 2 and r["sm_mhz"] == 2067.5 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]          # the warm-up's thermal flag is not counted
    assert r["power_w_max"] == 560.5
    c2 = bench.ClockSampler(0)
    c2.lines = [warm]
    c2.mark()                                        # a region shorter than one period
    c2.proc = P()
    r2 = c2.stop()
    assert r2["samples"] == 1 and r2["reasons"] == ["hw_thermal_slowdown"]


def test_both_arms_describe_the_workload_alike():
    """The device arm and the reference arm build `config` with the same function, so
    the lines of one workload carry the same object, including the L2 note."""
    import bench

    _, desc = bench.make_workload("grid64", None)
    a, b = bench.workload_config(desc, 1), bench.workload_config(dict(desc), 1)
    assert a == b and a["workload"] == "grid64" and a["parallelism"] == "single GPU"
    assert "fit in L2" in a["l2"]
    big = bench.workload_config({"workload": "delaunay1m"}, 4)
    assert "larger than L2" in big["l2"] and big["parallelism"] == "replicas"
