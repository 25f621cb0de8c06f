"""bench.py on the CPU: the algorithmic flop count that the roofline divides,
the workload part of the JSON line, and the reference arm's line (the oracle
timed on the host cores), which needs no GPU."""
import importlib.util
import json
import os
import subprocess
import sys

from paper_2412_02413_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fused_flops_per_frame():
    """Per (bin, row): 3 apertures x (6 nx phasor multiply + 5 nx log2 nx inverse
    FFT), plus 6 accumulations of 4 flops per pixel. 128 elements, 512 rows, 300
    bins: 2.89 GFLOP; 64 elements, 128 rows, 307 bins: 0.33 GFLOP."""
    b = _bench()
    assert b.fused_flops_per_frame(300, 512, 128, 3) == 300 * 512 * (3 * (6 * 128 + 5 * 128 * 7) + 24 * 128)
    assert b.fused_flops_per_frame(300, 512, 128, 3) == 2890137600.0
    assert round(b.fused_flops_per_frame(307, 128, 64, 3) / 1e9, 2) == 0.33
    assert b.fused_flops_per_frame(10, 4, 16, 1) == 10 * 4 * ((6 * 16 + 5 * 16 * 4) + 4 * 16)


def test_workload_config_names_the_workload():
    b = _bench()
    w = synth.workload(2)
    c = b.workload_config(w, 1)
    assert c == {"workload": w.name, "frames_per_step": 1, "n_elem": 128, "n_samples": 4096, "nx": 128,
                 "nz": 512, "n_bins": 300, "n_apod": 3}


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "frames/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"] == synth.workload(2).name
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["extrapolated"] is True and 0 < cb["sampled_fraction"] < 1
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_oracle_runs_mean_sd_and_extrapolation_label():
    """The CPU baseline's unit: runs of the oracle on a (bins x rows) sample,
    each scaled to a whole frame by the sampled fraction; mean and sd."""
    b = _bench()
    w = synth.workload(1)
    rf, _ = synth.make_frame(w, 0)
    r = b.oracle_runs(w, rf, 2, 4, 2, 3)
    assert r["runs"] == 3 and r["threads"] == 2 and r["value"] > 0 and r["sd"] >= 0
    assert r["extrapolated"] is True and r["sampled_fraction"] == 2 * 4 / (len(w.bins()) * w.nz)
