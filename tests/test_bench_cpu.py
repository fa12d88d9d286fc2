"""The benchmark's contract on the CPU: the reference arm (the FP64 oracle) prints one JSON line
with the keys the bench line promises, and the kernel counters stored in bench.py belong to
the frame kernel's current sources (else bench.py would report no traffic or issue figures)."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_counters_match_the_frame_kernel_sources():
    bench = _bench_module()
    assert bench.sources_digest() == bench.KERNEL_COUNTERS["sources_sha256_16"], (
        "the frame kernel's sources changed since its ncu capture: recapture the counters")
    assert bench.kernel_counters("bytes") == bench.KERNEL_COUNTERS["bytes"]


def test_reference_arm_prints_the_contract_line():
    pytest.importorskip("torch")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["unit"] == "frames/s" and line["higher_is_better"] is True
    assert line["config"]["workload"] == "frame1080p_u8_l3_g128"
    assert {"sigma_l", "lambda", "levels", "grid"} <= set(line["config"])
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
