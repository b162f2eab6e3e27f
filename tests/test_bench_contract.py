"""The benchmark's reference arm (the CPU oracle timed on the host cores) and
its JSON line, run here without a GPU: one line with the contract's keys on
rank 0, nothing on the other ranks, for the product, the triangular solve and
the echelon form."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def run_bench(*args, env_extra=None):
    env = dict(os.environ)
    for name in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(name, None)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def one_line(stdout):
    lines = [ln for ln in stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, stdout
    return json.loads(lines[0])


def check_common(d, steps):
    assert KEYS <= d.keys()
    assert d["impl"] == "reference"
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] >= 3
    assert d["data"] == "synthetic" and d["scaling"] == "weak"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_product():
    d = one_line(run_bench("--steps", "2", "--warmup", "0", "--ref-rows", "2"))
    check_common(d, 2)
    assert d["metric"].startswith("GF(2^e) matmul field-ops/s, 4096")
    assert d["unit"] == "field-ops/s" and d["higher_is_better"] is True and d["dtype"] == "u8"
    assert d["vs_baseline"] is None
    assert d["config"]["m"] == d["config"]["n"] == d["config"]["k"] == 4096 and d["config"]["e"] == 4
    assert "rows 0..1" in d["cpu_baseline"]["sample"]


def test_reference_arm_other_ranks_print_nothing():
    out = run_bench("--steps", "1", "--warmup", "0", "--ref-rows", "2",
                    env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.strip() == ""


def test_reference_arm_triangular_solve():
    d = one_line(run_bench("--workload", "trsm_gf16_4096", "--steps", "1", "--warmup", "0", "--ref-rows", "1"))
    check_common(d, 1)
    assert "triangular solve" in d["metric"] and d["unit"] == "field-ops/s"
    assert d["config"]["op"] == "trsm_upper_left" and d["config"]["m"] == 4096


def test_reference_arm_echelon_form():
    d = one_line(run_bench("--workload", "rref_gf256_1000", "--steps", "1", "--warmup", "0"))
    check_common(d, 1)
    assert d["unit"] == "ms" and d["higher_is_better"] is False
    # the paper's own time for this workload (Table 2): value / 81 ms
    assert d["vs_baseline"] == pytest.approx(d["value"] / 81.0)


def test_reference_arm_ple():
    d = one_line(run_bench("--workload", "ple_gf256_1000", "--steps", "1", "--warmup", "0"))
    check_common(d, 1)
    assert "PLE" in d["metric"] and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["config"]["op"] == "ple" and d["config"]["m"] == 1000
    assert d["vs_baseline"] is None
