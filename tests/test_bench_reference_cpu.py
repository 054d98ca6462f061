"""The reference arm of bench.py on the host (no GPU): `--impl reference`
times the oracle on a bounded sample of the workload and prints one JSON line
with the keys of the benchmark contract, its own cpu_baseline and an e2e
entry with no host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "uniform4096", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["unit"] == "cell-updates/s" and d["higher_is_better"] is True and d["value"] > 0
    per_step = d["config"]["sample_cells_per_step"]
    assert abs(d["value"] - per_step / (d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
    assert d["config"]["workload"] and d["config"]["cells"] == 4096
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_bench_states_the_tests_mixed_bounds():
    """The bound bench.py reports against (largest relative error of the
    mixed path per workload) is the one the parity tests enforce."""
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import bench
    import test_gpu_mixed_batched as t
    assert bench.STATED_MIXED_MAX == {"gmc256": t.BOUND_GMC["max"], "amr3000": t.BOUND_AMR["max"],
                                      "be": t.BOUND_AMR["max"], "uniform4096": t.BOUND_RANDOM["max"],
                                      "grf128": t.BOUND_RANDOM["max"]}
    assert bench.FCHEM_PROBE == t.FCHEM_PROBE
