"""The benchmark's JSON contract, checked on the CPU with its reference arm (the FP64
oracle timed on the host cores): one JSON line with the metric, the timing fields, the
baseline description and the end-to-end object.  The GPU arm prints the same keys plus
roofline, clocks and launch counts; it is exercised on the GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["value"] > 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_gaussian_mode_finds_the_oracle_count_of_every_solve():
    """bench.py --mode gauss prints the FP64 oracle's count beside each GPU solve; every
    (nu, column, cycle) it runs has one in the stored file."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1012_5379_gb300 import inputs as I
    counts = bench.gauss_oracle_iters(os.path.join(ROOT, "tests", "golden", "oracle_iters_gauss.json"))
    for nu in (1.0, 7.0):
        for k, nint in I.GAUSS_COLUMNS:
            for cycle in ("1,0", "1,1"):
                assert isinstance(counts[bench.gauss_key(nu, k, nint, cycle)], int)
    assert bench.gauss_oracle_iters(os.path.join(ROOT, "tests", "golden", "absent.json")) == {}
