"""The bench's reference arm on CPU: one JSON line with the contract's keys, the oracle as the timed program,
no host-device traffic, and the workload's L2 statement following the grid size."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "33",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "PF solves/s" and d["unit"] == "solves/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "pf_33_four_pores_NaCaCl"
    assert "fits in L2" in d["config"]["l2"]


def test_l2_statement_at_the_bench_size():
    sys.path.insert(0, ROOT)
    import bench
    args = type("A", (), dict(n=257, precision="mixed", tol_outer=1e-3, lin_tol=1e-6, accel_depth=0, inner_tol=0.1,
                              gpus=1))
    assert bench.config_of(args)["l2"].startswith("inputs larger than L2")
