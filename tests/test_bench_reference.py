"""bench.py's reference arm (the oracle timed on the host cores) runs without a GPU and prints one
JSON line with the contract's keys, on the same metric, unit and workload as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("2D periodic drop advection 64x64 quads p=3")


def test_summary_digest_of_a_line():
    """The line's last key digests every block present, in a few hundred characters."""
    import bench
    line = {"ms_per_step": 0.0234, "value": 5.89e10, "roofline": {"frac": 0.303}, "e2e": {"value": 1.75e10},
            "accuracy": {"l2_rel_alpha": 4.8e-9, "l2_rel_p": 4.9e-7, "l2_rel_u": 3e-5},
            "adjoint": {"adjoint_over_forward": 2.72, "forward_ms": 124.5, "backward_ms": 338.7},
            "batched": {"ms_per_step": 7.8, "value": 9.5e10, "speedup_vs_fp64": 13.0,
                        "accuracy": {"max_l2_rel_alpha": 1.5e-8, "max_l2_rel_p": float("nan"), "max_l2_rel_u": 2e-5}}}
    s = bench.summary(line)
    assert s["config2"]["us_per_step"] == 23.4 and s["config2"]["acc_500"] == [4.8e-9, 4.9e-7, 3e-5]
    assert s["config5"]["adjoint_over_forward"] == 2.72
    assert s["config4"]["acc_200_max"][1] != s["config4"]["acc_200_max"][1]  # a NaN stays a NaN
    assert "config3" not in s and "config1" not in s
    assert len(json.dumps(s)) < 1000


def test_batch_roofline_units():
    """The batched step's roofline: 168 B per node and stage, three stages a step, over the step time,
    against the measured HBM copy rate."""
    import bench
    r = bench.batch_roofline(nodes=1_000_000, ms_step=1.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 168 * 3 * 1_000_000 / 1e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
