"""The benchmark's JSON line (CPU only): the reference arm runs the FP64
oracle on the host, so its line can be produced and checked here; the GPU arm
shares the metric name and workload label with it."""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

REQUIRED = {"metric": str, "value": float, "unit": str, "n_gpus": int, "steps": int, "warmup": int,
            "ms_per_step": float, "higher_is_better": bool, "scaling": str, "dtype": str, "data": str,
            "config": dict, "cpu_baseline": dict, "e2e": dict}


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--size", "32"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key, typ in REQUIRED.items():
        assert isinstance(line[key], typ), key
    assert line["impl"] == "reference"
    assert line["vs_baseline"] is None
    assert line["value"] > 0 and line["unit"] == "MLUPS" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    import bench
    assert line["metric"] == bench.METRIC
    assert line["config"]["workload"].startswith("spherepack32_steady: 32^3 sphere pack")


def test_algorithmic_bytes_per_site():
    import bench
    assert bench.BYTES_STEP_FP32 == 272 and bench.BYTES_STEP_FP16 == 140
    assert bench.BYTES_COLLIDE_FP32 == 212 and bench.BYTES_COLLIDE_FP16 == 108
