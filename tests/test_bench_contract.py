"""The benchmark's output contract, checked on the host: the reference arm
(the oracle on the host cores) prints one JSON line with the keys the GPU arm
prints, and the algorithmic flop count of the volume kernel matches its
stated per-direction terms."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "DOF/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == "flat_plate_2d_60x24_N7" and d["config"]["dof"] == 460800
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_volume_flop_count_terms():
    import bench
    # flat plate: 2D, n = 8, affine: 29 + 2 (8n + 16 + 16 + 32 + 53 + 10n)
    assert bench.volume_flops_per_node(2, 8, True) == 29 + 2 * (64 + 16 + 16 + 32 + 53 + 80) == 551
    # curved elements: gradient 27 n and lifting 54 per direction
    assert bench.volume_flops_per_node(3, 4, False) == 34 + 3 * (108 + 40 + 54 + 48 + 68)
