"""The benchmark's JSON line: the keys and types the measurement contract
names, for the oracle arm on the host (CPU) and the GPU arm (GPU), on small
workloads (the 16384^2 grid is the default; these pass --workload)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=timeout, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def check_common(d):
    for k, t in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                 ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                 ("dtype", str), ("data", str), ("config", dict), ("e2e", dict)):
        assert isinstance(d[k], t), (k, d.get(k))
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert "workload" in d["config"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"]


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--workload", "c3:256", "--steps", "2", "--warmup", "3")
    check_common(d)
    assert d["impl"] == "reference" and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line():
    d = run_bench("--workload", "c3:512", "--steps", "16", "--warmup", "4", "--no-sweep", "--no-adjoint",
                  "--no-ensemble", "--no-cpu-baseline")
    check_common(d)
    assert d["dtype"] == "f32" and d["n_gpus"] == 1
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert d["gpu_launches"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["config"]["kernel"] == "tiled" and d["config"]["steps_per_launch"] == 4
    assert d["one_step"]["kernel"] == "stream" and d["one_step"]["value"] > 0
    runs = d["decomposition"]["runs"]                 # 1 x 2 and 1 x 4 strips of the same workload
    assert [r["parts"] for r in runs] == [2, 4] and all(r["value"] > 0 and r["halo"] == 4 for r in runs)
