"""The benchmark's JSON line on CPU: the reference arm (the CPU FP64 oracle) run
as a subprocess on the tiny workload, and the line assembly of the GPU arm
from fake kernel statistics (no GPU needed)."""
import json
import os
import subprocess
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"}


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert BASE_KEYS <= set(d) and d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "states/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    tf = d["cpu_baseline"]["tiny_full_solve"]                   # a complete oracle solve, measured
    assert tf["kind"] == "measured" and tf["nconv"] == 8 and tf["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "tiny" in d["config"]["workload"]


def test_gpu_arm_line_assembly():
    import bench
    names = ["col_inverse_fft", "plane_fft_vloc", "col_forward_fft", "nonlocal_project", "nonlocal_D", "nonlocal_add",
             "gram", "rotate", "vector", "dense_la", "nonlocal_project_fp64"]
    stats = {k: dict(launches=10, ms=100.0 * (i + 1), bytes=1e9 * (i + 1), flops=1e12 * (i + 1))
             for i, k in enumerate(names)}
    stats["nonlocal_project"]["ms"] = 5000.0
    args = types.SimpleNamespace(precision="mixed", no_cpu=True, no_fp64=True, steps=1, warmup=3, workload="wire")
    w = types.SimpleNamespace(n=(72, 72, 144), natom=256, nproj=8, nstates=256, e_ref=0.03, nbands=272)
    gv = np.zeros((193673, 3), dtype=np.int32)
    gv[:, 0] = np.arange(193673) % 57                                # 57 x 45 distinct (g0, g1) columns
    gv[:, 1] = (np.arange(193673) // 57) % 45
    ctx = types.SimpleNamespace(npw=193673, gvectors=lambda: gv)
    r = [dict(nconv=256, iters=125, iters_mixed=125, n_hpsi=75600, resid=np.zeros(256), status=0)]
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    d = bench.make_line(args, w, ctx, r, stats, 256, 31.0, 32.0, 256, clocks, 6793.4, 1980.5, "measured", 1,
                        np.zeros((272, 10), complex))
    assert BASE_KEYS <= set(d) | {"cpu_baseline"}
    assert d["value"] == 256 / 31.0 and d["ms_per_step"] == 31000.0
    roof = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(roof)
    assert roof["kernel"] == "nonlocal_project"                 # FP64 classes and dense_la are excluded
    assert roof["frac"] == roof["achieved"] / roof["peak"]
    assert roof["traffic"] is not None                          # an ncu ratio exists for this kernel
    assert d["e2e"]["h2d_bytes_per_step"] == 272 * 10 * 16
    assert d["gpu_launches"] == sum(v["launches"] for v in stats.values())
    hs = d["hpsi_algorithmic"]
    bands = stats["col_inverse_fft"]["bytes"] / ((193673 + 144 * 57 * 45) * 8.0)
    assert abs(hs["bands"] - bands) <= 1e-9 * bands
    assert hs["bytes_per_band"] == 2 * 193673 * 8 + 8 * 72 * 72 * 144 * 8
    json.dumps(d)
