"""The bench's JSON line: required keys and the roofline arithmetic (host only)."""
import argparse
import io
import json
import os
import sys
import types
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bench  # noqa: E402


class _Clk:
    def summary(self):
        return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}


def _line(H, W, k3_ms, tab_ms):
    wl = types.SimpleNamespace(image=np.zeros((H, W), np.uint8), radii=[24, 29, 36, 43, 53, 65, 79, 96],
                               t_min=40, sum_bits=32, sq_bits=64)
    args = argparse.Namespace(steps=2, warmup=3, no_cpu_baseline=True)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.emit(args, wl, 1, 2 * 0.4e-3, 1.0, [k3_ms] * 2, [0.4] * 2, 16, _Clk(), 10, None, [tab_ms] * 2)
    return json.loads(buf.getvalue().strip().splitlines()[-1])


def test_line_keys_and_per_scale_roofline():
    d = _line(4096, 4096, 1.0, 0.15)     # a slow launch: the per-scale model stays below the roof
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "tables_roofline",
              "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    # per-scale model: 8 passes over the four tables (u32 + u64 planes) plus the mask
    H = W = 4096
    tables = ((H + 1) * (W + 1) + (H + 1) * (W + 2)) * 12
    alg1 = 8 * tables + 8 * H * (W // 32) * 4
    assert abs(r["achieved"] - alg1 / 1.0e-3 / 1e9) < 1e-6 * r["achieved"]
    assert r["model"].startswith("Algorithm 1 per-scale")
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["compulsory"]["frac"] < r["frac"]
    t = d["tables_roofline"]
    assert abs(t["achieved"] - (H * W + tables) / 0.15e-3 / 1e9) < 1e-6 * t["achieved"]


def test_per_scale_fraction_never_quoted_above_one():
    d = _line(4096, 4096, 0.2, 0.15)       # per-scale bytes / time above the HBM roof
    r = d["roofline"]
    assert r["frac"] <= 1.0
    assert r["model"].startswith("compulsory")
    assert r["per_scale_above_peak"]["achieved"] > r["peak"]


def test_traffic_record_follows_kernel_code_not_comments(tmp_path):
    base = "// a comment\n__global__ void k(int *p) { /* note */ p[0] = 1; }\n"
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text(base)
    b.write_text(base.replace("a comment", "another comment").replace("note", "other"))
    c.write_text(base.replace("p[0] = 1", "p[0] = 2"))
    assert bench.kernel_code_sha256(str(a)) == bench.kernel_code_sha256(str(b))
    assert bench.kernel_code_sha256(str(a)) != bench.kernel_code_sha256(str(c))
    # the committed record matches the committed kernel
    assert bench.recorded_traffic(4096, 4096) is not None
