"""The bench's JSON line: required keys, the roofline arithmetic, the survival
report and the traffic record's code key (host only)."""
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

RADII2 = [24, 29, 36, 43, 53, 65, 79, 96]


def _wl(H, W, radii=RADII2, sum_bits=32, sq_bits=64):
    return types.SimpleNamespace(image=np.zeros((H, W), np.uint8), radii=radii, t_min=40, r=48,
                                 scales=[0.5 * 4 ** (i / 7) for i in range(8)], features=7,
                                 sum_bits=sum_bits, sq_bits=sq_bits, distractors=[], planted=(100, 100),
                                 s_true=1.0)


def _line(H, W, k3_ms, tab_ms, config=2):
    wl = _wl(H, W)
    args = argparse.Namespace(steps=2, warmup=3, no_cpu_baseline=True, config=config)
    m = {"k3_ms": [k3_ms] * 2, "tab_ms": [tab_ms] * 2, "step_ms": [0.4] * 2, "total_s": 0.8e-3,
         "launches": 16, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}, "survivors": 10,
         "value": 1.0}
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.emit(args, wl, 1, m, None, {})
    return json.loads(buf.getvalue().strip().splitlines()[-1])


def test_line_keys_and_per_scale_roofline():
    d = _line(4096, 4096, 1.0, 0.15)     # a slow launch: the per-scale model stays below the roof
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "tables_roofline",
              "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["config"]["workload"].startswith("config 2: single image 4096x4096")
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


def test_candidate_counts_of_the_configurations():
    import synth
    wl3 = types.SimpleNamespace(radii=synth.radii_for(64, synth.geometric_scales(0.35, 2.8, 16)))
    assert wl3.radii[0] == 22 and wl3.radii[-1] == 179
    assert bench.candidates(8192, 8192, wl3.radii) == 1034216188
    assert bench.candidates(4096, 4096, RADII2) == 127458510
    # config 3's compulsory bytes: u64/u64 tables once + 16 mask planes
    b = bench.compulsory_bytes(8192, 8192, 16, 64, 64, 0)
    assert abs(b / 1034216188 - 2.2) < 0.05


def test_survival_report_reads_covering_scales():
    wl = _wl(64, 64)
    wl.radii, wl.t_min, wl.r = [10, 14, 20], 10, 14
    wl.planted, wl.s_true = (30, 33), 1.0                  # covering scales: R/1 in [9, 15] -> 0, 1
    wl.distractors = [(20, 5, 1.03, 1.4), (40, 40, 0.97, 1.0)]
    mask = np.zeros((3, 64, 2), np.uint32)
    mask[2, 30, 1] |= np.uint32(1 << 1)                    # planted set only at a non-covering scale
    mask[2, 20, 0] |= np.uint32(1 << 5)                    # distractor 0 at scale 2: R/1.4 = 14.3, covering
    s = bench.survival(mask, wl)
    assert s["planted"]["survives"] is False and s["planted"]["scales_set"] == [2]
    assert s["distractors"] == {"total": 2, "survive_at_covering_scale": 1, "survive_at_any_scale": 1}
    mask[1, 30, 1] |= np.uint32(1 << 1)
    assert bench.survival(mask, wl)["planted"]["survives"] is True


def test_traffic_record_follows_kernel_code_not_comments(tmp_path):
    base = "// a comment\n__global__ void k(int *p) { /* note */ p[0] = 1; }\n"
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text(base)
    b.write_text(base.replace("a comment", "another comment").replace("note", "other"))
    c.write_text(base.replace("p[0] = 1", "p[0] = 2"))
    assert bench.code_sha256([str(a)]) == bench.code_sha256([str(b)])
    assert bench.code_sha256([str(a)]) != bench.code_sha256([str(c)])
    # a record is used only while its key matches the kernel's code and flags
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = prof / "k_screen_8192_traffic.txt"
    rec.write_text(f"dram_bytes_per_launch: 123\nkernel_code_sha256: {bench.kernel_code_sha256()}\n")
    assert bench.recorded_traffic(8192, 8192, root=str(tmp_path)) == 123
    rec.write_text("dram_bytes_per_launch: 123\nkernel_code_sha256: 00\n")
    assert bench.recorded_traffic(8192, 8192, root=str(tmp_path)) is None
    assert bench.recorded_traffic(8192, 8192, root=str(tmp_path / "none")) is None
    # ... and the number of packed filter windows the run uses
    rec.write_text(f"dram_bytes_per_launch: 7\nfilter_windows: 2\nkernel_code_sha256: {bench.kernel_code_sha256()}\n")
    assert bench.recorded_traffic(8192, 8192, root=str(tmp_path), n_windows=2) == 7
    assert bench.recorded_traffic(8192, 8192, root=str(tmp_path)) is None


def test_clock_samples_are_kept_only_inside_the_window():
    import datetime
    import tempfile
    c = bench.Clocks(0)
    c.f = tempfile.TemporaryFile(mode="w+")
    t0 = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def line(dt_ms, mhz, slowdown="Not Active"):
        ts = (t0 + datetime.timedelta(milliseconds=dt_ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, {mhz}, 2070, 500.0, 0x0, {slowdown}, Not Active, Not Active, Not Active\n"

    c.f.write(line(0, 1000) + line(100, 2070) + line(150, 2070, "Active") + line(400, 900) + "garbage\n")
    base = t0.timestamp()
    s = c.summary(base + 0.05, base + 0.2, "test window")
    assert s["samples"] == 2 and s["sm_mhz"] == 2070.0 and s["reasons"] == ["hw_slowdown"]
    assert c.count_between(base + 0.05) == 3
    empty = c.summary(base + 1.0, base + 2.0, "later")
    assert empty["samples"] == 0 and empty["sm_mhz"] is None
