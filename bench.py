"""Benchmark of the screening hot path on GB300.

One step = the whole path on one synthetic 4096x4096 image (the single-large-
image workload: 8 scales 0.5..2 of a radius-48 template, mean + variance +
contrast, uint32 sum / uint64 sum^2 tables):
  build_tables (upright + cone tables)  ->  screen_features (star features and
  thresholds -> bitmask)  ->  compact_mask (bitmask -> sorted survivor list).
`value` = candidate (position x scale) evaluations per second with the image
already resident in HBM; `e2e` = the same metric through screen_host() with the
image in pinned host memory and the count + list copied back every step.

--impl reference times the CPU oracle (the slow plain implementation the GPU
path is checked against) on the host cores instead.
Under torchrun each rank screens its own image (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate (position x scale) evaluations/s"
UNIT = "evals/s"


def candidates(H, W, radii):
    """Number of valid (scale, y, x) candidates: the star lies inside the image."""
    tot = 0
    for R in radii:
        n = 0
        while (2 * n + 1) ** 2 < 2 * R * R:
            n += 1
        h = R
        ylo, yhi = max(n, h) - 1, H - 1 - max(n, h)
        xlo, xhi = max(n, h) - 1, min(W - 1 - n, W - h)
        if yhi >= ylo and xhi >= xlo:
            tot += (yhi - ylo + 1) * (xhi - xlo + 1)
    return tot


def compulsory_bytes(H, W, n_scales, sum_bits, sq_bits, survivors):
    """Compulsory traffic of one screening pass with tables reused across scales:
    the four tables read once (full width), the mask written, the list written."""
    tables = ((H + 1) * (W + 1) + (H + 1) * (W + 2)) * (sum_bits + sq_bits) // 8
    return tables + n_scales * H * ((W + 31) // 32) * 4 + 8 * survivors


def per_scale_bytes(H, W, n_scales, sum_bits, sq_bits):
    """Algorithmic bytes of one screening launch under the per-scale model of
    Algorithm 1: every scale pass reads the four tables once and writes its mask."""
    tables = ((H + 1) * (W + 1) + (H + 1) * (W + 2)) * (sum_bits + sq_bits) // 8
    mask = n_scales * H * ((W + 31) // 32) * 4
    return n_scales * tables + mask


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) >= 8:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
                if any(r[2].replace(".", "").isdigit() for r in rows) else None}


def kernel_code_sha256(path):
    """SHA-256 of a CUDA source with its comments and whitespace removed, so a
    comment edit does not invalidate counters taken on the same code."""
    import hashlib
    import re
    text = open(path, encoding="utf-8").read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = " ".join(text.split())
    return hashlib.sha256(text.encode()).hexdigest()


def recorded_traffic(H, W):
    """DRAM bytes per k_screen launch from the committed ncu capture of the
    4096x4096 workload, or None if the kernel's code changed since."""
    path = os.path.join(ROOT, "profiles", "k_screen_4096_traffic.txt")
    if (H, W) != (4096, 4096) or not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if ":" in line and not line.startswith(("#", " ", "`")):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_1707_05647_gb300", "csrc", "features.cu")
    if rec.get("kernel_code_sha256") != kernel_code_sha256(src):
        return None
    return int(rec["dram_bytes_per_launch"])


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def oracle_baseline(wl, max_rows=None, threads=0, split=None, min_seconds=0.0):
    """CPU oracle on the host cores (threads = 0: all, OpenMP over rows in the
    screen); the sample (tables + screen of the first max_rows rows) is repeated
    until min_seconds have passed.  Returns (evals/s, sample, threads used,
    seconds).  split, a dict, receives the mean table-build and screen seconds."""
    import oracle
    img = wl.image if max_rows is None else wl.image[:max_rows]
    H, W = img.shape
    used = oracle.threads(threads if threads > 0 else (os.cpu_count() or 1))
    t_tab = t_all = 0.0
    reps = 0
    while reps == 0 or t_all < min_seconds:
        t0 = time.perf_counter()
        tb = oracle.Tables(img)
        t1 = time.perf_counter()
        oracle.screen_workload(img, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol, tables=tb)
        t_all += time.perf_counter() - t0
        t_tab += t1 - t0
        reps += 1
    if split is not None:
        split["tables_s"] = t_tab / reps
        split["screen_s"] = (t_all - t_tab) / reps
    n = candidates(H, W, wl.radii)
    sample = f"{H}x{W} rows of the same image, all {len(wl.radii)} scales, tables + screen"
    if reps > 1:
        sample += f", repeated {reps} times"
    return n * reps / t_all, sample, used, t_all


def oracle_threads(n):
    import oracle
    oracle.threads(n)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    wl = synth.config2()
    rows = 512
    for _ in range(args.warmup):
        oracle_baseline(wl, rows)
    vals, secs = [], []
    for _ in range(args.steps):
        v, sample, cores, dt = oracle_baseline(wl, rows)
        vals.append(v)
        secs.append(dt)
    value = len(secs) * candidates(rows, wl.image.shape[1], wl.radii) / sum(secs)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": config_dict(wl),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def config_dict(wl):
    H, W = wl.image.shape
    return {"workload": f"single large image: {H}x{W} u8, planted r=48 template, 8 scales 0.5-2, "
                        "mean+variance+contrast, u32 sum / u64 sum^2 tables",
            "image": f"{wl.image.shape[0]}x{wl.image.shape[1]}", "radii": wl.radii, "t_min": wl.t_min,
            "features": "mean+var+contrast", "tables": f"u{wl.sum_bits} sum / u{wl.sq_bits} sum^2",
            "l2": "flushed between timed steps (256 MiB write); tables 403 MB > L2",
            "candidates_per_step": candidates(*wl.image.shape, wl.radii)}


def run_ours(args):
    import torch
    import synth
    import paper_1707_05647_gb300 as scr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    wl = synth.config2(synth.BASE_SEED + 1 + 1000 * rank)
    if args.size != 4096:      # smaller case of the same recipe (profiling captures)
        wl.image = np.ascontiguousarray(wl.image[:args.size, :args.size])
    H, W = wl.image.shape
    S = len(wl.radii)
    ncand = candidates(H, W, wl.radii)
    ctx = scr.screen_init(local, 0)
    p = scr.Params(wl.radii, wl.features, wl.tol.mean_rel, wl.tol.std_rel, wl.tol.grad_rel, wl.tol.grad_abs)
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    stream = torch.cuda.current_stream()
    img = torch.from_numpy(wl.image).cuda()
    mask = torch.empty(scr.mask_words(S, H, W), dtype=torch.int32, device="cuda")
    cap = 1 << 22
    lst = torch.empty(cap, dtype=torch.int64, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(evs=None):
        tb = scr.build_tables(ctx, img, wl.sum_bits, wl.sq_bits, stream)
        if evs:
            evs[0].record(stream)
        scr.screen_features(ctx, tb, tm, p, mask, stream)
        if evs:
            evs[1].record(stream)
        scr.compact_mask(ctx, mask, S, H, W, lst, count, stream)
        scr.tables_release(ctx, tb)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = scr.screen_stats(ctx)["kernel_launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step(kev[k])
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = scr.screen_stats(ctx)["kernel_launches"] - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    k3_ms = [a.elapsed_time(b) for a, b in kev]
    tab_ms = [ev[k][0].elapsed_time(kev[k][0]) for k in range(args.steps)]
    total_s = sum(step_ms) / 1e3
    if dist:
        t = torch.tensor([total_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * ncand * args.steps / total_s
    n_surv = int(count.item())

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(scr, torch, ctx, wl, tm, p, cap, ncand, args)
    if rank == 0:
        emit(args, wl, world, total_s, value, k3_ms, step_ms, launches, clk, n_surv, e2e, tab_ms)
    scr.template_release(ctx, tm)
    scr.screen_shutdown(ctx)
    if dist:
        dist.destroy_process_group()


def run_e2e(scr, torch, ctx, wl, tm, p, cap, ncand, args):
    H, W = wl.image.shape
    img_host = torch.from_numpy(wl.image).pin_memory()
    lst_host = torch.empty(cap, dtype=torch.int64).pin_memory()
    for _ in range(2):
        scr.screen_host(ctx, img_host.numpy(), wl.sum_bits, wl.sq_bits, tm, p, lst_host.numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(10, min(args.steps, 100))
    for _ in range(e2e_steps):
        n_e2e, _ = scr.screen_host(ctx, img_host.numpy(), wl.sum_bits, wl.sq_bits, tm, p, lst_host.numpy())
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    return {"value": ncand / e2e_s, "unit": UNIT, "h2d_bytes_per_step": H * W,
            "d2h_bytes_per_step": 8 + 8 * min(n_e2e, cap), "steps": e2e_steps}


def emit(args, wl, world, total_s, value, k3_ms, step_ms, launches, clk, n_surv, e2e, tab_ms):
    H, W = wl.image.shape
    S = len(wl.radii)
    peak, src = measured_peak_gbs()
    k3 = statistics.mean(k3_ms) / 1e3
    alg = compulsory_bytes(H, W, S, wl.sum_bits, wl.sq_bits, n_surv)
    achieved = alg / k3 / 1e9
    alg1 = per_scale_bytes(H, W, S, wl.sum_bits, wl.sq_bits) / k3 / 1e9
    traffic = recorded_traffic(H, W)
    ncand = candidates(H, W, wl.radii)
    per_scale_model = ("Algorithm 1 per-scale: the 4 full-width tables read once per scale + mask "
                       f"({per_scale_bytes(H, W, S, wl.sum_bits, wl.sq_bits) / ncand:.1f} B/candidate)")
    compulsory = {"achieved": achieved, "frac": achieved / peak,
                  "model": f"compulsory (tables once across scales + mask + list): {alg} B/launch, "
                           f"{alg / ncand:.2f} B/candidate"}
    binding = ("on-chip: L1/L2 load latency and the L1 data pipe; DRAM traffic is the low "
               "planes of L1 and T1 once (ncu: L1 LSU wavefronts 66%, L1/TEX 72%, ALU pipe 52%, "
               "issue 62%, L2 48% of peak on the 3072^2 case)")
    if alg1 <= peak:
        # Algorithm 1's per-scale traffic, served partly from L2: the fraction of the HBM roof
        # that model implies (kept only while it stays below 1)
        roofline = {"bound": "hbm", "achieved": alg1, "peak": peak, "unit": "GB/s", "frac": alg1 / peak,
                    "traffic": traffic, "peak_source": src, "kernel": "k_screen", "kernel_ms": 1e3 * k3,
                    "model": per_scale_model, "compulsory": compulsory, "binding": binding}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "peak_source": src, "kernel": "k_screen", "kernel_ms": 1e3 * k3,
                    "model": compulsory["model"], "per_scale_above_peak": {"achieved": alg1, "model": per_scale_model},
                    "binding": binding}
    # table build: 1 B/px read + the four tables written, over the measured build time
    tb_s = statistics.mean(tab_ms) / 1e3
    tb_bytes = H * W + ((H + 1) * (W + 1) + (H + 1) * (W + 2)) * (wl.sum_bits + wl.sq_bits) // 8
    tables_roofline = {"bound": "hbm", "achieved": tb_bytes / tb_s / 1e9, "peak": peak, "unit": "GB/s",
                       "frac": tb_bytes / tb_s / 1e9 / peak, "build_ms": 1e3 * tb_s,
                       "model": f"1 B/px image read + tables written: {tb_bytes} B per build",
                       "kernels": "k_tab_reduce, k_tab_carry, k_tab_prefix, k_tab_write"}
    cpu = None
    if not args.no_cpu_baseline:
        split, split1 = {}, {}
        v, sample, cores, dt = oracle_baseline(wl, split=split, min_seconds=10.0)
        v1, sample1, _, dt1 = oracle_baseline(wl, 1024, threads=1, split=split1, min_seconds=10.0)
        oracle_threads(cores)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "seconds": round(dt, 2), "tables_s": round(split["tables_s"], 3),
               "screen_s": round(split["screen_s"], 3),
               "single_thread": {"value": v1, "sample": sample1, "seconds": round(dt1, 2),
                                 "tables_s": round(split1["tables_s"], 3), "screen_s": round(split1["screen_s"], 3)}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32+u64", "data": "synthetic",
        "config": config_dict(wl),
        "roofline": roofline,
        "tables_roofline": tables_roofline,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk.summary(), "survivors": n_surv,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
    }
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Configuration 4: many images x many templates, one batched run (CUDA graph)
    against per-request plain launches (screen_features + compact_mask per pair)
    on the same data, same outputs, same exactness."""
    import torch
    import synth
    import paper_1707_05647_gb300 as scr

    torch.cuda.set_device(0)
    bw = synth.batch_workload(n_images=args.images, n_templates=args.templates)
    pairs = bw.pairs
    ctx = scr.screen_init(0, 0)
    stream = torch.cuda.current_stream()
    tables = [scr.build_tables(ctx, torch.from_numpy(im).cuda(), bw.sum_bits, bw.sq_bits, stream) for im in bw.images]
    tmpls = [scr.template_features(ctx, ts.template, ts.r, max(ts.t_min, 2), bw.features) for ts in bw.templates]
    params = [scr.Params(ts.radii, bw.features, bw.tol.mean_rel, bw.tol.std_rel, bw.tol.grad_rel, bw.tol.grad_abs)
              for ts in bw.templates]
    n = len(pairs)
    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    offsets = torch.zeros(n, dtype=torch.int64, device="cuda")
    uw = sum(im.shape[0] * ((im.shape[1] + 31) // 32) for im in bw.images)
    union = torch.zeros(uw, dtype=torch.int32, device="cuda")
    nk = torch.zeros(2, dtype=torch.int64, device="cuda")

    def create(cap):
        keys = torch.zeros(max(cap, 1), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = scr.screen_batch_create(ctx, tables, tmpls, params, pairs, counts, keys, nk, offsets=offsets,
                                    union_mask=union, stream=stream)
        torch.cuda.synchronize()
        return b, keys, time.perf_counter() - t0

    # a first plan (tuned now) learns how many key slots a complete run needs;
    # the timed plan holds every survivor's key
    b, keys, plan_s = create(1 << 20)
    scr.screen_batch_run(b, stream)
    torch.cuda.synchronize()
    need = int(nk[1].item())
    if need > keys.numel():
        scr.screen_batch_release(ctx, b)
        del keys
        b, keys, plan_cached_s = create(((need >> 20) + 1) << 20)
    else:
        plan_cached_s = None
    info = scr.screen_batch_info(b)
    for _ in range(args.warmup):
        scr.screen_batch_run(b, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            scr.screen_batch_run(b, stream)
        e1.record(stream)
        torch.cuda.synchronize()
    batch_s = e0.elapsed_time(e1) / 1e3 / args.steps
    n_keys = int(nk[0].item())
    # per-request plain launches on the same pairs
    maxw = max(len(ts.radii) * im.shape[0] * ((im.shape[1] + 31) // 32)
               for im in bw.images for ts in bw.templates)
    mask = torch.empty(maxw, dtype=torch.int32, device="cuda")
    plst = torch.empty(max(1, int(counts.max().item())), dtype=torch.int64, device="cuda")
    pcnt = torch.zeros(n, dtype=torch.int64, device="cuda")

    def per_request():
        for p, (i, t) in enumerate(pairs):
            H, W = bw.images[i].shape
            S = len(bw.templates[t].radii)
            scr.screen_features(ctx, tables[i], tmpls[t], params[t], mask[:scr.mask_words(S, H, W)], stream)
            scr.compact_mask(ctx, mask, S, H, W, plst, pcnt[p:p + 1], stream)

    per_request()
    torch.cuda.synchronize()
    e0.record(stream)
    per_request()
    e1.record(stream)
    torch.cuda.synchronize()
    req_s = e0.elapsed_time(e1) / 1e3
    same = bool(torch.equal(pcnt, counts))
    print(json.dumps({
        "metric": METRIC, "workload": f"batched: {len(bw.images)} images (640x480..4096x3072, log-uniform) x "
                                      f"{len(bw.templates)} templates (r 8..64, 1..16 scales in [0.5, 2]), all pairs",
        "value": info["candidates"] / batch_s, "unit": UNIT, "ms_per_run": 1e3 * batch_s, "runs": args.steps,
        "per_request": {"value": info["candidates"] / req_s, "ms": 1e3 * req_s,
                        "how": "screen_features + compact_mask per pair (complete lists), stream-ordered, no host sync"},
        "speedup_vs_per_request": req_s / batch_s, "counts_identical": same,
        "candidates": info["candidates"], "survivors": n_keys, "keys_complete": int(nk[1].item()) <= keys.numel(),
        "plan": info, "plan_seconds": plan_s, "plan_seconds_tuned_cached": plan_cached_s,
        "clocks": clk.summary(), "data": "synthetic"}), flush=True)
    scr.screen_batch_release(ctx, b)
    scr.screen_shutdown(ctx)


def run_joint(args):
    """The joint-vector membership screen (three nested central areas, q = 4, 2,
    4 grey levels) on the 4096^2 workload, beside the interval screen on the
    same tables and the interval screen with the Prewitt test added (plus the
    moment-table build): device time per screen with CUDA events, survivors of
    each."""
    import torch
    import synth
    from fractions import Fraction
    import paper_1707_05647_gb300 as scr

    torch.cuda.set_device(0)
    wl = synth.config2()
    H, W = wl.image.shape
    S = len(wl.radii)
    area_radii, bands = synth.joint_areas(wl.r, wl.scales, 3)
    t_min = max(2, min(b[0] for b in bands))
    q = (Fraction(4), Fraction(2), Fraction(4))
    ctx = scr.screen_init(0, 0)
    st = torch.cuda.current_stream()
    tab = scr.build_tables(ctx, torch.from_numpy(wl.image).cuda(), wl.sum_bits, wl.sq_bits, st)
    tm = scr.template_features(ctx, wl.template, wl.r, t_min, wl.features)
    pj = scr.Params(wl.radii, wl.features)
    pi = scr.Params(wl.radii, wl.features, wl.tol.mean_rel, wl.tol.std_rel, wl.tol.grad_rel, wl.tol.grad_abs)
    tmi = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    mask = torch.empty(scr.mask_words(S, H, W), dtype=torch.int32, device="cuda")
    lst = torch.empty(1 << 24, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / args.steps

    joint_s = timed(lambda: scr.screen_joint(ctx, tab, tm, pj, area_radii, bands, q, mask, st))
    scr.compact_mask(ctx, mask, S, H, W, lst, cnt, st)
    torch.cuda.synchronize()
    n_joint = int(cnt.item())
    py, px = wl.planted
    m = mask.cpu().numpy().view(np.uint32).reshape(S, H, (W + 31) // 32)
    planted = any((int(m[s, py, px >> 5]) >> (px & 31)) & 1 for s in range(S))
    # the interval screen with the Prewitt test of the star's square added
    dimg = torch.from_numpy(wl.image).cuda()
    scr.build_moment_tables(ctx, tab, dimg, st)
    tmp = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features | scr.F_PREWITT)
    pp = scr.Params(wl.radii, wl.features | scr.F_PREWITT, wl.tol.mean_rel, wl.tol.std_rel, wl.tol.grad_rel,
                    wl.tol.grad_abs, Fraction(1, 10), Fraction(2))
    pw_s = timed(lambda: scr.screen_features(ctx, tab, tmp, pp, mask, st))
    scr.compact_mask(ctx, mask, S, H, W, lst, cnt, st)
    torch.cuda.synchronize()
    n_pw = int(cnt.item())
    m = mask.cpu().numpy().view(np.uint32).reshape(S, H, (W + 31) // 32)
    planted_pw = any((int(m[s, py, px >> 5]) >> (px & 31)) & 1 for s in range(S))
    mom_s = timed(lambda: scr.build_moment_tables(ctx, tab, dimg, st))
    int_s = timed(lambda: scr.screen_features(ctx, tab, tmi, pi, mask, st))
    scr.compact_mask(ctx, mask, S, H, W, lst, cnt, st)
    torch.cuda.synchronize()
    n_int = int(cnt.item())
    cand = 127458510
    print(json.dumps({
        "metric": "candidate (position x scale) evaluations/s", "workload":
            "joint membership: 4096x4096, r 48, 8 scales, 3 nested central areas, q = (4, 2, 4) grey levels",
        "value": cand / joint_s, "unit": "evals/s", "ms_per_screen": 1e3 * joint_s, "steps": args.steps,
        "survivors": n_joint, "pruned": 1 - n_joint / cand, "planted_survives": bool(planted),
        "interval_screen": {"ms_per_screen": 1e3 * int_s, "value": cand / int_s, "survivors": n_int,
                            "pruned": 1 - n_int / cand},
        "interval_with_prewitt": {"ms_per_screen": 1e3 * pw_s, "value": cand / pw_s, "survivors": n_pw,
                                  "planted_survives": bool(planted_pw), "moment_tables_ms": 1e3 * mom_s,
                                  "moment_tables_GBps": 2 * (H + 1) * (W + 1) * 8 / mom_s / 1e9},
        "data": "synthetic"}), flush=True)
    scr.screen_shutdown(ctx)


def run_serve(args):
    """Configuration 5: replay one seeded Poisson stream of uploads and screens
    through the serving loop, batched (continuous batching) and plain (one
    launch pair per screen), each on a fresh server warmed to the same resident
    set; latency = done - scheduled arrival, so a late submission counts."""
    import queue
    import threading
    import torch
    import synth
    import paper_1707_05647_gb300 as scr

    torch.cuda.set_device(0)
    rates = [float(r) for r in args.rates.split(",")]
    w = synth.serve_workload(duration=args.duration, rate=rates[0])
    ctx = scr.screen_init(0, 0)
    tmpls = [scr.template_features(ctx, ts.template, ts.r, max(ts.t_min, 2), 7) for ts in w.templates]
    params = {}
    for ev in w.events:
        if ev.kind == "screen" and (ev.template, ev.features) not in params:
            ts = w.templates[ev.template]
            params[(ev.template, ev.features)] = scr.Params(ts.radii, ev.features, w.tol.mean_rel, w.tol.std_rel,
                                                             w.tol.grad_rel, w.tol.grad_abs)
    cap = 1 << 18
    n_bufs = 1024   # list buffers in flight (2 GiB of host memory)

    def candidates(img_shape, radii):
        H, W = img_shape
        tot = 0
        for R in radii:
            n = scr_square_half(R)
            m = max(n, R)
            rows = (H - 1 - m) - (m - 1) + 1
            cols = min(W - 1 - n, W - R) - (m - 1) + 1
            tot += max(rows, 0) * max(cols, 0)
        return tot

    def replay(mode):
        s = scr.server_create(ctx, table_budget_bytes=w.table_budget, sum_bits=w.sum_bits, sq_bits=w.sq_bits,
                              mode=mode)
        uploads = []   # image id per upload, in order
        pending = []
        for k in w.warm:
            iid, rid = scr.server_upload(s, w.pool[k], borrow=True)
            uploads.append((iid, w.pool[k].shape))
            pending.append(rid)
        for rid in pending:
            r = scr.server_wait(s, rid)
            assert r["status"] == scr.SCR_OK, r
        warm_stats = scr.server_stats(s)
        bufs = queue.Queue()
        for _ in range(n_bufs):
            bufs.put(np.zeros(cap, np.uint64))
        results = {}
        lock = threading.Lock()
        meta, early = {}, {}          # request id -> (event index, buffer); results seen before their id
        state = {"done": 0, "expected": None}

        def record(k, buf, res):      # lock held
            results[k] = res
            state["done"] += 1
            if buf is not None:
                bufs.put(buf)

        def collect():                # completion order: a slow request holds no one else's buffer
            while True:
                with lock:
                    if state["expected"] is not None and state["done"] >= state["expected"]:
                        return
                try:
                    rid, res = scr.server_next(s, 100_000)
                except scr.ScreenError as e:
                    if e.code == scr.SCR_ETIMEOUT:
                        continue
                    raise
                with lock:
                    if rid in meta:
                        k, buf = meta.pop(rid)
                        record(k, buf, res)
                    else:
                        early[rid] = res

        th = threading.Thread(target=collect)
        th.start()
        t0 = scr.server_clock_ns() + 50_000_000
        cand = {}
        for k, ev in enumerate(w.events):
            due = t0 + int(ev.t * 1e9)
            while True:
                now = scr.server_clock_ns()
                if now >= due:
                    break
                if due - now > 300_000:
                    time.sleep((due - now - 200_000) / 1e9)
            if ev.kind == "upload":
                iid, rid = scr.server_upload(s, w.pool[ev.image], borrow=True, arrival_ns=due)
                uploads.append((iid, w.pool[ev.image].shape))
                buf = None
            else:
                iid, shape = uploads[ev.image]
                buf = bufs.get()
                rid = scr.server_screen(s, iid, tmpls[ev.template], params[(ev.template, ev.features)], buf,
                                        arrival_ns=due)
                cand[k] = candidates(shape, w.templates[ev.template].radii)
            with lock:
                if rid in early:
                    record(k, buf, early.pop(rid))
                else:
                    meta[rid] = (k, buf)
        with lock:
            state["expected"] = len(w.events)
        th.join()
        st = scr.server_stats(s)
        scr.server_destroy(s)
        scr_lat = np.array([(results[k]["done_ns"] - results[k]["arrival_ns"]) / 1e6 for k in cand])
        rebuilt = np.array([results[k]["built"] == 1 for k in cand])
        queue_ms = np.array([(results[k]["start_ns"] - results[k]["arrival_ns"]) / 1e6 for k in cand])
        up_lat = np.array([(results[k]["done_ns"] - results[k]["arrival_ns"]) / 1e6
                           for k, ev in enumerate(w.events) if ev.kind == "upload"])
        bad = sum(1 for r in results.values() if r["status"] not in (scr.SCR_OK, scr.SCR_EOVERFLOW))
        end = max(r["done_ns"] for r in results.values())
        span = (end - t0) / 1e9
        counts = {k: results[k]["count"] for k in cand}
        sizes = np.array([r["batch_size"] for r in results.values()])
        return {
            "screen_latency_ms": {"p50": float(np.percentile(scr_lat, 50)), "p99": float(np.percentile(scr_lat, 99)),
                                  "mean": float(scr_lat.mean()), "max": float(scr_lat.max())},
            "upload_latency_ms": {"p50": float(np.percentile(up_lat, 50)), "p99": float(np.percentile(up_lat, 99))},
            "screens_waiting_for_rebuild": int(rebuilt.sum()),
            "screen_latency_no_rebuild_ms": {"p50": float(np.percentile(scr_lat[~rebuilt], 50)),
                                             "p99": float(np.percentile(scr_lat[~rebuilt], 99))},
            "screen_start_delay_ms": {"p50": float(np.percentile(queue_ms, 50)),
                                      "p99": float(np.percentile(queue_ms, 99))},
            "builder_busy": (st["build_ns"] - warm_stats["build_ns"]) / 1e9 / span,
            "screener_busy": (st["screen_ns"] - warm_stats["screen_ns"]) / 1e9 / span,
            "screener_us_per_batch": {k: (st[k + "_ns"] - warm_stats[k + "_ns"]) / 1e3 / max(1, st["batches"] -
                                                                                       warm_stats["batches"])
                                      for k in ("plan", "wait", "copy")},
            "builder_us_per_build": {k: (st[k] - warm_stats[k]) / 1e3 / max(1, st["builds"] - warm_stats["builds"])
                                     for k in ("build_ns", "build_copy_ns", "build_alloc_ns", "build_run_ns",
                                               "build_gpu_ns")},
            "evals_per_s": sum(cand.values()) / span, "requests_per_s": len(w.events) / span,
            "span_s": span, "errors": bad,
            "overflowed_lists": sum(1 for k in cand if results[k]["status"] == scr.SCR_EOVERFLOW),
            "batches": st["batches"] - warm_stats["batches"], "mean_batch_size": float(sizes.mean()),
            "evictions": st["evictions"], "rebuilds": st["rebuilds"], "builds": st["builds"],
            "peak_resident_gb": st["peak_resident_bytes"] / 1e9, "launches": st["launches"] - warm_stats["launches"],
        }, counts

    batched, cb = replay(scr.SERVE_BATCHED)
    plain, cp = replay(scr.SERVE_PLAIN)
    n_screens = sum(1 for e in w.events if e.kind == "screen")
    head = w
    sweep = []
    for rate in rates[1:]:
        # same seed: same image pool, templates and warm set; a denser stream
        w = synth.serve_workload(duration=args.duration, rate=rate)
        assert [t.r for t in w.templates] == [t.r for t in head.templates]
        params.update({(ev.template, ev.features): scr.Params(w.templates[ev.template].radii, ev.features,
                                                               w.tol.mean_rel, w.tol.std_rel, w.tol.grad_rel,
                                                               w.tol.grad_abs)
                       for ev in w.events if ev.kind == "screen" and (ev.template, ev.features) not in params})
        b2, c2b = replay(scr.SERVE_BATCHED)
        p2, c2p = replay(scr.SERVE_PLAIN)
        sweep.append({"rate": rate, "requests": len(w.events), "counts_identical": c2b == c2p,
                      "batched": {k: b2[k] for k in ("screen_latency_ms", "evals_per_s", "requests_per_s",
                                                     "mean_batch_size", "errors")},
                      "plain": {k: p2[k] for k in ("screen_latency_ms", "evals_per_s", "requests_per_s",
                                                   "mean_batch_size", "errors")}})
    w = head
    print(json.dumps({
        "metric": "served screen latency p50/p99 (ms) and evaluations/s", "workload":
            f"serving: Poisson {w.rate:.0f} req/s for {w.duration:g} s ({len(w.events)} requests, "
            f"{len(w.events) - n_screens} uploads of side 256..8192 log-uniform, {n_screens} screens r 8..96, "
            f"1..16 scales, 2-3 features), {w.table_budget >> 30} GiB table budget, LRU eviction, "
            f"{len(w.warm)} warm uploads",
        "batched": batched, "plain": plain,
        "p99_speedup_vs_plain": plain["screen_latency_ms"]["p99"] / batched["screen_latency_ms"]["p99"],
        "p50_speedup_vs_plain": plain["screen_latency_ms"]["p50"] / batched["screen_latency_ms"]["p50"],
        "counts_identical": cb == cp, "list_cap": cap, "load_sweep": sweep, "data": "synthetic"}), flush=True)
    for t in tmpls:
        scr.template_release(ctx, t)
    scr.screen_shutdown(ctx)


def scr_square_half(R: int) -> int:
    """n with (2n-1)^2 < 2R^2 < (2n+1)^2, for counting valid positions in reports."""
    m = math.isqrt(2 * R * R)
    return (m + 1) // 2


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--size", type=int, default=4096,
                    help="crop the 4096x4096 image to size x size (smaller ncu captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "serve", "joint"])
    ap.add_argument("--duration", type=float, default=2.0, help="seconds of arrivals (serve workload)")
    ap.add_argument("--rates", default="2000,8000,16000",
                    help="arrival rates (req/s) of the serve workload; the first is the headline")
    ap.add_argument("--images", type=int, default=64)
    ap.add_argument("--templates", type=int, default=256)
    args = ap.parse_args()
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "joint":
        run_joint(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
