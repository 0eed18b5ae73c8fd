"""Seeded synthetic inputs for the screening path.

This module holds the input recipes only: images, templates, planted copies,
the scale lists and the tolerance rationals.  It contains none of the
screening arithmetic (no tables, no window sums, no features, no bounds), so
the CPU oracle and the CUDA path can both read its outputs without sharing any
of the method's code.

Workload shapes follow the paper's experiments (640x480 .. 1280x960 images,
32^2 .. 128^2 templates, scale range [0.5, 2], Table 1 of Sec. 6) scaled to the
five benchmark configurations below.  The paper's own datasets (MIT CSAIL,
VTB) are not available; these seeded blob fields stand in for them.

Image recipe (all configurations):
  float field = 128 + sum of 64 Gaussian blobs, centre uniform over the image,
  sigma ~ U[4, 40] px, amplitude ~ U[-96, 96] (each blob evaluated inside
  +-4 sigma); planted copies are written into the float field; then integer
  noise ~ U{-8..8} is added, the result rounded and clipped to 0..255.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

F_MEAN, F_VAR, F_GRAD = 1, 2, 4

BASE_SEED = 1000


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def blob_field(rng: np.random.Generator, H: int, W: int, n_blobs: int = 64,
               sigma=(4.0, 40.0), amp=(-96.0, 96.0), base: float = 128.0) -> np.ndarray:
    """Float64 H x W field: base + n_blobs isotropic Gaussian bumps."""
    f = np.full((H, W), base, dtype=np.float64)
    cy = rng.uniform(0, H, n_blobs)
    cx = rng.uniform(0, W, n_blobs)
    sg = rng.uniform(sigma[0], sigma[1], n_blobs)
    am = rng.uniform(amp[0], amp[1], n_blobs)
    for k in range(n_blobs):
        rad = 4.0 * sg[k]
        y0 = max(0, int(math.floor(cy[k] - rad)))
        y1 = min(H, int(math.ceil(cy[k] + rad)) + 1)
        x0 = max(0, int(math.floor(cx[k] - rad)))
        x1 = min(W, int(math.ceil(cx[k] + rad)) + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1, dtype=np.float64)[:, None] - cy[k]
        xx = np.arange(x0, x1, dtype=np.float64)[None, :] - cx[k]
        f[y0:y1, x0:x1] += am[k] * np.exp(-(yy * yy + xx * xx) / (2.0 * sg[k] * sg[k]))
    return f


def quantize_with_noise(f: np.ndarray, rng: np.random.Generator, noise: int = 8) -> np.ndarray:
    """Add integer noise U{-noise..noise}, round half away from zero, clip to uint8."""
    nz = rng.integers(-noise, noise + 1, size=f.shape, dtype=np.int16)
    g = np.floor(f + nz + 0.5)
    return np.clip(g, 0, 255).astype(np.uint8)


def bilinear(src: np.ndarray, ys: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """Bilinear sample of a 2-D float array at fractional (ys, xs) inside [0, n-1]."""
    h, w = src.shape
    y0 = np.clip(np.floor(ys).astype(np.int64), 0, h - 2)
    x0 = np.clip(np.floor(xs).astype(np.int64), 0, w - 2)
    fy = ys - y0
    fx = xs - x0
    a = src[y0, x0]
    b = src[y0, x0 + 1]
    c = src[y0 + 1, x0]
    d = src[y0 + 1, x0 + 1]
    return (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy


def plain_std(a: np.ndarray) -> float:
    """Plain population std of all pixels of a patch (template texture floor)."""
    return float(np.asarray(a, dtype=np.float64).std())


def paste(field_: np.ndarray, tmpl: np.ndarray, cy: float, cx: float, theta: float,
          scale: float, gain: float = 1.0) -> None:
    """Write a rotated, scaled copy of `tmpl` into the float field, in place.

    The template point q maps to image point c_I + scale * Rot(theta) (q - c_T),
    with c_T = (r + 1/2, r + 1/2) the template's star centre and c_I = (cy, cx).
    Every image pixel whose pre-image falls inside the template square takes the
    bilinear sample of the template there (times `gain`).
    """
    side = tmpl.shape[0]
    r = (side - 1) // 2
    cT = r + 0.5
    H, W = field_.shape
    ext = scale * (side + 2) * math.sqrt(2.0) / 2.0 + 2.0
    y0 = max(0, int(math.floor(cy - ext)))
    y1 = min(H, int(math.ceil(cy + ext)) + 1)
    x0 = max(0, int(math.floor(cx - ext)))
    x1 = min(W, int(math.ceil(cx + ext)) + 1)
    py, px = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    dy = (py - cy) / scale
    dx = (px - cx) / scale
    c, s = math.cos(theta), math.sin(theta)
    # inverse rotation Rot(-theta) applied to (dy, dx)
    qy = cT + c * dy + s * dx
    qx = cT - s * dy + c * dx
    inside = (qy >= 0) & (qy <= side - 1) & (qx >= 0) & (qx <= side - 1)
    vals = bilinear(tmpl.astype(np.float64), qy[inside], qx[inside])
    sub = field_[y0:y1, x0:x1]
    sub[inside] = gain * vals


def geometric_scales(s_min: float, s_max: float, count: int) -> list[float]:
    if count == 1:
        return [s_min]
    return [s_min * (s_max / s_min) ** (i / (count - 1)) for i in range(count)]


def radii_for(r: int, scales: list[float]) -> list[int]:
    """Star radius per scale, R_s = floor(r * s + 1/2)."""
    return [int(math.floor(r * s + 0.5)) for s in scales]


def t_min_for(r: int, scales: list[float]) -> int:
    """Smallest template central radius of a scale band, ceil(r / lambda)."""
    if len(scales) < 2:
        return r
    lam = scales[1] / scales[0]
    return int(math.ceil(r / lam - 1e-9))


@dataclass
class Tolerances:
    mean_rel: Fraction = Fraction(1, 20)
    std_rel: Fraction = Fraction(1, 10)
    grad_rel: Fraction = Fraction(1, 10)
    grad_abs: Fraction = Fraction(4, 1)


@dataclass
class Workload:
    name: str
    image: np.ndarray                 # uint8 H x W
    template: np.ndarray              # uint8 (2r+1) x (2r+1)
    r: int
    radii: list[int]
    t_min: int
    features: int
    tol: Tolerances
    sum_bits: int
    sq_bits: int
    planted: tuple[int, int]          # candidate (y*, x*) of the true match
    s_true: float
    theta: float
    scales: list[float] = field(default_factory=list)
    distractors: list[tuple[int, int, float, float]] = field(default_factory=list)   # (y, x, gain, scale)


def _pick_site(rng, H, W, side, margin, floor_std, img, tries=400):
    best = None
    for _ in range(tries):
        y0 = int(rng.integers(margin, H - margin - side))
        x0 = int(rng.integers(margin, W - margin - side))
        sd = plain_std(img[y0:y0 + side, x0:x0 + side])
        if best is None or sd > best[0]:
            best = (sd, y0, x0)
        if sd >= floor_std:
            return y0, x0
    return best[1], best[2]


def config1(seed: int = BASE_SEED + 0) -> Workload:
    """512x512 image, 33x33 rotated template cut from the image, R = 16, 1 scale."""
    rng = rng_for(seed)
    H = W = 512
    img = quantize_with_noise(blob_field(rng, H, W), rng)
    big, r = 49, 16
    side = 2 * r + 1
    off = (big - side) // 2
    # texture floor on the central 33x33 part of the cut
    y0, x0 = _pick_site(rng, H, W, big, 8, 16.0, img)
    while plain_std(img[y0 + off:y0 + off + side, x0 + off:x0 + off + side]) < 16.0:
        y0, x0 = _pick_site(rng, H, W, big, 8, 16.0, img)
    patch = img[y0:y0 + big, x0:x0 + big].astype(np.float64)
    theta = float(rng.uniform(0.0, 2.0 * math.pi))
    c = (big - 1) / 2.0 + 0.5          # 24.5: star centre of candidate (24, 24)
    ii, jj = np.mgrid[0:side, 0:side].astype(np.float64)
    dy = ii + off - c
    dx = jj + off - c
    cs, sn = math.cos(theta), math.sin(theta)
    sy = c + cs * dy - sn * dx
    sx = c + sn * dy + cs * dx
    tm = np.clip(np.floor(bilinear(patch, sy, sx) + 0.5), 0, 255).astype(np.uint8)
    return Workload(name="512x512, R=16, 1 scale, mean+var, u32/u32",
                    image=img, template=tm, r=r, radii=[16], t_min=16,
                    features=F_MEAN | F_VAR, tol=Tolerances(), sum_bits=32, sq_bits=32,
                    planted=(y0 + 24, x0 + 24), s_true=1.0, theta=theta, scales=[1.0])


def _template_from_source(rng, r, src_side=512):
    side = 2 * r + 1
    src = quantize_with_noise(blob_field(rng, src_side, src_side), rng)
    y0, x0 = _pick_site(rng, src_side, src_side, side, 4, 16.0, src)
    return src[y0:y0 + side, x0:x0 + side].copy()


def _planted_workload(name, seed, H, r, s_min, s_max, n_scales, sum_bits, sq_bits,
                      n_distractors=0, distractor_gain=0.03, true_range=(0.5, 2.0)) -> Workload:
    rng = rng_for(seed)
    W = H
    fld = blob_field(rng, H, W)
    trng = rng_for(seed + 7919)
    tmpl = _template_from_source(trng, r)
    s_true = float(math.exp(rng.uniform(math.log(true_range[0]), math.log(true_range[1]))))
    theta = float(rng.uniform(0.0, 2.0 * math.pi))
    side = 2 * r + 1
    margin = int(math.ceil(s_max * side)) + 8
    ys = int(rng.integers(margin, H - margin))
    xs = int(rng.integers(margin, W - margin))
    distractors = []
    for _ in range(n_distractors):
        dy = int(rng.integers(margin, H - margin))
        dx = int(rng.integers(margin, W - margin))
        g = 1.0 + (distractor_gain if rng.integers(0, 2) else -distractor_gain)
        d_theta = float(rng.uniform(0, 2 * math.pi))
        d_scale = float(math.exp(rng.uniform(math.log(0.5), math.log(2.0))))
        paste(fld, tmpl, dy + 0.5, dx + 0.5, d_theta, d_scale, gain=g)
        distractors.append((dy, dx, g, d_scale))
    # the true copy is pasted last so no distractor overwrites it
    paste(fld, tmpl, ys + 0.5, xs + 0.5, theta, s_true)
    img = quantize_with_noise(fld, rng)
    scales = geometric_scales(s_min, s_max, n_scales)
    return Workload(name=name, image=img, template=tmpl, r=r, radii=radii_for(r, scales),
                    t_min=t_min_for(r, scales), features=F_MEAN | F_VAR | F_GRAD,
                    tol=Tolerances(), sum_bits=sum_bits, sq_bits=sq_bits,
                    planted=(ys, xs), s_true=s_true, theta=theta, scales=scales,
                    distractors=distractors)


def config2(seed: int = BASE_SEED + 1) -> Workload:
    """4096x4096, planted r=48 template, 8 scales 0.5..2, 3 features, u32 sum / u64 sum^2."""
    return _planted_workload("4096x4096, r=48, 8 scales 0.5-2, 3 features, u32/u64",
                             seed, 4096, 48, 0.5, 2.0, 8, 32, 64)


def config3(seed: int = BASE_SEED + 2) -> Workload:
    """8192x8192, r=64, 16 scales 0.35..2.8, 3 features, u64/u64, 8 distractors (+-3%)."""
    return _planted_workload("8192x8192, r=64, 16 scales 0.35-2.8, 3 features, u64/u64",
                             seed, 8192, 64, 0.35, 2.8, 16, 64, 64, n_distractors=8)


def small_planted(seed: int, H: int = 384, r: int = 20, n_scales: int = 4,
                  s_min: float = 0.6, s_max: float = 1.6, sum_bits: int = 32,
                  sq_bits: int = 64) -> Workload:
    """Reduced planted workload (config 2's recipe at a size the oracle finishes fast)."""
    return _planted_workload(f"{H}x{H}, r={r}, {n_scales} scales", seed, H, r, s_min, s_max,
                             n_scales, sum_bits, sq_bits, true_range=(s_min, s_max))


def random_image(seed: int, H: int, W: int, kind: str = "uniform") -> np.ndarray:
    """Small seeded test images: uniform noise, constant, ramps, blobs."""
    rng = rng_for(seed)
    if kind == "uniform":
        return rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    if kind == "blobs":
        return quantize_with_noise(blob_field(rng, H, W, n_blobs=max(4, H * W // 4096)), rng)
    if kind == "max":
        return np.full((H, W), 255, dtype=np.uint8)
    if kind == "zero":
        return np.zeros((H, W), dtype=np.uint8)
    raise ValueError(kind)


CONFIGS = {1: config1, 2: config2, 3: config3}


@dataclass
class TemplateSpec:
    template: np.ndarray          # uint8 (2r+1) x (2r+1)
    r: int
    scales: list[float]
    radii: list[int]
    t_min: int


@dataclass
class BatchWorkload:
    """Many images of uneven size against many templates (gallery search)."""
    images: list[np.ndarray]
    templates: list[TemplateSpec]
    pairs: list[tuple[int, int]]                 # (image index, template index)
    features: int
    tol: Tolerances
    sum_bits: int
    sq_bits: int
    plants: list[list[tuple[int, int, int, float]]]   # per image: (template, y, x, scale)


def _batch_templates(rng, n, r_range, scale_range, max_scales):
    out = []
    for k in range(n):
        r = int(rng.integers(r_range[0], r_range[1] + 1))
        ns = int(rng.integers(1, max_scales + 1))
        if ns == 1:
            scales = [1.0]
        else:
            scales = geometric_scales(scale_range[0], scale_range[1], ns)
        trng = rng_for(int(rng.integers(0, 2 ** 31)))
        tm = _template_from_source(trng, r, src_side=max(192, 4 * (2 * r + 1)))
        out.append(TemplateSpec(tm, r, scales, radii_for(r, scales), t_min_for(r, scales)))
    return out


def batch_workload(seed: int = BASE_SEED + 3, n_images: int = 64, n_templates: int = 256,
                   area_range=(640 * 480, 4096 * 3072), r_range=(8, 64), scale_range=(0.5, 2.0),
                   max_scales: int = 16, plants_per_image: int = 4, all_pairs: bool = True) -> BatchWorkload:
    """Configuration 4: images with log-uniform area (4:3), templates with r ~ U{8..64}
    and 1..16 geometric scales in [0.5, 2]; 4 planted copies per image, placed
    so that no two copies overlap (a copy that fits nowhere is left out)."""
    rng = rng_for(seed)
    templates = _batch_templates(rng, n_templates, r_range, scale_range, max_scales)
    images, plants = [], []
    for _ in range(n_images):
        area = math.exp(rng.uniform(math.log(area_range[0]), math.log(area_range[1])))
        H = max(8, int(round(math.sqrt(area * 3.0 / 4.0))))
        W = max(8, int(round(H * 4.0 / 3.0)))
        fld = blob_field(rng, H, W)
        pl, placed = [], []
        for _p in range(plants_per_image):
            t = int(rng.integers(0, n_templates))
            ts = templates[t]
            s = float(math.exp(rng.uniform(math.log(ts.scales[0]), math.log(ts.scales[-1] * 1.0001))))
            margin = int(math.ceil(s * (2 * ts.r + 1))) + 4
            if H <= 2 * margin or W <= 2 * margin:
                continue
            # copies do not overlap: a later paste would overwrite part of an
            # earlier copy (reach = half-diagonal of the pasted square)
            reach = s * (2 * ts.r + 1) * math.sqrt(0.5) + 2
            for _try in range(64):
                y = int(rng.integers(margin, H - margin))
                x = int(rng.integers(margin, W - margin))
                if all(math.hypot(y - py, x - px) > reach + pr for (py, px, pr) in placed):
                    break
            else:
                continue
            placed.append((y, x, reach))
            paste(fld, ts.template, y + 0.5, x + 0.5, float(rng.uniform(0, 2 * math.pi)), s)
            pl.append((t, y, x, s))
        images.append(quantize_with_noise(fld, rng))
        plants.append(pl)
    pairs = [(i, t) for i in range(n_images) for t in range(n_templates)] if all_pairs else []
    return BatchWorkload(images, templates, pairs, F_MEAN | F_VAR | F_GRAD, Tolerances(), 32, 64, plants)


@dataclass
class ServeEvent:
    t: float            # arrival time, seconds after the start of the stream
    kind: str           # "upload" or "screen"
    image: int          # upload: pool index; screen: index in the upload sequence (warm uploads first)
    template: int = -1  # screen: template index
    features: int = 0   # screen: feature bits (2 or 3 features)


@dataclass
class ServeWorkload:
    """Configuration 5: a Poisson stream of uploads and screens against resident tables."""
    pool: list[np.ndarray]          # distinct images the uploads draw their pixels from
    templates: list[TemplateSpec]
    warm: list[int]                 # pool indices uploaded before the stream starts
    events: list[ServeEvent]
    tol: Tolerances
    rate: float
    duration: float
    table_budget: int
    sum_bits: int = 32
    sq_bits: int = 64


def serve_workload(seed: int = BASE_SEED + 4, duration: float = 2.0, rate: float = 2000.0,
                   upload_frac: float = 0.1, n_pool: int = 16, n_templates: int = 64,
                   side_range=(256, 8192), r_range=(8, 96), max_scales: int = 16,
                   table_budget: int = 120 << 30, warm_fill: float = 0.85,
                   table_bytes_per_px: int = 24) -> ServeWorkload:
    """Poisson arrivals at `rate`/s for `duration` s; a fraction upload_frac are
    uploads of a square image with side log-uniform in side_range (pixels drawn
    from a pool of n_pool blob images, stratified over the log-side range), the rest screen a uniformly chosen
    uploaded image with a template of radius U{8..96}, 1..16 geometric scales in
    [0.5, min(2, 181/r)] and 2 (mean, variance) or 3 (plus contrast) features.
    Before the stream, warm uploads fill warm_fill of the table budget (table
    bytes estimated at table_bytes_per_px) so that eviction starts early."""
    rng = rng_for(seed)
    pool = []
    lo, hi = math.log(side_range[0]), math.log(side_range[1])
    for k in range(n_pool):   # stratified over the log-side range
        side = int(round(math.exp(lo + (k + rng.uniform()) / n_pool * (hi - lo))))
        pool.append(quantize_with_noise(blob_field(rng, side, side), rng))
    templates = []
    for _ in range(n_templates):
        r = int(rng.integers(r_range[0], r_range[1] + 1))
        ns = int(rng.integers(1, max_scales + 1))
        hi = min(2.0, 181.0 / r)
        scales = [1.0] if ns == 1 else geometric_scales(0.5, hi, ns)
        trng = rng_for(int(rng.integers(0, 2 ** 31)))
        tm = _template_from_source(trng, r, src_side=max(192, 4 * (2 * r + 1)))
        templates.append(TemplateSpec(tm, r, scales, radii_for(r, scales), t_min_for(r, scales)))
    warm, filled = [], 0
    while filled < warm_fill * table_budget:
        k = int(rng.integers(0, n_pool))
        warm.append(k)
        filled += pool[k].size * table_bytes_per_px
    events, t, n_up = [], 0.0, len(warm)
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        if rng.random() < upload_frac:
            events.append(ServeEvent(t, "upload", int(rng.integers(0, n_pool))))
            n_up += 1
        else:
            feats = F_MEAN | F_VAR | (F_GRAD if rng.random() < 0.5 else 0)
            events.append(ServeEvent(t, "screen", int(rng.integers(0, n_up)), int(rng.integers(0, n_templates)),
                                     feats))
    return ServeWorkload(pool, templates, warm, events, Tolerances(), rate, duration, table_budget)


def joint_areas(r: int, scales: list[float], n_areas: int):
    """Nested central areas for the joint membership screen: at scale s the
    star radii of areas j = 0..n_areas-1 are floor(R_s / lambda^j + 1/2)
    (area 0 is R_s itself), and area j's band of template central radii is
    [ceil(r / lambda^(j+1)), floor(r / lambda^j)], lambda the ratio of
    consecutive scales (area 0's band is [t_min, r]).  A single scale uses
    lambda = 2^(1/4)."""
    lam = scales[1] / scales[0] if len(scales) > 1 else 2 ** 0.25
    radii = radii_for(r, scales)
    area_radii = [[int(math.floor(R / lam ** j + 0.5)) for j in range(n_areas)] for R in radii]
    bands = [(int(math.ceil(r / lam ** (j + 1) - 1e-9)), int(math.floor(r / lam ** j + 1e-9)))
             for j in range(n_areas)]
    return area_radii, bands


@dataclass
class FrameSequence:
    frames: list[np.ndarray]          # uint8 H x W each
    template: np.ndarray              # uint8 (2r+1) x (2r+1)
    r: int
    radii: list[int]
    t_min: int
    features: int
    tol: Tolerances
    sum_bits: int
    sq_bits: int
    planted: list[tuple[int, int]]    # per frame: candidate (y*, x*) of the target
    s_true: list[float]               # per frame: the target's scale


def frame_sequence(seed: int, n_frames: int = 6, H: int = 256, W: int = 320, r: int = 16, n_scales: int = 4,
                   s_min: float = 0.6, s_max: float = 1.6, sum_bits: int = 32, sq_bits: int = 64) -> FrameSequence:
    """A short synthetic video for the tracking use of the screen (the paper
    screens every frame of a tracking sequence for the target, Sec. 6): one
    blob-field scene larger than the frame, seen through a window that pans a
    few pixels per frame, with the target (a template cut from its own field)
    pasted at a drifting position, rotating and changing scale from frame to
    frame; each frame has its own noise."""
    rng = rng_for(seed)
    pad = 64
    scene = blob_field(rng, H + 2 * pad, W + 2 * pad)
    tmpl = _template_from_source(rng_for(seed + 7919), r)
    scales = geometric_scales(s_min, s_max, n_scales)
    side = 2 * r + 1
    margin = int(math.ceil(s_max * side)) + 8
    ys = float(rng.uniform(margin, H - margin))
    xs = float(rng.uniform(margin, W - margin))
    vy, vx = (float(v) for v in rng.uniform(-3.0, 3.0, 2))
    theta = float(rng.uniform(0.0, 2.0 * math.pi))
    s_now = float(math.exp(rng.uniform(math.log(s_min), math.log(s_max))))
    frames, planted, s_list = [], [], []
    for k in range(n_frames):
        oy, ox = pad + (k * 2) % pad, pad - (k * 3) % pad
        fld = scene[oy:oy + H, ox:ox + W].copy()
        cy = int(min(max(ys + k * vy, margin), H - margin))
        cx = int(min(max(xs + k * vx, margin), W - margin))
        s_k = min(max(s_now * (1.0 + 0.02 * k), s_min), s_max)
        paste(fld, tmpl, cy + 0.5, cx + 0.5, theta + 0.05 * k, s_k)
        frames.append(quantize_with_noise(fld, rng))
        planted.append((cy, cx))
        s_list.append(s_k)
    return FrameSequence(frames=frames, template=tmpl, r=r, radii=radii_for(r, scales),
                         t_min=t_min_for(r, scales), features=F_MEAN | F_VAR | F_GRAD, tol=Tolerances(),
                         sum_bits=sum_bits, sq_bits=sq_bits, planted=planted, s_true=s_list)
