"""Packed-plane pre-filter (screen_set_filter) against the oracle.

The packed planes are compared element by element with their definition on
the oracle's exact tables (bits kS..kS+15 of the sum table in the low half,
bits kQ..kQ+15 of the squares' table in the high half).  Masks and lists of
screens on tables that carry packed planes are compared word by word and key
by key with the oracle, which has no filter: the filter may only skip exact
reads of candidates that fail (a variance certainly below the interval), so
every result must be unchanged.  The plan (screen_filter_plan) is checked
too, so the cases that must exercise the filter do.  Integer results,
tolerance 0."""
import dataclasses
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
import paper_1707_05647_gb300 as scr
from paper_1707_05647_gb300 import ScreenError
from gpu_helpers import params_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    yield c
    scr.screen_shutdown(c)


def _packed(a, b, kS, kQ):
    m = np.uint64(0xFFFF)
    return ((a >> np.uint64(kS)) & m) | (((b >> np.uint64(kQ)) & m) << np.uint64(16))


@pytest.mark.parametrize("H,W", [(1, 1), (2, 3), (33, 191), (32, 192), (65, 193), (40, 383), (96, 959),
                                 (33, 960), (100, 961), (300, 1000)])
@pytest.mark.parametrize("bits", [(32, 32), (32, 64), (64, 64)])
def test_packed_planes_bit_exact(ctx, H, W, bits):
    img = synth.random_image(H * 53 + W, H, W, "uniform")
    windows = [(0, 0), (9, 16)] if (H + W) % 2 else [(14, 5), (3, 11)]
    scr.screen_set_filter(ctx, windows)
    try:
        tb = scr.build_tables(ctx, torch.from_numpy(img).cuda(), bits[0], bits[1])
    finally:
        scr.screen_set_filter(ctx, [])
    try:
        L1, L2 = oracle.upright_tables(img)
        T1, T2 = oracle.cone_tables(img)
        for w, (kS, kQ) in enumerate(windows):
            for k, (a, b) in enumerate(((L1, L2), (T1, T2))):
                got = scr.tables_copy_to_host(ctx, tb, 6 + 2 * w + k)
                want = _packed(a, b, kS, kQ)
                assert got.shape == want.shape
                if not np.array_equal(got, want):
                    bad = np.argwhere(got != want)
                    raise AssertionError(f"window {w} plane {k}: {len(bad)} entries differ, first {bad[:5].tolist()}")
        # the exact tables are unchanged by the extra planes
        for which, ref in enumerate((L1, L2, T1, T2)):
            want = ref if bits[which % 2] == 64 else ref & np.uint64(0xFFFFFFFF)
            assert np.array_equal(scr.tables_copy_to_host(ctx, tb, which), want), which
    finally:
        scr.tables_release(ctx, tb)


def _screen(ctx, wl, windows):
    """Filtered screen of wl through screen_positions; (mask, list, count, plan)."""
    H, W = wl.image.shape
    scr.screen_set_filter(ctx, windows)
    try:
        tb = scr.build_tables(ctx, torch.from_numpy(np.ascontiguousarray(wl.image)).cuda(), wl.sum_bits, wl.sq_bits)
    finally:
        scr.screen_set_filter(ctx, [])
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    p = params_of(wl)
    try:
        plan = scr.screen_filter_plan(tb, tm, p)
        mask = torch.full((scr.mask_words(len(wl.radii), H, W),), -1, dtype=torch.int32, device="cuda")
        cap = len(wl.radii) * H * W
        lst = torch.zeros(cap, dtype=torch.int64, device="cuda")
        n, over = scr.screen_positions(ctx, tb, tm, p, mask, lst)
        assert not over
        got = mask.cpu().numpy().view(np.uint32).reshape(len(wl.radii), H, (W + 31) // 32)
        return got, lst[:n].cpu().numpy().view(np.uint64), n, plan
    finally:
        scr.tables_release(ctx, tb)
        scr.template_release(ctx, tm)


def _suggested(ctx, wl, max_windows=2):
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    try:
        return scr.screen_filter_windows(tm, params_of(wl), max_windows)
    finally:
        scr.template_release(ctx, tm)


def _check_equal(got, lst, n, ref):
    if not np.array_equal(got, ref["mask"]):
        bad = np.argwhere(got != ref["mask"])
        raise AssertionError(f"{len(bad)} mask words differ, first {bad[:5].tolist()}")
    assert n == ref["count"]
    assert np.array_equal(lst, ref["list"])


FEATURES = [scr.F_MEAN | scr.F_VAR | scr.F_GRAD, scr.F_MEAN | scr.F_VAR, scr.F_MEAN, scr.F_VAR,
            scr.F_MEAN | scr.F_GRAD, scr.F_GRAD]


@pytest.mark.parametrize("seed", [11, 12])
@pytest.mark.parametrize("bits", [(32, 32), (32, 64), (64, 64)])
@pytest.mark.parametrize("features", FEATURES)
def test_filtered_screen_equals_oracle(ctx, seed, bits, features):
    wl = synth.small_planted(seed, H=384, r=20, n_scales=4, sum_bits=bits[0], sq_bits=bits[1])
    wl = dataclasses.replace(wl, features=features)
    ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
    windows = _suggested(ctx, wl)
    if features & scr.F_VAR:
        assert windows, "the variance test is on: a window is suggested"
    else:
        assert windows == []
        windows = [(4, 12), (7, 15)]   # planes present, but no scale may use them
    got, lst, n, plan = _screen(ctx, wl, windows)
    if features & scr.F_VAR:
        assert any(w >= 0 for w in plan), plan
    else:
        assert all(w == -1 for w in plan), plan
    _check_equal(got, lst, n, ref)


# windows chosen to stress the filter's edges: the narrowest shifts (most
# scales have no usable window), one window only, and the widest shifts
# (wide boxes, almost nothing rejected)
@pytest.mark.parametrize("windows", [[(0, 0)], [(2, 9), (4, 12)], [(6, 14)], [(14, 16)], [(5, 13), (8, 16)]])
def test_filtered_screen_any_windows(ctx, windows):
    wl = synth.small_planted(21, H=400, r=24, n_scales=5, sum_bits=32, sq_bits=64)
    ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
    got, lst, n, plan = _screen(ctx, wl, windows)
    assert all(-1 <= w < len(windows) for w in plan)
    _check_equal(got, lst, n, ref)


# images whose star sums sit at the ends of a window's range or beyond it:
# saturated (S = 255 A, above the mean interval), empty (S = 0, the low half
# wraps to small negative sums), uniform noise (high variance) and a half
# saturated, half empty image (sums across the whole range); templates are
# taken from a planted workload so the intervals are realistic, and the
# narrowest windows make the range conditions bind
@pytest.mark.parametrize("kind", ["max", "zero", "uniform", "split"])
@pytest.mark.parametrize("windows", [None, [(0, 0), (4, 12)], [(9, 16)]])
def test_filtered_screen_extreme_images(ctx, kind, windows):
    wl = synth.small_planted(41, H=288, r=20, n_scales=4, sum_bits=32, sq_bits=32)
    if kind == "split":
        img = synth.random_image(7, 288, 288, "max")
        img[:, 144:] = 0
    else:
        img = synth.random_image(7, 288, 288, kind)
    wl = dataclasses.replace(wl, image=img)
    ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
    if windows is None:
        windows = _suggested(ctx, wl)
    got, lst, n, plan = _screen(ctx, wl, windows)
    assert all(-1 <= w < len(windows) for w in plan)
    _check_equal(got, lst, n, ref)


# wide intervals (tolerances of 90%) so that many candidates pass: the filter
# must keep every one of them
def test_filtered_screen_keeps_everything_that_passes(ctx):
    wl = synth.small_planted(43, H=256, r=16, n_scales=3, sum_bits=32, sq_bits=64)
    tol = dataclasses.replace(wl.tol, mean_rel=Fraction(9, 10), std_rel=Fraction(9, 10))
    wl = dataclasses.replace(wl, tol=tol, features=scr.F_MEAN | scr.F_VAR)
    ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
    windows = _suggested(ctx, wl)
    got, lst, n, plan = _screen(ctx, wl, windows)
    _check_equal(got, lst, n, ref)
    assert n == ref["count"] > 0


@pytest.mark.parametrize("H,W", [(40, 65535), (65535, 40)])
def test_filtered_screen_maximum_dimension(ctx, H, W):
    """The largest side the boundary accepts (65535) on a thin image, with
    packed planes: keys with y or x near 2^16, the last partial warp span of
    a row, and the packed planes' last columns."""
    img = synth.random_image(H ^ W, H, W, "uniform")
    r = 10
    tm = img[:2 * r + 1, :2 * r + 1].copy()
    wl = synth.Workload("max side", img, tm, r, [6, 9, 13, 17], 7, scr.F_MEAN | scr.F_VAR | scr.F_GRAD,
                        synth.Tolerances(Fraction(1, 50), Fraction(1, 20), Fraction(1, 5), Fraction(4)),
                        32, 64, (0, 0), 1.0, 0.0)
    ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
    windows = _suggested(ctx, wl)
    got, lst, n, plan = _screen(ctx, wl, windows)
    assert any(w >= 0 for w in plan), (windows, plan)
    assert ref["count"] > 0
    _check_equal(got, lst, n, ref)


@pytest.mark.parametrize("seed", [93, 95])
@pytest.mark.parametrize("kind", ["plain", "split"])
@pytest.mark.parametrize("windows", [None, [(9, 16)]])
def test_filtered_screen_largest_radius(ctx, seed, kind, windows):
    """Stars up to radius 181, the largest the boundary accepts (pooled area
    A = 131058, where the filter's constants span their widest range), on a
    400 x 700 image whose 256-candidate warp spans are fully valid at every
    scale, so the batched pre-filter path runs.  The template samples the
    image centre at stride 9, so the large stars' means and variances fall
    inside its intervals: some candidates pass at every scale.  The split
    image inverts the right part, which moves sums across the range."""
    H, W = 400, 700
    img = synth.random_image(seed, H, W, "blobs")
    cy, cx = H // 2, W // 2
    tm = np.ascontiguousarray(img[cy - 180:cy + 181:9, cx - 180:cx + 181:9])
    if kind == "split":
        img = img.copy()
        img[:, cx + 60:] = 255 - img[:, cx + 60:]
    bits = (32, 32) if seed % 2 else (64, 64)
    wl = synth.Workload("largest radius", img, tm, 20, [120, 150, 181], 10,
                        scr.F_MEAN | scr.F_VAR | scr.F_GRAD,
                        synth.Tolerances(Fraction(1, 20), Fraction(1, 10), Fraction(1, 2), Fraction(8)),
                        bits[0], bits[1], (cy, cx), 9.0, 0.0)
    ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
    if windows is None:
        windows = _suggested(ctx, wl)
    got, lst, n, plan = _screen(ctx, wl, windows)
    assert plan[-1] >= 0, (windows, plan)                   # R = 181 pre-filters
    per_scale = [int(((ref["list"] >> np.uint64(48)) == s).sum()) for s in range(3)]
    assert min(per_scale) > 0, per_scale
    _check_equal(got, lst, n, ref)


def _config3_crop(side=1024):
    """The 8192 x 8192 16-scale image cropped around its planted match."""
    wl = synth.config3()
    y, x = wl.planted
    y0 = min(max(y - side // 2, 0), wl.image.shape[0] - side)
    x0 = min(max(x - side // 2, 0), wl.image.shape[1] - side)
    img = np.ascontiguousarray(wl.image[y0:y0 + side, x0:x0 + side])
    return dataclasses.replace(wl, image=img, planted=(y - y0, x - x0))


def test_filtered_screen_config3_crop(ctx):
    wl = _config3_crop()
    ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
    windows = _suggested(ctx, wl)
    got, lst, n, plan = _screen(ctx, wl, windows)
    assert all(w >= 0 for w in plan), (windows, plan)   # every scale filtered on this workload
    _check_equal(got, lst, n, ref)
    y, x = wl.planted
    assert any((got[s, y, x >> 5] >> (x & 31)) & 1 for s in range(len(wl.radii)))


def test_filtered_full_size_config3(ctx):
    """The 8192 x 8192 headline workload in the bench's launch sequence with the
    suggested windows: every mask word and key against the oracle."""
    wl = synth.config3()
    H, W = wl.image.shape
    S = len(wl.radii)
    windows = _suggested(ctx, wl)
    assert len(windows) == 2
    stream = torch.cuda.current_stream()
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    p = params_of(wl)
    scr.screen_set_filter(ctx, windows)
    try:
        tb = scr.build_tables(ctx, torch.from_numpy(wl.image).cuda(), wl.sum_bits, wl.sq_bits, stream)
    finally:
        scr.screen_set_filter(ctx, [])
    try:
        assert all(w >= 0 for w in scr.screen_filter_plan(tb, tm, p))
        mask = torch.empty(scr.mask_words(S, H, W), dtype=torch.int32, device="cuda")
        cap = 1 << 22
        lst = torch.empty(cap, dtype=torch.int64, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        scr.screen_features(ctx, tb, tm, p, mask, stream)
        scr.compact_mask(ctx, mask, S, H, W, lst, count, stream)
        torch.cuda.synchronize()
        ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
        got = mask.cpu().numpy().view(np.uint32).reshape(ref["mask"].shape)
        n = int(count.item())
        _check_equal(got, lst[:n].cpu().numpy().view(np.uint64), n, ref)
    finally:
        scr.tables_release(ctx, tb)
        scr.template_release(ctx, tm)


def test_filtered_screen_host_and_frames(ctx):
    fs = synth.frame_sequence(5003, n_frames=4)
    want = [oracle.screen_workload(f, fs.template, fs.r, fs.t_min, fs.radii, fs.features, fs.tol)["list"]
            for f in fs.frames]
    p = scr.Params(fs.radii, fs.features, fs.tol.mean_rel, fs.tol.std_rel, fs.tol.grad_rel, fs.tol.grad_abs)
    tm = scr.template_features(ctx, fs.template, fs.r, fs.t_min, fs.features)
    windows = scr.screen_filter_windows(tm, p)
    assert windows
    H, W = fs.frames[0].shape
    cap = max(len(w) for w in want) + 16
    scr.screen_set_filter(ctx, windows)
    try:
        for k, im in enumerate(fs.frames):
            lst = np.zeros(cap, np.uint64)
            n, over = scr.screen_host(ctx, im, fs.sum_bits, fs.sq_bits, tm, p, lst)
            assert not over and np.array_equal(lst[:n], want[k]), k
        f = scr.frames_create(ctx, H, W, fs.sum_bits, fs.sq_bits, tm, p, cap, 2)
    finally:
        scr.screen_set_filter(ctx, [])
    try:
        lists = [torch.zeros(cap, dtype=torch.int64).pin_memory().numpy().view(np.uint64) for _ in fs.frames]
        tickets = []
        for k, im in enumerate(fs.frames):
            if len(tickets) == 2:
                kk, t = tickets.pop(0)
                n, over = scr.frames_wait(f, t)
                assert not over and np.array_equal(lists[kk][:n], want[kk]), kk
            tickets.append((k, scr.frames_submit(f, im, lists[k])))
        for kk, t in tickets:
            n, over = scr.frames_wait(f, t)
            assert not over and np.array_equal(lists[kk][:n], want[kk]), kk
    finally:
        scr.frames_destroy(f)
        scr.template_release(ctx, tm)


def test_prewitt_reads_exact_corners_only(ctx):
    wl = synth.small_planted(31, H=256, r=16, n_scales=3)
    feats = wl.features | scr.F_PREWITT
    img = torch.from_numpy(wl.image).cuda()
    scr.screen_set_filter(ctx, [(4, 12)])
    try:
        tb = scr.build_tables(ctx, img, wl.sum_bits, wl.sq_bits)
    finally:
        scr.screen_set_filter(ctx, [])
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, feats)
    try:
        scr.build_moment_tables(ctx, tb, img)
        p = scr.Params(wl.radii, feats, wl.tol.mean_rel, wl.tol.std_rel, wl.tol.grad_rel, wl.tol.grad_abs)
        assert scr.screen_filter_plan(tb, tm, p) == [-1] * len(wl.radii)
    finally:
        scr.tables_release(ctx, tb)
        scr.template_release(ctx, tm)


@pytest.mark.parametrize("windows", [[(0, 0)] * 3, [(15, 0)], [(0, 17)], [(-1, 4)]])
def test_set_filter_rejects_bad_windows(ctx, windows):
    with pytest.raises(ScreenError) as e:
        scr.screen_set_filter(ctx, windows)
    assert e.value.code == scr.SCR_EINVAL
