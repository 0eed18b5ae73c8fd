"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit for bit.

Tables are compared modulo 2^bits element by element; masks word by word;
lists key by key.  Everything is integer, so the tolerance is zero."""
import numpy as np
import pytest

import oracle
import synth
import paper_1707_05647_gb300 as scr
from gpu_helpers import gpu_run, oracle_run, params_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    yield c
    scr.screen_shutdown(c)


def _tables_equal(ctx, tb, img, bits):
    L1, L2 = oracle.upright_tables(img)
    T1, T2 = oracle.cone_tables(img)
    for which, ref in enumerate((L1, L2, T1, T2)):
        b = bits[which % 2]
        got = scr.tables_copy_to_host(ctx, tb, which)
        want = ref if b == 64 else (ref & np.uint64(0xFFFFFFFF))
        if not np.array_equal(got, want):
            bad = np.argwhere(got != want)
            raise AssertionError(f"table {which} ({b} bits) differs at {len(bad)} entries, first {bad[:5].tolist()}")


SIZES = [(1, 1), (1, 7), (9, 1), (2, 3), (31, 33), (33, 31), (64, 80), (100, 961), (97, 1921),
         (70, 1920), (65, 2881), (300, 1000), (513, 513), (40, 2000)]


@pytest.mark.parametrize("H,W", SIZES)
@pytest.mark.parametrize("bits", [(32, 32), (32, 64), (64, 32), (64, 64)])
def test_tables_bit_exact(ctx, H, W, bits):
    img = synth.random_image(H * 131 + W, H, W, "uniform")
    dimg = torch.from_numpy(img).cuda()
    tb = scr.build_tables(ctx, dimg, bits[0], bits[1])
    try:
        _tables_equal(ctx, tb, img, bits)
    finally:
        scr.tables_release(ctx, tb)


# widths around the table writer's 192-column warp tiles and the band
# reduction's 960-column tiles (one column short, exact, one past), heights
# around the 32-row bands
EDGE_SIZES = [(33, 191), (32, 192), (65, 193), (40, 383), (31, 384), (35, 385), (96, 959), (33, 960),
              (64, 1152), (1, 192), (32, 1)]


@pytest.mark.parametrize("H,W", EDGE_SIZES)
@pytest.mark.parametrize("bits", [(32, 64), (64, 64)])
@pytest.mark.parametrize("kind", ["uniform", "max"])
def test_tables_tile_edges(ctx, H, W, bits, kind):
    img = synth.random_image(H * 7 + W, H, W, kind)
    tb = scr.build_tables(ctx, torch.from_numpy(img).cuda(), bits[0], bits[1])
    try:
        _tables_equal(ctx, tb, img, bits)
    finally:
        scr.tables_release(ctx, tb)


@pytest.mark.parametrize("kind", ["max", "zero", "blobs"])
def test_tables_special_images(ctx, kind):
    H, W = 257, 1100
    img = synth.random_image(3, H, W, kind)
    tb = scr.build_tables(ctx, torch.from_numpy(img).cuda(), 32, 64)
    try:
        _tables_equal(ctx, tb, img, (32, 64))
    finally:
        scr.tables_release(ctx, tb)


@pytest.mark.parametrize("W,pitch,off", [(37, 37, 0), (37, 40, 0), (100, 128, 3), (961, 1000, 5)])
def test_tables_pitched_and_unaligned_image(ctx, W, pitch, off):
    H = 45
    img = synth.random_image(W + pitch, H, W, "uniform")
    buf = torch.zeros(H * pitch + off + 8, dtype=torch.uint8, device="cuda")
    view = buf[off:off + H * pitch].view(H, pitch)
    view[:, :W].copy_(torch.from_numpy(img))
    tb = scr.build_tables(ctx, view[:, :W], 64, 64, H=H, W=W, pitch=pitch)
    try:
        _tables_equal(ctx, tb, img, (64, 64))
    finally:
        scr.tables_release(ctx, tb)


def test_template_sums_and_bounds(ctx):
    wl = synth.small_planted(2003)
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    ref = oracle.template_sums(wl.template, wl.r, wl.t_min)
    for (t, S, Q, Si) in ref:
        assert scr.template_sums(tm, t) == (S, Q, Si), t
    hulls = oracle.template_hulls(ref, wl.features)
    want = np.array([oracle.scale_bounds(hulls, R, wl.tol, wl.features).as_row() for R in wl.radii])
    got = scr.screen_bounds(tm, params_of(wl))
    assert np.array_equal(got, want)
    scr.template_release(ctx, tm)


def _compare(g, o):
    assert np.array_equal(g["bounds"], o["bounds"])
    if not np.array_equal(g["mask"], o["mask"]):
        bad = np.argwhere(g["mask"] != o["mask"])
        raise AssertionError(f"mask differs in {len(bad)} words, first {bad[:5].tolist()}")
    assert g["count"] == o["count"]
    assert np.array_equal(g["list"], o["list"][:len(g["list"])])


@pytest.mark.parametrize("seed", [1000, 1001, 1002, 1003])
def test_config1_mask_and_list_bit_exact(ctx, seed):
    wl = synth.config1(seed)
    g, o = gpu_run(ctx, wl), oracle_run(wl)
    _compare(g, o)
    y, x = wl.planted
    assert (g["mask"][0, y, x >> 5] >> (x & 31)) & 1
    scr.tables_release(ctx, g["tables"])


@pytest.mark.parametrize("seed", [2000, 2001, 2005, 2011])
@pytest.mark.parametrize("bits", [(32, 32), (64, 64), (32, 64)])
def test_reduced_planted_bit_exact(ctx, seed, bits):
    wl = synth.small_planted(seed, sum_bits=bits[0], sq_bits=bits[1])
    g, o = gpu_run(ctx, wl), oracle_run(wl)
    _compare(g, o)
    scr.tables_release(ctx, g["tables"])


@pytest.mark.parametrize("features", [0, 1, 2, 3, 4, 5, 6, 7])
def test_feature_combinations(ctx, features):
    wl = synth.small_planted(2002, H=200, r=12, n_scales=3)
    wl.features = features if features & 4 else features
    wl.tol = synth.Tolerances(synth.Fraction(1, 5), synth.Fraction(1, 3), synth.Fraction(1, 3), synth.Fraction(6))
    g, o = gpu_run(ctx, wl), oracle_run(wl)
    _compare(g, o)
    scr.tables_release(ctx, g["tables"])


@pytest.mark.parametrize("H,W", [(100, 33), (37, 250), (64, 64), (161, 97)])
def test_ragged_sizes_and_large_radii(ctx, H, W):
    rng = np.random.default_rng(H * W)
    img = synth.random_image(H + W, H, W, "blobs")
    r = 10
    tm = img[:2 * r + 1, :2 * r + 1].copy() if min(H, W) > 2 * r else synth.random_image(1, 2 * r + 1, 2 * r + 1, "blobs")
    radii = sorted(set(int(v) for v in rng.integers(2, 60, 5)))
    wl = synth.Workload("ragged", img, tm, r, radii, 5, 7,
                        synth.Tolerances(synth.Fraction(1, 3), synth.Fraction(1, 2), synth.Fraction(1, 2),
                                         synth.Fraction(10)), 32, 64, (0, 0), 1.0, 0.0)
    g, o = gpu_run(ctx, wl), oracle_run(wl)
    _compare(g, o)
    scr.tables_release(ctx, g["tables"])


@pytest.mark.parametrize("H,W", [(40, 65535), (65535, 40)])
def test_maximum_dimension(ctx, H, W):
    """The largest side the boundary accepts (65535), on a thin image: 2048
    bands or 342 writer tiles, keys with y or x near 2^16; tables and the
    screen against the oracle."""
    img = synth.random_image(H ^ W, H, W, "uniform")
    tb = scr.build_tables(ctx, torch.from_numpy(img).cuda(), 32, 64)
    try:
        _tables_equal(ctx, tb, img, (32, 64))
    finally:
        scr.tables_release(ctx, tb)
    r = 10
    tm = img[:2 * r + 1, :2 * r + 1].copy()
    wl = synth.Workload("max side", img, tm, r, [6, 9, 13, 17], 7, 7,
                        synth.Tolerances(synth.Fraction(1, 50), synth.Fraction(1, 20), synth.Fraction(1, 5),
                                         synth.Fraction(4)), 32, 64, (0, 0), 1.0, 0.0)
    g, o = gpu_run(ctx, wl), oracle_run(wl)
    assert o["count"] > 0
    _compare(g, o)
    scr.tables_release(ctx, g["tables"])


def test_list_overflow_reports_true_count(ctx):
    wl = synth.config1(1000)
    wl.tol = synth.Tolerances(synth.Fraction(1, 2), synth.Fraction(9, 10))
    o = oracle_run(wl)
    assert o["count"] > 100
    g = gpu_run(ctx, wl, cap=50)
    assert g["overflow"] and g["count"] == o["count"]
    assert np.array_equal(g["list"], o["list"][:50])
    assert np.array_equal(g["mask"], o["mask"])
    scr.tables_release(ctx, g["tables"])


def test_screen_host_matches_oracle(ctx):
    wl = synth.small_planted(2001)
    o = oracle_run(wl)
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    lst = np.zeros(o["count"] + 10, np.uint64)
    n, over = scr.screen_host(ctx, wl.image, wl.sum_bits, wl.sq_bits, tm, params_of(wl), lst)
    assert not over and n == o["count"]
    assert np.array_equal(lst[:n], o["list"])


@pytest.mark.parametrize("pinned_list", [False, True])
@pytest.mark.parametrize("short", [False, True])
def test_screen_host_list_buffers(ctx, pinned_list, short):
    """A pinned list buffer takes the one-synchronisation path (keys written by
    the device into host memory); a pageable one the copy-back path.  Both give
    the oracle's list, and a short buffer its first keys with the exact count."""
    wl = synth.small_planted(2003)
    o = oracle_run(wl)
    assert o["count"] > 4
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    cap = o["count"] - 3 if short else o["count"] + 10
    if pinned_list:
        lst = torch.full((cap,), -1, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
    else:
        lst = np.full(cap, np.uint64(2**64 - 1), np.uint64)
    img = torch.from_numpy(wl.image).pin_memory().numpy() if pinned_list else wl.image
    n, over = scr.screen_host(ctx, img, wl.sum_bits, wl.sq_bits, tm, params_of(wl), lst)
    assert n == o["count"] and over == short
    k = min(n, cap)
    assert np.array_equal(lst[:k], o["list"][:k])
    assert np.all(lst[k:] == np.uint64(2**64 - 1))


def test_budget_is_enforced(ctx):
    small = scr.screen_init(0, 1 << 20)
    try:
        img = torch.zeros((512, 512), dtype=torch.uint8, device="cuda")
        with pytest.raises(scr.ScreenError) as e:
            scr.build_tables(small, img, 64, 64)
        assert e.value.code == scr.SCR_EBUDGET
        assert scr.screen_stats(small)["bytes_in_use"] == 0
    finally:
        scr.screen_shutdown(small)


def test_bad_arguments_rejected(ctx):
    img = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(scr.ScreenError) as e:
        scr.build_tables(ctx, img, 16, 64)
    assert e.value.code == scr.SCR_EINVAL
    tm = scr.template_features(ctx, np.zeros((9, 9), np.uint8), 4, 2, 7)
    tb = scr.build_tables(ctx, img, 32, 32)
    mask = torch.zeros(16, dtype=torch.int32, device="cuda")
    for radii in ([1], [182], list(range(2, 40))):
        with pytest.raises(scr.ScreenError) as e:
            scr.screen_features(ctx, tb, tm, scr.Params(radii, 7), mask)
        assert e.value.code == scr.SCR_EINVAL
    with pytest.raises(scr.ScreenError):   # mask too small for 2 scales
        scr.screen_features(ctx, tb, tm, scr.Params([2, 3], 7), mask[:8])
    scr.tables_release(ctx, tb)
    scr.template_release(ctx, tm)
