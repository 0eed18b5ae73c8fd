"""Prewitt gradient feature on the GPU against the oracle (oracle/prewitt.py):
moment tables bit-exact; masks of the interval screen with the Prewitt test,
alone and with the other features, over table widths and ragged sizes;
unsupported paths rejected."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import prewitt
import paper_1707_05647_gb300 as scr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PTOL = (Fraction(1, 10), Fraction(2))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    yield c
    scr.screen_shutdown(c)


def _tables(ctx, img, bits=(32, 64)):
    d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    tab = scr.build_tables(ctx, d, bits[0], bits[1])
    scr.build_moment_tables(ctx, tab, d)
    return tab


@pytest.mark.parametrize("H,W", [(1, 1), (7, 300), (300, 7), (257, 1031), (1200, 900),
                                 (32, 256), (33, 255), (31, 257), (64, 1024), (65, 2049), (96, 513),
                                 (65535, 40), (40, 65535)])
def test_moment_tables_bit_exact(ctx, H, W):
    img = synth.random_image(H * 7 + W, H, W)
    tab = _tables(ctx, img)
    Mx, My = prewitt.moment_tables(img)
    assert np.array_equal(scr.tables_copy_to_host(ctx, tab, 4).astype(np.int64), Mx)
    assert np.array_equal(scr.tables_copy_to_host(ctx, tab, 5).astype(np.int64), My)
    scr.tables_release(ctx, tab)


@pytest.mark.parametrize("features", [8, 9, 11, 15, 12])
@pytest.mark.parametrize("bits", [(32, 64), (64, 64)])
def test_prewitt_screen_matches_oracle(ctx, features, bits):
    wl = synth.small_planted(seed=6000 + features, H=256, r=16, n_scales=4)
    tab = _tables(ctx, wl.image, bits)
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, 15)
    p = scr.Params(wl.radii, features, wl.tol.mean_rel, wl.tol.std_rel, wl.tol.grad_rel, wl.tol.grad_abs,
                   PTOL[0], PTOL[1])
    H, W = wl.image.shape
    S = len(wl.radii)
    mask = torch.full((scr.mask_words(S, H, W),), -1, dtype=torch.int32, device="cuda")
    scr.screen_features(ctx, tab, tm, p, mask)
    torch.cuda.synchronize()
    got = mask.cpu().numpy().view(np.uint32).reshape(S, H, (W + 31) // 32)
    want = prewitt.screen_workload_prewitt(wl.image, wl.template, wl.r, wl.t_min, wl.radii, features, wl.tol, PTOL)
    assert want["count"] > 0
    assert np.array_equal(got, want["mask"])
    # the list through the usual compaction
    lst = torch.zeros(max(1, want["count"]), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    scr.compact_mask(ctx, mask, S, H, W, lst, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == want["count"]
    assert np.array_equal(lst.cpu().numpy().view(np.uint64)[:want["count"]], want["list"])
    scr.tables_release(ctx, tab)
    scr.template_release(ctx, tm)


def test_prewitt_ragged_and_planted(ctx):
    wl = synth.small_planted(seed=6100, H=256, r=12, n_scales=3)
    img = np.ascontiguousarray(wl.image[:203, :171])
    tab = _tables(ctx, img)
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, 15)
    p = scr.Params(wl.radii, 15, prewitt_rel=PTOL[0], prewitt_abs=PTOL[1])
    H, W = img.shape
    S = len(wl.radii)
    mask = torch.zeros(scr.mask_words(S, H, W), dtype=torch.int32, device="cuda")
    scr.screen_features(ctx, tab, tm, p, mask)
    torch.cuda.synchronize()
    got = mask.cpu().numpy().view(np.uint32).reshape(S, H, (W + 31) // 32)
    want = prewitt.screen_workload_prewitt(img, wl.template, wl.r, wl.t_min, wl.radii, 15, wl.tol, PTOL)
    assert np.array_equal(got, want["mask"])
    scr.tables_release(ctx, tab)
    scr.template_release(ctx, tm)


def test_prewitt_needs_moments_and_template_and_is_rejected_elsewhere(ctx):
    wl = synth.small_planted(seed=6200, H=128, r=10, n_scales=2)
    d = torch.from_numpy(wl.image).cuda()
    tab = scr.build_tables(ctx, d, 32, 64)
    tm7 = scr.template_features(ctx, wl.template, wl.r, wl.t_min, 7)
    tm15 = scr.template_features(ctx, wl.template, wl.r, wl.t_min, 15)
    p = scr.Params(wl.radii, 9)
    H, W = wl.image.shape
    mask = torch.zeros(scr.mask_words(len(wl.radii), H, W), dtype=torch.int32, device="cuda")
    for tm in (tm15, tm7):   # no moment tables yet; then a template without Prewitt moments
        with pytest.raises(scr.ScreenError) as e:
            scr.screen_features(ctx, tab, tm, p, mask)
        assert e.value.code == scr.SCR_EINVAL
        scr.build_moment_tables(ctx, tab, d)
    scr.screen_features(ctx, tab, tm15, p, mask)                 # now it runs
    with pytest.raises(scr.ScreenError) as e:
        scr.screen_joint(ctx, tab, tm15, p, [[R] for R in wl.radii], [(wl.t_min, wl.r)], (4, 2, 4), mask)
    assert e.value.code == scr.SCR_EUNSUPPORTED
    with pytest.raises(scr.ScreenError) as e:
        scr.screen_batch_create(ctx, [tab], [tm15], [p], [(0, 0)], torch.zeros(1, dtype=torch.int64, device="cuda"),
                                torch.zeros(16, dtype=torch.int64, device="cuda"),
                                torch.zeros(2, dtype=torch.int64, device="cuda"))
    assert e.value.code == scr.SCR_EUNSUPPORTED
    scr.tables_release(ctx, tab)
