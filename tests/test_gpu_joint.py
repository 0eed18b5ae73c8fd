"""Joint-vector membership screen on the GPU (screen_joint) against the oracle
(oracle/joint.py): every mask word, bit-exact, over feature combinations, one
to three nested central areas, quantisation factors, table widths, ragged
sizes, and sampled rows of the 4096^2 workload; invalid arguments rejected."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import joint
import paper_1707_05647_gb300 as scr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    yield c
    scr.screen_shutdown(c)


def _gpu_mask(ctx, img, tmpl, r, t_min, radii, area_radii, bands, features, q, bits=(32, 64)):
    H, W = img.shape
    tab = scr.build_tables(ctx, torch.from_numpy(np.ascontiguousarray(img)).cuda(), bits[0], bits[1])
    tm = scr.template_features(ctx, tmpl, r, t_min, 7)
    p = scr.Params(radii, features)
    mask = torch.full((scr.mask_words(len(radii), H, W),), -1, dtype=torch.int32, device="cuda")
    scr.screen_joint(ctx, tab, tm, p, area_radii, bands, q, mask)
    torch.cuda.synchronize()
    out = mask.cpu().numpy().view(np.uint32).reshape(len(radii), H, (W + 31) // 32)
    scr.tables_release(ctx, tab)
    scr.template_release(ctx, tm)
    return out


def _oracle_mask(img, tmpl, r, t_min, radii, area_radii, bands, features, q, rows=None):
    sums = oracle.template_sums(tmpl, r, t_min)
    return joint.screen_joint(oracle.Tables(img), sums, radii, area_radii, bands, features, q, rows=rows)


CASES = [  # (features, n_areas, q)
    (7, 3, (4, 2, 4)), (7, 1, (6, 3, 6)), (3, 2, (Fraction(5, 2), Fraction(3, 2), 1)), (1, 1, (3, 1, 1)),
    (2, 3, (1, Fraction(7, 4), 1)), (4, 2, (1, 1, Fraction(9, 2))), (5, 3, (5, 1, 7)), (6, 1, (1, 2, 5)),
]


@pytest.mark.parametrize("features,n_areas,qs", CASES)
def test_joint_matches_oracle(ctx, features, n_areas, qs):
    wl = synth.small_planted(seed=4000 + features * 10 + n_areas, H=256, r=16, n_scales=4)
    area_radii, bands = synth.joint_areas(wl.r, wl.scales, n_areas)
    t_min = max(2, min(b[0] for b in bands))
    q = tuple(Fraction(v) for v in qs)
    want, _, cnt = _oracle_mask(wl.image, wl.template, wl.r, t_min, wl.radii, area_radii, bands, features, q)
    got = _gpu_mask(ctx, wl.image, wl.template, wl.r, t_min, wl.radii, area_radii, bands, features, q)
    assert cnt > 0
    assert np.array_equal(got, want)


@pytest.mark.parametrize("bits", [(32, 32), (64, 64)])
@pytest.mark.parametrize("H,W", [(161, 97), (200, 300), (97, 520)])
def test_joint_ragged_sizes_and_table_widths(ctx, bits, H, W):
    """Widths with a partial last warp of 8 mask words (97: 4 words; 300: 10;
    520: 17), heights off the 32-row bands."""
    rng = np.random.default_rng(77)
    wl = synth.small_planted(seed=4100, H=max(256, H, W), r=12, n_scales=3)
    img = np.ascontiguousarray(wl.image[:H, :W])
    area_radii, bands = synth.joint_areas(wl.r, wl.scales, 3)
    t_min = max(2, min(b[0] for b in bands))
    q = (Fraction(9, 2), Fraction(5, 2), Fraction(11, 2))
    want, _, _ = _oracle_mask(img, wl.template, wl.r, t_min, wl.radii, area_radii, bands, 7, q)
    got = _gpu_mask(ctx, img, wl.template, wl.r, t_min, wl.radii, area_radii, bands, 7, q, bits=bits)
    assert np.array_equal(got, want)
    del rng


def test_joint_sampled_rows_of_the_4096_workload(ctx):
    wl = synth.config2()
    area_radii, bands = synth.joint_areas(wl.r, wl.scales, 3)
    t_min = max(2, min(b[0] for b in bands))
    q = (Fraction(4), Fraction(2), Fraction(4))
    got = _gpu_mask(ctx, wl.image, wl.template, wl.r, t_min, wl.radii, area_radii, bands, 7, q, bits=(32, 64))
    rows = sorted(set([100, 101, 777, 2048, 2049, 3900, wl.planted[0]]))
    want, _, _ = _oracle_mask(wl.image, wl.template, wl.r, t_min, wl.radii, area_radii, bands, 7, q, rows=rows)
    for y in rows:
        assert np.array_equal(got[:, y], want[:, y]), y
    # the planted match survives at a covering scale
    py, px = wl.planted
    assert any((got[s, py, px >> 5] >> (px & 31)) & 1 for s in range(len(wl.radii)))


def test_joint_rejects_bad_arguments(ctx):
    wl = synth.small_planted(seed=4200, H=128, r=10, n_scales=2)
    tab = scr.build_tables(ctx, torch.from_numpy(wl.image).cuda(), 32, 64)
    tm = scr.template_features(ctx, wl.template, wl.r, 6, 7)
    p = scr.Params(wl.radii, 7)
    H, W = wl.image.shape
    mask = torch.zeros(scr.mask_words(len(wl.radii), H, W), dtype=torch.int32, device="cuda")
    good_ar, good_b = [[R] for R in wl.radii], [(6, 10)]
    bad = [
        (good_ar, [(5, 10)], (4, 2, 4)),                        # band below the template's t_min
        (good_ar, [(6, 11)], (4, 2, 4)),                        # band above r
        ([[R + 1] for R in wl.radii], good_b, (4, 2, 4)),       # area larger than the scale's star
        ([[1] for R in wl.radii], good_b, (4, 2, 4)),           # area radius below 2
        (good_ar, good_b, (Fraction(1, 17), 2, 4)),             # q denominator above 16
        (good_ar, good_b, (0, 2, 4)),                           # q = 0
        (good_ar, good_b, (65537, 2, 4)),                       # q numerator above 2^16
    ]
    for ar, bands, q in bad:
        with pytest.raises(scr.ScreenError) as e:
            scr.screen_joint(ctx, tab, tm, p, ar, bands, q, mask)
        assert e.value.code == scr.SCR_EINVAL
    with pytest.raises(scr.ScreenError) as e:                   # no feature enabled
        scr.screen_joint(ctx, tab, tm, scr.Params(wl.radii, 0), good_ar, good_b, (4, 2, 4), mask)
    assert e.value.code == scr.SCR_EINVAL
    scr.tables_release(ctx, tab)
    scr.template_release(ctx, tm)
