"""Pins of the oracle's bounds, mask and list: the exact rational definition of
the screen (Sec. 5, Algorithm 1 with interval tests), evaluated from brute-force
pixel sums, and the planted-match invariant ("never missing the best match",
abstract and Sec. 6).  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import brute
from oracle.bounds import Hulls, scale_bounds, star_geometry, template_features


def _in_rational_box(S, Q, Si, R, hulls, tol, features):
    """Survival by the rational definition (no integer bounds)."""
    g = star_geometry(R)
    A, Ain, Aring = g["A"], g["Ain"], g["Aring"]
    ok = True
    if features & 1:
        mu = Fraction(S, A)
        ok &= (1 - tol.mean_rel) * hulls.mu_lo <= mu <= (1 + tol.mean_rel) * hulls.mu_hi
    if features & 2:
        v = Fraction(A * Q - S * S, A * A)
        ok &= (1 - tol.std_rel) ** 2 * hulls.v_lo <= v <= (1 + tol.std_rel) ** 2 * hulls.v_hi
    if features & 4:
        c = Fraction(Si * Aring - (S - Si) * Ain, Ain * Aring)
        lo = hulls.g_lo - tol.grad_rel * abs(hulls.g_lo) - tol.grad_abs
        hi = hulls.g_hi + tol.grad_rel * abs(hulls.g_hi) + tol.grad_abs
        ok &= lo <= c <= hi
    return bool(ok)


def test_bounds_are_tightest_integers():
    rng = np.random.default_rng(1)
    tol = synth.Tolerances(Fraction(1, 20), Fraction(1, 10), Fraction(1, 10), Fraction(4))
    for _ in range(300):
        R = int(rng.integers(2, 200))
        g = star_geometry(R)
        A, D = g["A"], g["Ain"] * g["Aring"]
        mu = sorted(Fraction(int(rng.integers(0, 255 * 997)), 997) for _ in range(2))
        v = sorted(Fraction(int(rng.integers(0, 16000 * 991)), 991) for _ in range(2))
        gg = sorted(Fraction(int(rng.integers(-200 * 983, 200 * 983)), 983) for _ in range(2))
        h = Hulls(mu[0], mu[1], v[0], v[1], gg[0], gg[1])
        b = scale_bounds(h, R, tol, 7)
        lo_m, hi_m = (1 - tol.mean_rel) * h.mu_lo * A, (1 + tol.mean_rel) * h.mu_hi * A
        assert b.S_lo >= lo_m and b.S_lo - 1 < lo_m
        assert b.S_hi <= hi_m and b.S_hi + 1 > hi_m
        lo_v, hi_v = (1 - tol.std_rel) ** 2 * h.v_lo * A * A, (1 + tol.std_rel) ** 2 * h.v_hi * A * A
        assert b.V_lo >= lo_v and b.V_lo - 1 < lo_v
        assert b.V_hi <= hi_v and b.V_hi + 1 > hi_v
        lo_g = (h.g_lo - tol.grad_rel * abs(h.g_lo) - tol.grad_abs) * D
        hi_g = (h.g_hi + tol.grad_rel * abs(h.g_hi) + tol.grad_abs) * D
        assert b.N_lo >= lo_g and b.N_lo - 1 < lo_g
        assert b.N_hi <= hi_g and b.N_hi + 1 > hi_g


def test_template_features_closed_form():
    # constant template: mean c, variance 0, contrast 0
    r = 10
    tm = np.full((2 * r + 1, 2 * r + 1), 93, np.uint8)
    for (t, S, Q, Si) in oracle.template_sums(tm, r, 5):
        mu, v, c = template_features(t, S, Q, Si)
        assert mu == 93 and v == 0 and c == 0


@pytest.mark.parametrize("features", [1, 3, 7, 4, 0])
def test_mask_equals_rational_definition(features):
    H, W = 44, 52
    img = synth.random_image(21, H, W, "blobs")
    r = 9
    tmpl = img[10:10 + 2 * r + 1, 14:14 + 2 * r + 1].copy()
    radii = [5, 6, 8, 9]
    t_min = 6
    tol = synth.Tolerances(Fraction(1, 5), Fraction(1, 3), Fraction(1, 3), Fraction(4))
    res = oracle.screen_workload(img, tmpl, r, t_min, radii, features, tol)
    hulls = res["hulls"]
    mask = res["mask"]
    for s, R in enumerate(radii):
        g = star_geometry(R)
        for y in range(H):
            for x in range(W):
                bit = (int(mask[s, y, x >> 5]) >> (x & 31)) & 1
                inside = (y - g["h"] + 1 >= 0 and y + g["h"] <= H - 1 and
                          x - g["h"] + 1 >= 0 and x + g["h"] - 1 <= W - 1 and
                          y - g["n"] + 1 >= 0 and y + g["n"] <= H - 1 and
                          x - g["n"] + 1 >= 0 and x + g["n"] <= W - 1)
                if not inside:
                    assert bit == 0
                    continue
                S, Q, _ = brute.star_sums(img, y, x, g["n"], g["h"])
                Si, _, _ = brute.star_sums(img, y, x, g["ni"], g["hi"])
                assert bit == _in_rational_box(S, Q, Si, R, hulls, tol, features), (s, y, x)
    # the template's own site survives at the template's own radius
    assert (mask[radii.index(9), 10 + r, (14 + r) >> 5] >> ((14 + r) & 31)) & 1


def test_list_is_sorted_mask_bits():
    img = synth.random_image(5, 70, 90, "blobs")
    r = 8
    tmpl = img[30:47, 40:57].copy()
    tol = synth.Tolerances(Fraction(1, 4), Fraction(1, 2), Fraction(1, 2), Fraction(8))
    res = oracle.screen_workload(img, tmpl, r, 6, [6, 7, 8, 10], 7, tol)
    mask, lst = res["mask"], res["list"]
    S, H, Ww = mask.shape
    bits = np.unpackbits(mask.view(np.uint8).reshape(S, H, Ww, 4)[..., ::-1], axis=-1)
    bits = bits.reshape(S, H, Ww, 4 * 8)[..., ::-1].reshape(S, H, Ww * 32)[:, :, :90]
    s, y, x = np.nonzero(bits)
    keys = (s.astype(np.uint64) << 48) | (y.astype(np.uint64) << 24) | x.astype(np.uint64)
    assert res["count"] == len(keys) > 0
    assert np.array_equal(lst, keys)
    assert np.all(np.diff(lst.astype(np.int64)) > 0)


@pytest.mark.parametrize("seed", list(range(1000, 1008)))
def test_config1_planted_match_survives(seed):
    wl = synth.config1(seed)
    res = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii,
                                 wl.features, wl.tol)
    y, x = wl.planted
    assert (res["mask"][0, y, x >> 5] >> (x & 31)) & 1, "planted match screened out"
    assert res["count"] < 231842 // 4        # the screen prunes most candidates


def _planted_survival(wl):
    """Survival of the planted candidate at each scale, by brute-force sums."""
    sums = oracle.template_sums(wl.template, wl.r, wl.t_min)
    hulls = oracle.template_hulls(sums, wl.features)
    y, x = wl.planted
    out = []
    for R in wl.radii:
        g = star_geometry(R)
        S, Q, _ = brute.star_sums(wl.image, y, x, g["n"], g["h"])
        Si, _, _ = brute.star_sums(wl.image, y, x, g["ni"], g["hi"])
        out.append(_in_rational_box(S, Q, Si, R, hulls, wl.tol, wl.features))
    return out


def _covering(wl):
    return [wl.t_min - 1 <= R / wl.s_true <= wl.r + 1 for R in wl.radii]


@pytest.mark.parametrize("seed", list(range(2000, 2012)))
def test_reduced_planted_match_survives(seed):
    wl = synth.small_planted(seed)
    surv = _planted_survival(wl)
    assert any(s and c for s, c in zip(surv, _covering(wl))), (surv, wl.s_true)


@pytest.mark.slow
@pytest.mark.parametrize("cfg", [2, 3])
def test_large_config_planted_match_survives(cfg):
    wl = synth.CONFIGS[cfg]()
    surv = _planted_survival(wl)
    assert any(s and c for s, c in zip(surv, _covering(wl))), (surv, wl.s_true)


@pytest.mark.parametrize("seed", [5001, 5002, 5003])
def test_tracked_target_survives_in_every_frame(seed):
    """The frame-sequence workload (a panning scene with a drifting, rotating,
    rescaling target): the target's own candidate survives at a covering scale
    in every frame, from brute-force star sums."""
    import types
    fs = synth.frame_sequence(seed)
    for k, img in enumerate(fs.frames):
        wl = types.SimpleNamespace(image=img, template=fs.template, r=fs.r, t_min=fs.t_min, radii=fs.radii,
                                   features=fs.features, tol=fs.tol, planted=fs.planted[k], s_true=fs.s_true[k])
        surv = _planted_survival(wl)
        assert any(s and c for s, c in zip(surv, _covering(wl))), (k, surv, wl.s_true)
