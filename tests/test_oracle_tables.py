"""Pins of the oracle's tables and window sums against things other than itself:
numpy's cumulative sums (a textbook routine), brute-force pixel-set sums,
closed forms, and a flip invariance.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from synth import random_image

SIZES = [(1, 1), (1, 7), (9, 1), (2, 3), (13, 17), (33, 31), (64, 80)]


@pytest.mark.parametrize("H,W", SIZES)
def test_upright_equals_numpy_cumsum(H, W):
    img = random_image(11 + H * 7 + W, H, W)
    L1, L2 = oracle.upright_tables(img)
    v = img.astype(np.uint64)
    ref1 = np.zeros((H + 1, W + 1), np.uint64)
    ref2 = np.zeros((H + 1, W + 1), np.uint64)
    ref1[1:, 1:] = np.cumsum(np.cumsum(v, 0), 1)
    ref2[1:, 1:] = np.cumsum(np.cumsum(v * v, 0), 1)
    assert np.array_equal(L1, ref1)
    assert np.array_equal(L2, ref2)
    assert int(L1[H, W]) == int(v.sum())          # total of the image


@pytest.mark.parametrize("H,W", [(1, 1), (1, 5), (5, 1), (4, 4), (13, 17), (20, 9), (31, 33)])
def test_cone_equals_brute_force(H, W):
    img = random_image(5 + H * 3 + W, H, W)
    T1, T2 = oracle.cone_tables(img)
    assert T1.shape == (H + 1, W + 2)
    for a in range(H + 1):
        for b in range(W + 2):
            r, c = a - 1, b - 1
            if r < 0:
                assert T1[a, b] == 0 and T2[a, b] == 0
                continue
            assert int(T1[a, b]) == brute.cone_entry(img, r, c, 1), (a, b)
            assert int(T2[a, b]) == brute.cone_entry(img, r, c, 2), (a, b)


def test_cone_closed_form_all_ones():
    H, W = 20, 45
    img = np.ones((H, W), np.uint8)
    T1, _ = oracle.cone_tables(img)
    for r in range(H):
        for c in range(r, W - r):            # cone fully inside horizontally
            assert int(T1[r + 1, c + 1]) == (r + 1) ** 2
    Z1, Z2 = oracle.cone_tables(np.zeros((H, W), np.uint8))
    assert not Z1.any() and not Z2.any()


def test_square_half_definition():
    for R in range(1, 400):
        n = oracle.square_half(R)
        assert (2 * n - 1) ** 2 < 2 * R * R < (2 * n + 1) ** 2
        assert n == int(math.floor(R / math.sqrt(2.0) + 0.5))   # rounding of R/sqrt(2)
        assert n == oracle.star_geometry(R)["n"]


def _valid_positions(H, W, R):
    g = oracle.star_geometry(R)
    n, h = g["n"], g["h"]
    out = []
    for y in range(H):
        for x in range(W):
            if (y - n + 1 >= 0 and y + n <= H - 1 and x - n + 1 >= 0 and x + n <= W - 1 and
                    y - h + 1 >= 0 and y + h <= H - 1 and x - h + 1 >= 0 and x + h - 1 <= W - 1):
                out.append((y, x))
    return out


@pytest.mark.parametrize("kind", ["uniform", "blobs", "max"])
def test_star_sums_equal_brute_force(kind):
    H, W = 40, 44
    img = random_image(77, H, W, kind)
    tb = oracle.Tables(img)
    rng = np.random.default_rng(3)
    for R in range(1, 13):
        g = oracle.star_geometry(R)
        pos = _valid_positions(H, W, R)
        assert pos, R
        if len(pos) > 120:
            pos = [pos[i] for i in rng.choice(len(pos), 120, replace=False)]
        ys = [p[0] for p in pos]
        xs = [p[1] for p in pos]
        f = tb.features_at(R, ys, xs)
        for i, (y, x) in enumerate(pos):
            S, Q, A = brute.star_sums(img, y, x, g["n"], g["h"])
            assert A == g["A"]
            assert f[i, 5] == 1
            assert f[i, 0] == S and f[i, 1] == Q
            assert f[i, 3] == A * Q - S * S
            if g["ri"] >= 1:
                Si, _, Ai = brute.star_sums(img, y, x, g["ni"], g["hi"])
                assert Ai == g["Ain"]
                assert f[i, 2] == Si
                assert f[i, 4] == Si * g["Aring"] - (S - Si) * g["Ain"]


def test_invalid_positions_flagged():
    H, W = 30, 30
    tb = oracle.Tables(random_image(1, H, W))
    R = 6
    valid = set(_valid_positions(H, W, R))
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    f = tb.features_at(R, ys.ravel(), xs.ravel())
    for i, (y, x) in enumerate(zip(ys.ravel(), xs.ravel())):
        assert f[i, 5] == ((int(y), int(x)) in valid)
    g = oracle.star_geometry(R)
    # valid range: y in [R-1, H-1-R], x in [R-1, W-R] for R >= 2
    assert valid == {(y, x) for y in range(R - 1, H - R) for x in range(R - 1, W - R + 1)}
    assert len(valid) == (H - 2 * R + 1) * (W - 2 * R + 2)
    assert g["n"] <= R - 1


def test_shape_areas_on_ones_image():
    img = np.ones((60, 60), np.uint8)
    for h in range(1, 20):
        m = brute.diamond_mask(60, 60, 30, 30, h)
        assert int(m.sum()) == 2 * h * h                      # diamond holds 2h^2 pixels
    tb = oracle.Tables(img)
    for R in range(2, 20):
        g = oracle.star_geometry(R)
        f = tb.features_at(R, [30], [30])[0]
        assert f[0] == g["A"] and f[1] == g["A"] and f[2] == g["Ain"]


def test_closed_form_constant_image():
    for c in (0, 1, 17, 200, 255):
        tb = oracle.Tables(np.full((50, 52), c, np.uint8))
        for R in (2, 5, 9, 12):
            g = oracle.star_geometry(R)
            f = tb.features_at(R, [20, 25], [20, 26])
            assert (f[:, 0] == c * g["A"]).all()
            assert (f[:, 1] == c * c * g["A"]).all()
            assert (f[:, 3] == 0).all() and (f[:, 4] == 0).all()


def test_closed_form_ramps():
    a, b = 2, 11
    H, W = 60, 100
    col = (a * np.arange(W)[None, :] + b).repeat(H, 0).astype(np.uint8)
    row = (a * np.arange(H)[:, None] + b).repeat(W, 1).astype(np.uint8)
    tc, tr = oracle.Tables(col), oracle.Tables(row)
    for R in (2, 3, 7, 10):
        g = oracle.star_geometry(R)
        n, h = g["n"], g["h"]
        for (y, x) in [(20, 30), (25, 51), (30, 70)]:
            # diamond is symmetric about column x: mean a*x + b; square about x + 1/2
            S = tc.features_at(R, [y], [x])[0, 0]
            assert S == 4 * n * n * (a * x + b) + 2 * n * n * a + 2 * h * h * (a * x + b)
            # both shapes are symmetric about row y + 1/2
            S = tr.features_at(R, [y], [x])[0, 0]
            assert 2 * S == g["A"] * (2 * a * y + a + 2 * b)


def test_vertical_flip_invariance():
    H, W = 45, 50
    img = random_image(9, H, W, "uniform")
    t0, t1 = oracle.Tables(img), oracle.Tables(img[::-1].copy())
    for R in (2, 4, 7, 11):
        pos = _valid_positions(H, W, R)
        ys = np.array([p[0] for p in pos])
        xs = np.array([p[1] for p in pos])
        f0 = t0.features_at(R, ys, xs)
        f1 = t1.features_at(R, H - 2 - ys, xs)
        assert np.array_equal(f0, f1)


def test_template_sums_equal_brute_force():
    r = 14
    tm = random_image(4, 2 * r + 1, 2 * r + 1, "blobs")
    sums = oracle.template_sums(tm, r, 9)
    for (t, S, Q, Si) in sums:
        g = oracle.star_geometry(t)
        bS, bQ, _ = brute.star_sums(tm, r, r, g["n"], g["h"])
        bSi, _, _ = brute.star_sums(tm, r, r, g["ni"], g["hi"])
        assert (S, Q, Si) == (bS, bQ, bSi)


def _golden_maps():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "star_weights.txt")
    maps, cur = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("R "):
            t = line.split()
            cur = (int(t[1]), int(t[3]), int(t[5]))
            maps[cur] = []
        else:
            maps[cur].append([int(v) for v in line.split()])
    return {k: np.array(v) for k, v in maps.items()}


def test_star_weights_match_hand_derived_golden():
    """Delta image: the oracle's star sum at (y, x) is the weight of the pixel's offset."""
    H, W = 24, 24
    py, px = 12, 12
    img = np.zeros((H, W), np.uint8)
    img[py, px] = 1
    tb = oracle.Tables(img)
    for (R, dy0, dx0), wmap in _golden_maps().items():
        got = np.zeros_like(wmap)
        for i in range(wmap.shape[0]):
            for j in range(wmap.shape[1]):
                # pixel offset (dy0+i, dx0+j) from candidate (y, x) => candidate at pixel - offset
                y, x = py - (dy0 + i), px - (dx0 + j)
                got[i, j] = tb.features_at(R, [y], [x])[0, 0]
        assert np.array_equal(got, wmap), (R, got)
        assert int(wmap.sum()) == oracle.star_geometry(R)["A"]
        bw = brute.star_weights(H, W, py, px, oracle.star_geometry(R)["n"], R)
        assert np.array_equal(bw[py + dy0:py + dy0 + wmap.shape[0], px + dx0:px + dx0 + wmap.shape[1]], wmap)
        assert int(bw.sum()) == int(wmap.sum())
