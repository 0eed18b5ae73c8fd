"""Pins of the Prewitt gradient oracle (oracle/prewitt.py): moment tables
against direct double sums; square moments against direct pixel sums; the
linear-ramp closed form m^2 = a^2 + b^2; transpose symmetry; the integer bounds
as the tightest integers of the rational inequalities; the mask against a
brute-force restatement."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import prewitt
from oracle.bounds import star_geometry


def _img(seed, H, W):
    return synth.random_image(seed, H, W)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 9), (7, 1), (6, 11), (13, 8)])
def test_moment_tables_are_double_sums(H, W):
    img = _img(H * 100 + W, H, W).astype(np.int64)
    Mx, My = prewitt.moment_tables(img)
    for a in range(H + 1):
        for b in range(W + 1):
            assert Mx[a, b] == sum(x * img[y, x] for y in range(a) for x in range(b))
            assert My[a, b] == sum(y * img[y, x] for y in range(a) for x in range(b))


def _tables(img):
    Mx, My = prewitt.moment_tables(img)
    L1 = np.zeros_like(Mx)
    L1[1:, 1:] = np.cumsum(np.cumsum(np.asarray(img, np.int64), axis=0), axis=1)
    return L1, Mx, My


@pytest.mark.parametrize("kind", ["uniform", "blobs", "max"])
def test_square_moments_are_pixel_sums(kind):
    img = synth.random_image(17, 60, 70, kind=kind).astype(np.int64)
    L1, Mx, My = _tables(img)
    rng = np.random.default_rng(3)
    for R in range(1, 13):
        n = star_geometry(R)["n"]
        if n < 1:
            continue
        m = max(n, R)
        for _ in range(6):
            y = int(rng.integers(m - 1, 60 - m))
            x = int(rng.integers(m - 1, min(69 - n, 70 - R) + 1))
            S, gx, gy = prewitt.square_moments(L1, Mx, My, R, [y], [x])
            ys = np.arange(y - n + 1, y + n + 1)[:, None]
            xs = np.arange(x - n + 1, x + n + 1)[None, :]
            block = img[y - n + 1:y + n + 1, x - n + 1:x + n + 1]
            assert S[0] == block.sum()
            assert gx[0] == ((2 * xs - 2 * x - 1) * block).sum()
            assert gy[0] == ((2 * ys - 2 * y - 1) * block).sum()


def test_j2_is_the_sum_of_squared_doubled_offsets():
    for n in range(1, 40):
        k = np.arange(-n + 1, n + 1)
        assert prewitt.j2(n) == 2 * n * int(((2 * k - 1) ** 2).sum())


@pytest.mark.parametrize("alpha,beta,gamma", [(10, 3, 0), (200, -2, 1), (40, 1, 2), (128, 0, -1)])
def test_linear_ramp_gives_its_slope(alpha, beta, gamma):
    H = W = 56
    yy, xx = np.mgrid[0:H, 0:W]
    img = alpha + beta * xx + gamma * yy
    assert img.min() >= 0 and img.max() <= 255
    L1, Mx, My = _tables(img)
    for R in (2, 5, 9, 14):
        n = star_geometry(R)["n"]
        m = max(n, R)
        for (y, x) in [(m - 1, m - 1), (H - 1 - m, min(W - 1 - n, W - R)), (27, 30)]:
            _, gx, gy = prewitt.square_moments(L1, Mx, My, R, [y], [x])
            assert prewitt.phi2(int(gx[0]), int(gy[0]), n) == (beta * beta + gamma * gamma) * n * n


def test_transpose_swaps_the_components():
    img = synth.random_image(23, 40, 40).astype(np.int64)
    L1, Mx, My = _tables(img)
    L1t, Mxt, Myt = _tables(img.T.copy())
    for R in (3, 6, 10):
        for (y, x) in [(12, 17), (20, 9), (25, 25)]:
            _, gx, gy = prewitt.square_moments(L1, Mx, My, R, [y], [x])
            _, gxt, gyt = prewitt.square_moments(L1t, Mxt, Myt, R, [x], [y])
            assert gx[0] == gyt[0] and gy[0] == gxt[0]


def test_bounds_are_the_tightest_integers():
    rng = np.random.default_rng(9)
    for _ in range(300):
        lo = Fraction(int(rng.integers(0, 4000)), int(rng.integers(1, 97)))
        hi = lo + Fraction(int(rng.integers(0, 4000)), int(rng.integers(1, 97)))
        tau = Fraction(int(rng.integers(0, 30)), 100)
        delta = Fraction(int(rng.integers(0, 20)), int(rng.integers(1, 9)))
        R = int(rng.integers(2, 120))
        L, U = prewitt.g2_bounds(lo, hi, R, tau, delta)
        n = star_geometry(R)["n"]
        J = prewitt.j2(n)
        qlo = max(Fraction(0), (1 - tau) ** 2 * lo - delta * delta) * J * J / (4 * n * n)
        qhi = ((1 + tau) ** 2 * hi + delta * delta) * J * J / (4 * n * n)
        assert L >= qlo and L - 1 < qlo
        assert U <= qhi and U + 1 > qhi


def test_mask_matches_the_definition():
    wl = synth.small_planted(seed=5100, H=96, r=8, n_scales=3)
    py, px = wl.planted
    img = wl.image[max(0, py - 20):py + 20, max(0, px - 22):px + 22]
    H, W = img.shape
    lo, hi = prewitt.hull_phi2(wl.template, 8, 5, 8)
    radii = [5, 6, 8]
    bounds = [prewitt.g2_bounds(lo, hi, R, Fraction(1, 10), Fraction(2)) for R in radii]
    L1, Mx, My = _tables(img)
    mask = prewitt.prewitt_mask(L1, Mx, My, H, W, radii, bounds)
    want = np.zeros_like(mask)
    imgi = img.astype(np.int64)
    for s, R in enumerate(radii):
        g = star_geometry(R)
        n, m = g["n"], max(g["n"], g["h"])
        for y in range(m - 1, H - m):
            for x in range(m - 1, min(W - 1 - n, W - R) + 1):
                block = imgi[y - n + 1:y + n + 1, x - n + 1:x + n + 1]
                gx = int(((2 * np.arange(x - n + 1, x + n + 1) - 2 * x - 1)[None, :] * block).sum())
                gy = int(((2 * np.arange(y - n + 1, y + n + 1) - 2 * y - 1)[:, None] * block).sum())
                p2 = Fraction(4 * n * n * (gx * gx + gy * gy), prewitt.j2(n) ** 2)   # (m n)^2
                if max(Fraction(0), Fraction(81, 100) * lo - 4) <= p2 <= Fraction(121, 100) * hi + 4:
                    want[s, y, x >> 5] |= np.uint32(1 << (x & 31))
    assert np.array_equal(mask, want)
    assert 0 < int(sum(bin(int(v)).count("1") for v in want.ravel())) < sum(
        (H - 2 * max(star_geometry(R)["n"], R) + 1) * (W - 2 * R + 2) for R in radii)
