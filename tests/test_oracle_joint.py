"""Pins of the joint membership oracle (oracle/joint.py): the integer forms of
the quantiser against Q(f) = floor(f/q + 1/2) on exact rationals; the template
cells against the paper's neighbours Q(f - q/2), Q(f + q/2); the whole screen
against a brute-force restatement (pixel sums, rationals, a direct loop over
the band); a degenerate case; planted-match survival."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import brute, joint
from oracle.bounds import star_geometry

pytestmark = pytest.mark.filterwarnings("ignore")


def Q_exact(f: Fraction, q: Fraction) -> int:
    return math.floor(f / q + Fraction(1, 2))


def Q_std_exact(V: int, A: int, q: Fraction) -> int:
    """floor(sqrt(V)/A/q + 1/2) by exact comparison of squares (no square root)."""
    x2 = Fraction(V, A * A) / (q * q)          # (sigma / q)^2
    c = 0
    while Fraction(2 * c + 1, 2) ** 2 <= x2:    # sigma/q >= c + 1/2
        c += 1
    return c


def rand_q(rng):
    return Fraction(rng.randint(1, 40), rng.randint(1, 16))


def test_mean_and_contrast_quantisers_match_the_rational_definition():
    rng = random.Random(5)
    for _ in range(3000):
        A = rng.randint(1, 131058)
        S = rng.randint(0, 255 * A)
        q = rand_q(rng)
        assert int(joint.q_mean(S, A, q)) == Q_exact(Fraction(S, A), q)
        Ain, Aring = rng.randint(1, 40000), rng.randint(1, 90000)
        N = rng.randint(-255 * Ain * Aring, 255 * Ain * Aring)
        assert int(joint.q_contrast(N, Ain, Aring, q)) == Q_exact(Fraction(N, Ain * Aring), q)


def test_mean_quantiser_at_exact_half_steps():
    # f/q + 1/2 an integer: the quantiser rounds half up
    for q in (Fraction(4), Fraction(5, 2), Fraction(7, 3)):
        for c in range(0, 60):
            f = (Fraction(2 * c + 1, 2)) * q          # exactly c + 1/2 cells
            A = f.denominator * 6
            S = int(f * A)
            assert int(joint.q_mean(S, A, q)) == c + 1 == Q_exact(Fraction(S, A), q)


def test_std_quantiser_matches_exact_square_comparisons():
    rng = random.Random(6)
    for _ in range(2000):
        A = rng.randint(1, 131058)
        V = rng.randint(0, (A * A * 65025) // 4)
        q = rand_q(rng)
        assert int(joint.q_std(V, A, q)) == Q_std_exact(V, A, q)
    # boundaries: sigma/q exactly c + 1/2 (V a perfect square at the right scale)
    for c in range(0, 40):
        q = Fraction(3, 2)
        A = 4
        sigma2 = (Fraction(2 * c + 1, 2) * q) ** 2 * A * A   # V with sqrt(V)/A/q = c + 1/2
        if sigma2.denominator == 1:
            assert int(joint.q_std(int(sigma2), A, q)) == c + 1 == Q_std_exact(int(sigma2), A, q)


def test_template_cells_are_the_paper_neighbours():
    rng = random.Random(7)
    for _ in range(400):
        t = rng.randint(2, 90)
        g = star_geometry(t)
        A, Ain, Aring = g["A"], g["Ain"], g["Aring"]
        Sin = rng.randint(0, 255 * Ain)
        S = Sin + rng.randint(0, 255 * Aring)
        # a feasible sum of squares: between S^2/A and 255*S
        Q = rng.randint(-(-S * S // A), max(-(-S * S // A), 255 * S))
        q = (rand_q(rng), rand_q(rng), rand_q(rng))
        c = joint.template_floor_cells(t, S, Q, Sin, 7, q)
        mu = Fraction(S, A)
        assert c[0] == Q_exact(mu - q[0] / 2, q[0]) and c[0] + 1 == Q_exact(mu + q[0] / 2, q[0])
        V = A * Q - S * S
        # floor(sigma / q): largest k with k*q <= sigma, by squares
        k = 0
        while ((k + 1) * q[1]) ** 2 <= Fraction(V, A * A):
            k += 1
        assert c[1] == k
        gr = Fraction(Sin * Aring - (S - Sin) * Ain, Ain * Aring)
        assert c[2] == Q_exact(gr - q[2] / 2, q[2]) and c[2] + 1 == Q_exact(gr + q[2] / 2, q[2])


def _brute_joint_mask(img, tmpl, r, radii, area_radii, bands, features, q):
    """The membership screen from its definition: star and inner-star sums by
    direct pixel sums, features as rationals, Q by exact comparison, and the
    band walked for every candidate."""
    H, W = img.shape

    def feats(im, y, x, R):
        g = star_geometry(R)
        S, Qs, A = brute.star_sums(im, y, x, g["n"], g["h"])
        Si, _, Ai = brute.star_sums(im, y, x, g["ni"], g["hi"])
        assert A == g["A"] and Ai == g["Ain"]
        return S, Qs, Si, g

    def cells(S, Qs, Si, g, mode):   # mode 'q': candidate Q(f); 'floor': floor(f/q)
        A, Ain, Aring = g["A"], g["Ain"], g["Aring"]
        out = []
        if features & 1:
            f = Fraction(S, A)
            out.append(Q_exact(f, q[0]) if mode == "q" else math.floor(f / q[0]))
        if features & 2:
            V = A * Qs - S * S
            if mode == "q":
                out.append(Q_std_exact(V, A, q[1]))
            else:
                k = 0
                while ((k + 1) * q[1]) ** 2 <= Fraction(V, A * A):
                    k += 1
                out.append(k)
        if features & 4:
            f = Fraction(Si * Aring - (S - Si) * Ain, Ain * Aring)
            out.append(Q_exact(f, q[2]) if mode == "q" else math.floor(f / q[2]))
        return out

    tcells = {}
    for j, (lo, hi) in enumerate(bands):
        tcells[j] = [cells(*feats(tmpl, r, r, t), "floor") for t in range(lo, hi + 1)]
    Ww = (W + 31) // 32
    mask = np.zeros((len(radii), H, Ww), np.uint32)
    for s, R in enumerate(radii):
        g = star_geometry(R)
        m = max(g["n"], g["h"])
        for y in range(m - 1, H - m):
            for x in range(m - 1, min(W - 1 - g["n"], W - g["h"]) + 1):
                ok = True
                for j in range(len(bands)):
                    c = cells(*feats(img, y, x, area_radii[s][j]), "q")
                    if not any(all(b <= ci <= b + 1 for ci, b in zip(c, base)) for base in tcells[j]):
                        ok = False
                        break
                if ok:
                    mask[s, y, x >> 5] |= np.uint32(1 << (x & 31))
    return mask


@pytest.mark.parametrize("features,qs", [(7, (4, 3, 6)), (3, (Fraction(5, 2), 2, 1)), (5, (3, 1, Fraction(7, 2))),
                                         (2, (1, Fraction(3, 2), 1))])
def test_joint_screen_matches_brute_force(features, qs):
    wl = synth.small_planted(seed=2100 + features, H=96, r=8, n_scales=3)
    py, px = wl.planted                      # a 34 x 41 window around the planted copy
    y0, x0 = max(0, py - 17), max(0, px - 20)
    img, tmpl = wl.image[y0:y0 + 34, x0:x0 + 41], wl.template
    radii = [5, 6, 7]
    area_radii = [[5, 4, 3], [6, 5, 4], [7, 6, 5]]
    bands = [(6, 8), (5, 6), (4, 5)]
    q = tuple(Fraction(v) for v in qs)
    sums = oracle.template_sums(tmpl, 8, 4)
    mask, lst, cnt = joint.screen_joint(oracle.Tables(img), sums, radii, area_radii, bands, features, q)
    want = _brute_joint_mask(img, tmpl, 8, radii, area_radii, bands, features, q)
    assert np.array_equal(mask, want)
    assert cnt == int(sum(bin(int(w)).count("1") for w in want.ravel()))
    assert cnt > 0


def test_coarse_quantiser_keeps_every_valid_candidate():
    wl = synth.small_planted(seed=2200, H=128, r=10, n_scales=2)
    tb = oracle.Tables(wl.image)
    q = (Fraction(1000), Fraction(1000), Fraction(1000))
    radii = [7, 9]
    area_radii = [[7, 5], [9, 7]]
    bands = [(8, 10), (6, 8)]
    sums = oracle.template_sums(wl.template, 10, 5)
    mask, lst, cnt = joint.screen_joint(tb, sums, radii, area_radii, bands, 7, q)
    n_valid = 0
    for R in radii:
        g = star_geometry(R)
        m = max(g["n"], g["h"])
        n_valid += (128 - 2 * m + 1) * (min(127 - g["n"], 128 - g["h"]) - (m - 1) + 1)
    assert cnt == n_valid


def test_joint_is_exactly_the_membership_of_the_cells():
    # a candidate whose cells equal a template radius's cells passes; moving one
    # feature two cells away fails (checked on the set itself)
    sums = [(6, 10000, 900000, 3000)]
    q = (Fraction(4), Fraction(3), Fraction(5))
    F = joint.membership_set(sums, (6, 6), 7, q)
    base = joint.template_floor_cells(6, 10000, 900000, 3000, 7, q)
    assert len(F) == 8 and base in F
    assert tuple(b + 1 for b in base) in F
    assert (base[0] + 2, base[1], base[2]) not in F and (base[0] - 1, base[1], base[2]) not in F


@pytest.mark.parametrize("seed", range(3000, 3010))
def test_planted_match_survives_the_joint_screen(seed):
    """Statistical pin, as for the interval screen: with q = (4, 2, 4) grey
    levels and three nested central areas the planted copy survives at a scale
    whose radius covers its true size."""
    wl = synth.small_planted(seed, H=256, r=16, n_scales=4)
    area_radii, bands = synth.joint_areas(wl.r, wl.scales, 3)
    sums = oracle.template_sums(wl.template, wl.r, max(2, min(b[0] for b in bands)))
    q = (Fraction(4), Fraction(2), Fraction(4))
    mask, _, cnt = joint.screen_joint(oracle.Tables(wl.image), sums, wl.radii, area_radii, bands, 7, q)
    py, px = wl.planted
    hit = [s for s in range(len(wl.radii)) if (mask[s, py, px >> 5] >> (px & 31)) & 1]
    cover = [s for s, R in enumerate(wl.radii) if wl.t_min - 1 <= R / wl.s_true <= wl.r + 1]
    assert set(hit) & set(cover)
    assert cnt < 0.05 * len(wl.radii) * wl.image.size        # and it prunes
