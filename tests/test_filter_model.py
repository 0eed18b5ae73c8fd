"""A model of the screening kernel's packed-plane pre-filter, on the CPU.

The kernel bounds a candidate's pooled sums S and Q from the signed sum of
its star's eight packed corners (each corner holding bits kS..kS+15 of the sum
table and bits kQ..kQ+15 of the squares' table) and rejects the candidate when
A Q - S^2 is certainly below the variance interval, in single precision, with
a rounding margin added on the host.  This test restates those steps with
numpy on the oracle's exact tables.  Every value the kernel rounds is an
integer here, so each rounding is taken once, from the exact integer, as a
fused multiply-add does: the model's decisions are the kernel's.  It checks
the two facts the kernel's exactness rests on:

* within a window's range (S <= S_hi' <= 2^kS (2^16 - 8) and
  Q <= Q_hi' <= 2^kQ (2^16 - 16)), the biased packed sum (s + 4, q + 8 with
  the low half's carry) puts S and Q in open boxes:
  2^kS (s + 4 - 8) < S < 2^kS (s + 4) and 2^kQ (q + 8 - 16) < Q < 2^kQ (q + 8);
* no candidate that passes the exact mean and variance tests is rejected.

The GPU tests compare the kernel's masks with the oracle on the windows the
host picks; this runs the argument on every window whose range holds a scale,
on images whose sums reach both ends of that range."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle.bounds import scale_bounds, star_geometry, template_hulls

F32 = np.float32
U = 2.0 ** -24


def _toward_down(v):
    """Largest float32 at or below each double of v."""
    v = np.asarray(v, np.float64)
    x = v.astype(F32)
    return np.where(x.astype(np.float64) > v, np.nextafter(x, F32(-np.inf)), x)


def _packed(a, b, kS, kQ):
    return ((a >> kS) & 0xFFFF) | (((b >> kQ) & 0xFFFF) << 16)


def _keep(A, kS, kQ, s4, q8, S_lo, V_lo):
    """The kernel's single-precision decision for biased fields s4 = s + 4 and
    q8 = q + 8 (+ carry): keep unless round(round(A 2^kQ q8) - m^2) is below
    V_lo - M rounded down, m = max(2^kS (s4 - 8), S_lo rounded down),
    M = 4 u (A 2^kQ 65535 + |V_lo|) + 1, u = 2^-24.  S_lo and V_lo are
    scalars or one per candidate."""
    c = A * (1 << kQ)
    slo = np.maximum((s4 - 8) << kS, _toward_down(S_lo).astype(np.int64))
    x = (c * q8).astype(np.float64).astype(F32).astype(np.int64)     # c q8 < 2^49: exact in a double
    lhs = (x - slo * slo).astype(F32)                                  # one rounding, as the fma
    v = np.asarray(V_lo, np.int64).astype(np.float64)                  # |V_lo| < 2^53 here: exact
    vlo = _toward_down(v - (4 * U * (c * 65535.0 + np.abs(v)) + 1))
    return lhs >= vlo


def _model(img, tmpl, r, t_min, radii, features, tol, windows, slack=None):
    """Run the model over every scale and every window that holds it; returns
    (candidates whose boxes were checked, filter decisions made, rejections,
    in-range candidates below the variance's lower bound by more than a
    quarter of it, rejections among those).  With slack set, a scale uses
    only windows at most that many bits coarser than its narrowest usable
    shifts, as the host assigns them."""
    assert features & 2, "the pre-filter tests the variance's lower bound"
    tb = oracle.Tables(img)
    L1, L2 = tb.L1.astype(np.int64), tb.L2.astype(np.int64)
    T1, T2 = tb.T1.astype(np.int64), tb.T2.astype(np.int64)
    hulls = template_hulls(oracle.template_sums(tmpl, r, t_min), features)
    H, W = img.shape
    boxed = decided = rejected = far = far_rejected = 0
    for R in radii:
        g = star_geometry(R)
        n, h, A = g["n"], g["h"], g["A"]
        b = scale_bounds(hulls, R, tol, features)
        S_lo = max(b.S_lo, 0) if features & 1 else 0
        S_hi = min(b.S_hi, 255 * A) if features & 1 else 255 * A
        Q_hi = min(max(0, b.V_hi + S_hi * S_hi) // A, 65025 * A)
        ys = np.arange(R - 1, H - R)
        xs = np.arange(R - 1, min(W - 1 - n, W - R) + 1)
        if len(ys) == 0 or len(xs) == 0:
            continue
        Y, X = np.meshgrid(ys, xs, indexing="ij")

        def star(T, C):
            sq = T[Y + n + 1, X + n + 1] - T[Y - n + 1, X + n + 1] - T[Y + n + 1, X - n + 1] + T[Y - n + 1, X - n + 1]
            dm = C[Y + h + 1, X + 1] - C[Y + 1, X - h + 1] - C[Y + 1, X + h + 1] + C[Y - h + 1, X + 1]
            return sq + dm

        S, Q = star(L1, T1), star(L2, T2)
        passes = (S >= b.S_lo) & (S <= b.S_hi) & (A * Q - S * S >= b.V_lo) & (A * Q - S * S <= b.V_hi)
        inrange = (S <= S_hi) & (Q <= Q_hi)
        ks_min = next(k for k in range(64) if S_hi <= (1 << k) * (65536 - 8))
        kq_min = next(k for k in range(64) if Q_hi <= (1 << k) * (65536 - 16))
        for kS, kQ in windows:
            if kS < ks_min or kQ < kq_min:
                continue            # the window's range does not hold this scale
            if slack is not None and (kS > ks_min + slack or kQ > kq_min + slack):
                continue
            # 32-bit wrapping sum of the packed corners plus the folded offsets
            biased = (star(_packed(L1, L2, kS, kQ), _packed(T1, T2, kS, kQ)) + (8 << 16) + 4) & 0xFFFFFFFF
            s4 = biased & 0xFFFF
            q8 = biased >> 16
            box = (S > (s4 - 8) << kS) & (S < s4 << kS) & (Q > (q8 - 16) << kQ) & (Q < q8 << kQ)
            assert np.all(box | ~inrange), (R, kS, kQ, int((~box & inrange).sum()))
            boxed += int(inrange.sum())
            keep = _keep(A, kS, kQ, s4, q8, S_lo, b.V_lo)
            bad = passes & ~keep
            assert not np.any(bad), (R, kS, kQ, np.argwhere(bad)[:3].tolist())
            decided += S.size
            rejected += int((~keep).sum())
            below = (A * Q - S * S < b.V_lo - b.V_lo // 4) & inrange
            far += int(below.sum())
            far_rejected += int((below & ~keep).sum())
    return boxed, decided, rejected, far, far_rejected


WINDOWS = [(0, 0), (2, 9), (3, 11), (4, 12), (5, 12), (5, 13), (6, 14), (8, 16), (9, 16), (14, 16)]
WIDE = synth.Tolerances(Fraction(9, 10), Fraction(9, 10), Fraction(1, 10), Fraction(4))


@pytest.mark.parametrize("kind", ["planted", "uniform", "max", "zero", "split", "checker"])
def test_filter_model_extreme_images(kind):
    """With the mean test off (features 2) a scale's range is the whole
    [0, 255 A] x [0, 65025 A], reached by the saturated image; with it on and
    wide intervals (features 3) the range ends inside.  Half-saturated and
    checkered images put S and Q at levels between."""
    wl = synth.small_planted(51, H=128, r=12, n_scales=3, sum_bits=32, sq_bits=64)
    if kind == "planted":
        img = wl.image
    elif kind == "split":
        img = synth.random_image(5, 128, 128, "max")
        img[:, 64:] = 0
    elif kind == "checker":
        yy, xx = np.mgrid[0:128, 0:128]
        img = np.where((yy + xx) % 2 == 0, 255, 0).astype(np.uint8)
    else:
        img = synth.random_image(5, 128, 128, kind)
    boxed = decided = 0
    for features in (2, 3):
        b, d, *_ = _model(img, wl.template, wl.r, wl.t_min, wl.radii, features, WIDE, WINDOWS)
        boxed, decided = boxed + b, decided + d
    assert boxed > 0 and decided > 0


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_filter_model_planted(seed):
    """Default intervals on planted images: the model keeps every passing
    candidate and, with windows near the narrowest usable, rejects nearly every
    candidate whose variance is well below the interval."""
    wl = synth.small_planted(seed, H=192, r=14, n_scales=4, sum_bits=32, sq_bits=64)
    _, decided, rejected, far, far_rejected = _model(wl.image, wl.template, wl.r, wl.t_min, wl.radii,
                                                     wl.features, wl.tol, WINDOWS, slack=3)
    assert decided > 0 and far > 0 and far_rejected > 0.9 * far


def test_filter_model_near_zero_variance():
    """A flat template makes the variance interval hug zero, where the
    margin's constant term matters: flat patches must still pass."""
    wl = synth.small_planted(65, H=128, r=12, n_scales=3, sum_bits=32, sq_bits=64)
    tmpl = np.full_like(wl.template, 128)
    img = synth.random_image(7, 128, 128, "uniform")
    img[20:100, 20:100] = 128
    boxed, decided, *_ = _model(img, tmpl, wl.r, wl.t_min, wl.radii, 3, wl.tol, WINDOWS)
    assert decided > 0



@pytest.mark.parametrize("R", [2, 3, 8, 22, 64, 128, 181])
def test_filter_arithmetic_edges(R):
    """The decision on its own, at the worst corners of the boxes: for S and Q
    anywhere in a window's range with A Q >= S^2, take the largest s + 4 and
    the smallest q + 8 whose boxes still hold them, set V_lo = A Q - S^2 (the
    candidate passes the variance test with nothing to spare) and S_lo = 0 or
    S; the kernel must keep it, on every window of every radius (A up to
    131058, the area at the largest radius 181)."""
    rng = np.random.default_rng(R)
    A = star_geometry(R)["A"]
    n = 512
    for kS in range(15):
        for kQ in range(17):
            S_top = min(255 * A, (1 << kS) * (65536 - 8))
            Q_top = min(65025 * A, (1 << kQ) * (65536 - 16))
            Q = np.concatenate([rng.integers(0, Q_top + 1, n - 2), [Q_top, max(Q_top - 1, 0)]])
            root = np.minimum(np.array([math.isqrt(int(A * q)) for q in Q], np.int64), S_top)
            pick = rng.integers(0, 3, n)
            S = np.where(pick == 0, root,
                         np.where(pick == 1, root - rng.integers(0, 64, n), (rng.random(n) * (root + 1)).astype(np.int64)))
            S = S.clip(0)
            s4 = -(-S >> kS) + 7                      # ceil(S / 2^kS) + 7: S just above 2^kS (s4 - 8)
            q8 = (Q >> kQ) + 1                        # Q just below 2^kQ q8
            assert np.all(s4 <= 0xFFFF) and np.all(q8 <= 0xFFFF)
            assert np.all((S > (s4 - 8) << kS) & (S < s4 << kS) & (Q > (q8 - 16) << kQ) & (Q < q8 << kQ))
            V = A * Q - S * S
            assert np.all(V >= 0)
            for S_lo in (np.zeros(n, np.int64), S):
                keep = _keep(A, kS, kQ, s4, q8, S_lo, V)
                assert np.all(keep), (R, kS, kQ, np.argwhere(~keep)[:3].ravel().tolist())
