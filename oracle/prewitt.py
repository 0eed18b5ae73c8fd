"""Prewitt gradient magnitude of the star's square -- TEST INFRASTRUCTURE ONLY
(imported by tests/ and bench.py's reference arm).

Follows Sec. 3 (the horizontal and vertical gradients of a 2n x 2n patch as
inner products with the extended Prewitt ramps, Eq. S_y, from the summed-area
map of x * I, Eq. T_x, and its vertical counterpart) and Sec. 4 (the gradient
magnitude, robust to rotation).  Readings:

* Moments are taken about the patch's own centre (the ramp of the Prewitt
  kernel is centred on the patch): the square covering rows y-n+1..y+n and
  columns x-n+1..x+n has centre (y + 1/2, x + 1/2).  Doubled to stay integer:
  Gx2 = sum (2x' - 2x - 1) I,  Gy2 = sum (2y' - 2y - 1) I.
* From moment tables Mx(a, b) = sum_{y<a, x<b} x I and My(a, b) =
  sum_{y<a, x<b} y I (laid out like the upright table):
  Gx2 = 2 * [Mx window] - (2x + 1) * S_sq,  Gy2 = 2 * [My window] - (2y + 1) * S_sq,
  with the window read at the same four corners as the square's sum S_sq.
* The magnitude is normalised like the Prewitt ramp's response to a linear
  ramp: with J2 = sum over the square of (2x' - 2x - 1)^2 = (2n)^2 (4n^2 - 1) / 3
  (the same for rows), a ramp of slope (a, b) gives Gx2 = a J2 / 2, so the
  slope magnitude is m = 2 |(Gx2, Gy2)| / J2 grey levels per pixel.  The
  feature is phi = m * n, the intensity change over the square's half-side: a
  template scaled by k has slopes divided by k and squares of k times the
  half-side, so phi is the quantity that a candidate at radius R shares with the
  template's central square of radius R / k (the band reading used for every
  feature).  phi^2 = 4 n^2 (Gx2^2 + Gy2^2) / J2^2.
* The paper defines the gradient for the square patch only; the star's
  diamond does not enter this feature.
* Interval test on squares (no square root): with the hull [p_lo, p_hi] of the
  template's central squares' phi^2 over the band, a candidate passes when
  phi^2 in [max(0, (1-tau)^2 p_lo - delta^2), (1+tau)^2 p_hi + delta^2], i.e.
  Gx2^2 + Gy2^2 in [ceil(lo J2^2 / (4 n^2)), floor(hi J2^2 / (4 n^2))].
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from .bounds import star_geometry


def moment_tables(img: np.ndarray):
    """(Mx, My): (H+1) x (W+1) int64, Mx[a, b] = sum_{y<a, x<b} x I(y, x)."""
    img = np.asarray(img, dtype=np.int64)
    H, W = img.shape
    xs = np.arange(W, dtype=np.int64)[None, :]
    ys = np.arange(H, dtype=np.int64)[:, None]
    Mx = np.zeros((H + 1, W + 1), np.int64)
    My = np.zeros((H + 1, W + 1), np.int64)
    Mx[1:, 1:] = np.cumsum(np.cumsum(xs * img, axis=0), axis=1)
    My[1:, 1:] = np.cumsum(np.cumsum(ys * img, axis=0), axis=1)
    return Mx, My


def j2(n: int) -> int:
    """sum over the 2n x 2n square of (2x' - 2x - 1)^2 = (2n)^2 (4n^2 - 1) / 3."""
    return (2 * n) * (2 * n) * (4 * n * n - 1) // 3


def square_moments(L1: np.ndarray, Mx: np.ndarray, My: np.ndarray, R: int, ys, xs):
    """(S_sq, Gx2, Gy2) of the square of the star of radius R at (ys, xs)."""
    n = star_geometry(R)["n"]
    ys = np.asarray(ys, np.int64)
    xs = np.asarray(xs, np.int64)
    a1, a0, b1, b0 = ys + n + 1, ys - n + 1, xs + n + 1, xs - n + 1

    def window(T):
        return T[a1, b1] - T[a0, b1] - T[a1, b0] + T[a0, b0]

    S = window(np.asarray(L1, np.int64))
    Gx2 = 2 * window(Mx) - (2 * xs + 1) * S
    Gy2 = 2 * window(My) - (2 * ys + 1) * S
    return S, Gx2, Gy2


def phi2(gx2: int, gy2: int, n: int) -> Fraction:
    """phi^2 = 4 n^2 (Gx2^2 + Gy2^2) / J2^2 of a square of half-side n."""
    return Fraction(4 * n * n * (gx2 * gx2 + gy2 * gy2), j2(n) ** 2)


def template_phi2(tmpl: np.ndarray, r: int, t: int) -> Fraction:
    """phi^2 of the template's central square of the star of radius t (centre (r, r))."""
    Mx, My = moment_tables(tmpl)
    L1 = np.zeros_like(Mx)
    L1[1:, 1:] = np.cumsum(np.cumsum(np.asarray(tmpl, np.int64), axis=0), axis=1)
    _, gx, gy = square_moments(L1, Mx, My, t, [r], [r])
    return phi2(int(gx[0]), int(gy[0]), star_geometry(t)["n"])


def hull_phi2(tmpl: np.ndarray, r: int, t_lo: int, t_hi: int):
    vals = [template_phi2(tmpl, r, t) for t in range(t_lo, t_hi + 1)]
    return min(vals), max(vals)


def g2_bounds(p_lo: Fraction, p_hi: Fraction, R: int, tau, delta):
    """Inclusive integer bounds on Gx2^2 + Gy2^2 at star radius R."""
    tau, delta = Fraction(tau), Fraction(delta)
    lo = max(Fraction(0), (1 - tau) ** 2 * p_lo - delta * delta)
    hi = (1 + tau) ** 2 * p_hi + delta * delta
    n = star_geometry(R)["n"]
    J = j2(n)
    return math.ceil(lo * J * J / (4 * n * n)), math.floor(hi * J * J / (4 * n * n))


def prewitt_mask(L1, Mx, My, H: int, W: int, radii, bounds) -> np.ndarray:
    """(S, H, ceil(W/32)) mask words: valid candidates whose Gx2^2 + Gy2^2 lies in
    bounds[s] (exact Python integers for the 128-bit squares)."""
    Ww = (W + 31) // 32
    mask = np.zeros((len(radii), H, Ww), np.uint32)
    for s, R in enumerate(radii):
        g = star_geometry(R)
        m = max(g["n"], g["h"])
        y0, y1 = m - 1, H - 1 - m
        x0, x1 = m - 1, min(W - 1 - g["n"], W - g["h"])
        if y1 < y0 or x1 < x0:
            continue
        yy, xx = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), indexing="ij")
        ys, xs = yy.ravel(), xx.ravel()
        _, gx, gy = square_moments(L1, Mx, My, R, ys, xs)
        lo, hi = bounds[s]
        ok = np.fromiter((lo <= a * a + b * b <= hi for a, b in zip(gx.tolist(), gy.tolist())), bool, len(ys))
        for y, x in zip(ys[ok].tolist(), xs[ok].tolist()):
            mask[s, y, x >> 5] |= np.uint32(1 << (x & 31))
    return mask


def screen_workload_prewitt(img, tmpl, r: int, t_min: int, radii, features: int, tol, ptol, tables=None):
    """Interval screen (mean, variance, contrast as in oracle.screen_workload)
    and, with feature bit 8, the Prewitt test: a candidate survives when it
    passes every enabled test.  ptol = (tau, delta) of the Prewitt interval."""
    from . import Tables, screen_workload

    tb = tables if tables is not None else Tables(img)
    base = screen_workload(img, tmpl, r, t_min, radii, features & 7, tol, tables=tb)
    mask = base["mask"].copy()
    if features & 8:
        H, W = tb.H, tb.W
        Mx, My = moment_tables(tb.img)
        p_lo, p_hi = hull_phi2(tmpl, r, t_min, r)
        bounds = [g2_bounds(p_lo, p_hi, R, ptol[0], ptol[1]) for R in radii]
        mask &= prewitt_mask(np.asarray(tb.L1, np.int64), Mx, My, H, W, radii, bounds)
    S, H, Ww = mask.shape
    keys = []
    for s, y, w in zip(*np.nonzero(mask)):
        bits = int(mask[s, y, w])
        while bits:
            b = (bits & -bits).bit_length() - 1
            bits &= bits - 1
            keys.append((int(s) << 48) | (int(y) << 24) | (int(w) * 32 + b))
    lst = np.array(sorted(keys), np.uint64)
    return dict(mask=mask, list=lst, count=len(keys))
