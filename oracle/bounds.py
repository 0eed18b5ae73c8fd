"""Template feature hulls and per-scale integer bounds, in exact rationals.

TEST INFRASTRUCTURE ONLY (part of the oracle; see oracle/__init__.py).

Paper passages followed (arXiv 1707.05647):
  * Sec. 4: the octagonal star is a square and a 45-degree diamond "of the same
    size" superposed.  Reading: the diamond's half-diagonal is the star radius
    R, the square's half-side n is R/sqrt(2) rounded (the unique integer with
    (2n-1)^2 < 2R^2 < (2n+1)^2), and the star pools the two sums over the
    pooled area A = 4n^2 + 2R^2 (the exact pixel counts of the two shapes).
  * Sec. 3, Eq. S_sigma: variance = second moment / area - mean^2; scaled by
    A^2 this is the integer V = A*Q - S^2.
  * Sec. 5, central areas: the contrast feature compares the mean of the inner
    star of radius floor(R/2) with the mean of the rest (the ring):
    g = S_in/A_in - S_ring/A_ring, scaled by A_in*A_ring to N.
  * Sec. 5, Eq. F_n and Algorithm 1: a scale band accepts any feature value of
    the template's central area for central radii in [r/lambda, r]; here one
    closed interval (the hull) per feature, widened by the tolerances.
  * Sec. 5, quantiser Q(f) = floor(f/q + 1/2) with neighbours +-q/2: replaced by
    exact interval tests; every interval is closed, low bound rounded up, high
    bound rounded down.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from fractions import Fraction

I64_MIN = -(1 << 63)
I64_MAX = (1 << 63) - 1


def _square_half(R: int) -> int:
    n = 0
    while (2 * n + 1) ** 2 < 2 * R * R:
        n += 1
    return n


def star_geometry(R: int) -> dict:
    """n, h, inner radius, pooled areas of the star of radius R (Sec. 4, Sec. 5)."""
    n = _square_half(R)
    h = R
    ri = R // 2
    ni = _square_half(ri)
    A = 4 * n * n + 2 * h * h
    Ain = 4 * ni * ni + 2 * ri * ri
    return dict(R=R, n=n, h=h, ri=ri, ni=ni, hi=ri, A=A, Ain=Ain, Aring=A - Ain)


@dataclass
class Hulls:
    mu_lo: Fraction
    mu_hi: Fraction
    v_lo: Fraction
    v_hi: Fraction
    g_lo: Fraction | None
    g_hi: Fraction | None


def template_features(t: int, S: int, Q: int, Sin: int):
    """(mean, variance, contrast) of the template's central star of radius t, exact."""
    g = star_geometry(t)
    A, Ain, Aring = g["A"], g["Ain"], g["Aring"]
    mu = Fraction(S, A)
    v = Fraction(A * Q - S * S, A * A)
    c = Fraction(Sin * Aring - (S - Sin) * Ain, Ain * Aring) if Ain > 0 else None
    return mu, v, c


def template_hulls(sums, features: int) -> Hulls:
    """Hull of each feature over the central radii t of the band (Eq. F_n)."""
    mus, vs, gs = [], [], []
    for (t, S, Q, Sin) in sums:
        mu, v, g = template_features(t, S, Q, Sin)
        mus.append(mu)
        vs.append(v)
        if features & 4:
            if g is None:
                raise ValueError("contrast needs central radius >= 2")
            gs.append(g)
    return Hulls(min(mus), max(mus), min(vs), max(vs),
                 min(gs) if gs else None, max(gs) if gs else None)


@dataclass
class ScaleBounds:
    S_lo: int
    S_hi: int
    V_lo: int
    V_hi: int
    N_lo: int
    N_hi: int

    def as_row(self):
        return [self.S_lo, self.S_hi, self.V_lo, self.V_hi, self.N_lo, self.N_hi]


def _clamp(v: int) -> int:
    return max(I64_MIN, min(I64_MAX, v))


def scale_bounds(h: Hulls, R: int, tol, features: int) -> ScaleBounds:
    """Inclusive integer bounds on S, V, N at star radius R.

    mean:      S/A      in [(1-tm) mu_lo, (1+tm) mu_hi]
    std:       sqrt(V)/A in [(1-ts) sd_lo, (1+ts) sd_hi]  (squared: no root)
    contrast:  N/(Ain*Aring) in [g_lo - tg|g_lo| - dg, g_hi + tg|g_hi| + dg]
    Disabled features get the full int64 range.
    """
    g = star_geometry(R)
    A, Ain, Aring = g["A"], g["Ain"], g["Aring"]
    tm, ts, tg, dg = (Fraction(tol.mean_rel), Fraction(tol.std_rel),
                      Fraction(tol.grad_rel), Fraction(tol.grad_abs))
    S_lo, S_hi = I64_MIN, I64_MAX
    V_lo, V_hi = I64_MIN, I64_MAX
    N_lo, N_hi = I64_MIN, I64_MAX
    if features & 1:
        S_lo = math.ceil((1 - tm) * h.mu_lo * A)
        S_hi = math.floor((1 + tm) * h.mu_hi * A)
    if features & 2:
        V_lo = math.ceil((1 - ts) ** 2 * h.v_lo * A * A)
        V_hi = math.floor((1 + ts) ** 2 * h.v_hi * A * A)
    if features & 4:
        D = Ain * Aring
        N_lo = math.ceil((h.g_lo - tg * abs(h.g_lo) - dg) * D)
        N_hi = math.floor((h.g_hi + tg * abs(h.g_hi) + dg) * D)
    return ScaleBounds(*[_clamp(v) for v in (S_lo, S_hi, V_lo, V_hi, N_lo, N_hi)])
