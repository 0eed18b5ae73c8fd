"""Joint-vector membership screen over nested central areas -- TEST
INFRASTRUCTURE ONLY (imported by tests/ and bench.py's reference arm).

This restates, for the octagonal star of Sec. 4, the exact membership test of
Sec. 5 (Algorithm 1 with the feature set F_n of Eq. F_n and the quantiser Q)
and the check of several central areas that closes Sec. 5:

* A feature value f is quantised with the paper's uniform quantiser
  Q(f) = floor(f / q + 1/2), one factor q per feature (mean, standard
  deviation, inner-star contrast; all in grey levels).
* The template side marks, for every central radius t of an area's band,
  the cells Q(f_t - q/2) and Q(f_t + q/2) of each feature (the paper's
  neighbour marking), jointly: the cell vectors in the product of those pairs.
  Q(f - q/2) = floor(f/q) and Q(f + q/2) = floor(f/q) + 1 exactly.
* A candidate passes an area when the vector of its quantised features is a
  marked cell vector; it survives when it passes every area (the paper marks a
  patch unmatched if any one of its central areas does not match).

Readings (the paper states the test for one feature and square patches): area
j of a candidate at scale s is the star of radius area_radii[s][j] at the same
centre (area 0 is the scale's own star); its band is an inclusive range of the
template's own central radii; the standard deviation of a star is
sqrt(V) / A with V = A*Q - S^2; the contrast is N / (A_in * A_ring) as in the
interval screen.  Everything is exact integer arithmetic: the formulas below
are the quantiser written for integer sums, and tests pin each of them against
Q evaluated on exact rationals.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from .bounds import star_geometry

MEAN, VAR, GRAD = 1, 2, 4


def _isqrt_vec(z: np.ndarray) -> np.ndarray:
    """floor(sqrt(z)) of non-negative int64 values below 2^62, exactly."""
    z = np.asarray(z, dtype=np.int64)
    w = np.floor(np.sqrt(z.astype(np.float64))).astype(np.int64)
    for _ in range(2):
        w = np.where(w * w > z, w - 1, w)
        w = np.where((w + 1) * (w + 1) <= z, w + 1, w)
    return w


def _floordiv(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.floor_divide(np.asarray(a, dtype=np.int64), np.asarray(b, dtype=np.int64))


# ---- quantiser on a candidate's integer sums: Q(f) = floor(f/q + 1/2) --------

def q_mean(S, A, q: Fraction):
    """Q(S / A): floor((2*S*qd + A*qn) / (2*A*qn))."""
    qn, qd = q.numerator, q.denominator
    return _floordiv(2 * np.asarray(S, np.int64) * qd + np.asarray(A, np.int64) * qn, 2 * np.asarray(A, np.int64) * qn)


def q_std(V, A, q: Fraction):
    """Q(sqrt(V) / A): with w = isqrt(4*qd^2*V), floor((w + A*qn) / (2*A*qn))."""
    qn, qd = q.numerator, q.denominator
    w = _isqrt_vec(4 * qd * qd * np.asarray(V, np.int64))
    A = np.asarray(A, np.int64)
    return _floordiv(w + A * qn, 2 * A * qn)


def q_contrast(N, Ain, Aring, q: Fraction):
    """Q(N / (Ain*Aring)): floor((2*N*qd + Ain*Aring*qn) / (2*Ain*Aring*qn)), signed."""
    qn, qd = q.numerator, q.denominator
    D = np.asarray(Ain, np.int64) * np.asarray(Aring, np.int64)
    return _floordiv(2 * np.asarray(N, np.int64) * qd + D * qn, 2 * D * qn)


# ---- template side: floor(f / q), the lower of the two marked cells ----------

def template_floor_cells(t: int, S: int, Q: int, Sin: int, features: int, q) -> tuple:
    """(floor(mu/q), floor(sigma/q), floor(g/q)) of the template's central star of
    radius t, for the enabled features, in that order."""
    g = star_geometry(t)
    A, Ain, Aring = g["A"], g["Ain"], g["Aring"]
    out = []
    if features & MEAN:
        qn, qd = q[0].numerator, q[0].denominator
        out.append((S * qd) // (A * qn))
    if features & VAR:
        qn, qd = q[1].numerator, q[1].denominator
        V = A * Q - S * S
        out.append(math.isqrt(V * qd * qd) // (A * qn))
    if features & GRAD:
        qn, qd = q[2].numerator, q[2].denominator
        N = Sin * Aring - (S - Sin) * Ain
        out.append((N * qd) // (Ain * Aring * qn))
    return tuple(out)


def membership_set(sums, band, features: int, q) -> set:
    """F for one area: every cell vector in the product of {c, c + 1} over the
    enabled features, for the template's central radii t in band (inclusive)."""
    cells = set()
    for (t, S, Q, Sin) in sums:
        if band[0] <= t <= band[1]:
            base = template_floor_cells(t, S, Q, Sin, features, q)
            k = len(base)
            for bits in range(1 << k):
                cells.add(tuple(base[i] + ((bits >> i) & 1) for i in range(k)))
    return cells


def candidate_cells(tables, rho: int, ys, xs, features: int, q) -> np.ndarray:
    """Quantised feature vectors (one row per candidate) of the stars of radius
    rho centred at (ys, xs)."""
    f = tables.features_at(rho, ys, xs)   # S, Q, S_in, V, N, valid
    g = star_geometry(rho)
    cols = []
    if features & MEAN:
        cols.append(q_mean(f[:, 0], g["A"], q[0]))
    if features & VAR:
        cols.append(q_std(f[:, 3], g["A"], q[1]))
    if features & GRAD:
        cols.append(q_contrast(f[:, 4], g["Ain"], g["Aring"], q[2]))
    return np.stack(cols, axis=1) if cols else np.zeros((len(ys), 0), np.int64)


def screen_joint(tables, sums, radii, area_radii, bands, features: int, q, rows=None):
    """Mask words (S, H, ceil(W/32)), ascending key list and count of the joint
    membership screen.  area_radii[s][j]: star radius of area j at scale s;
    bands[j] = (t_lo, t_hi): area j's band of template central radii.  rows:
    evaluate only these image rows (the rest of the mask stays 0)."""
    H, W = tables.H, tables.W
    S = len(radii)
    n_areas = len(bands)
    sets = [membership_set(sums, bands[j], features, q) for j in range(n_areas)]
    Ww = (W + 31) // 32
    mask = np.zeros((S, H, Ww), np.uint32)
    keys = []
    for s, R in enumerate(radii):
        g = star_geometry(R)
        m = max(g["n"], g["h"])
        y0, y1 = m - 1, H - 1 - m
        x0, x1 = m - 1, min(W - 1 - g["n"], W - g["h"])
        if y1 < y0 or x1 < x0:
            continue
        ys_all = np.arange(y0, y1 + 1)
        if rows is not None:
            ys_all = ys_all[np.isin(ys_all, np.asarray(rows))]
        yy, xx = np.meshgrid(ys_all, np.arange(x0, x1 + 1), indexing="ij")
        ys, xs = yy.ravel(), xx.ravel()
        alive = np.ones(len(ys), bool)
        for j in range(n_areas):
            cells = candidate_cells(tables, area_radii[s][j], ys, xs, features, q)
            alive &= np.fromiter((tuple(c) in sets[j] for c in cells.tolist()), bool, len(ys))
        ys, xs = ys[alive], xs[alive]
        for y, x in zip(ys.tolist(), xs.tolist()):
            mask[s, y, x >> 5] |= np.uint32(1 << (x & 31))
            keys.append((s << 48) | (y << 24) | x)
    lst = np.array(sorted(keys), np.uint64)
    return mask, lst, len(keys)
