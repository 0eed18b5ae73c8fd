"""Brute-force pixel-set sums, no tables -- TEST INFRASTRUCTURE ONLY.

Direct restatement of the regions the paper's table lookups sum over, used to
pin the oracle's tables and corner formulas on small images:
  * upright table  L(a, b) = sum_{y<a, x<b} I          (Sec. 3, Eq. T_1)
  * square         rows y-n+1..y+n, columns x-n+1..x+n  (Sec. 3, Eq. S_1)
  * cone           y <= r, |x - c| <= r - y             (Sec. 4, triangular map)
  * diamond        |x'-x| <= h-1, y-h+|x'-x| < y' <= y+h-|x'-x|   (Sec. 4)
  * star           square + diamond, pooled             (Sec. 4, Eq. S_os)
"""
from __future__ import annotations

import numpy as np


def upright_entry(img: np.ndarray, a: int, b: int) -> int:
    return int(img[:a, :b].astype(np.int64).sum())


def cone_entry(img: np.ndarray, r: int, c: int, power: int = 1) -> int:
    H, W = img.shape
    tot = 0
    for y in range(0, min(r, H - 1) + 1):
        d = r - y
        lo, hi = max(0, c - d), min(W - 1, c + d)
        if lo <= hi:
            tot += int((img[y, lo:hi + 1].astype(np.int64) ** power).sum())
    return tot


def square_mask(H: int, W: int, y: int, x: int, n: int) -> np.ndarray:
    m = np.zeros((H, W), np.int64)
    m[y - n + 1:y + n + 1, x - n + 1:x + n + 1] = 1
    return m


def diamond_mask(H: int, W: int, y: int, x: int, h: int) -> np.ndarray:
    m = np.zeros((H, W), np.int64)
    for xx in range(x - h + 1, x + h):
        d = abs(xx - x)
        m[y - h + d + 1:y + h - d + 1, xx] = 1
    return m


def star_weights(H: int, W: int, y: int, x: int, n: int, h: int) -> np.ndarray:
    """Per-pixel weight of the star: 1 in square or diamond only, 2 in both."""
    return square_mask(H, W, y, x, n) + diamond_mask(H, W, y, x, h)


def star_sums(img: np.ndarray, y: int, x: int, n: int, h: int):
    """(S, Q, area) of the star by direct weighted pixel sums."""
    H, W = img.shape
    w = star_weights(H, W, y, x, n, h)
    v = img.astype(np.int64)
    return int((w * v).sum()), int((w * v * v).sum()), int(w.sum())
