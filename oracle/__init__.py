"""CPU oracle for the screening path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
arm may import this package.  The CUDA library and its Python binding never
import it, and it imports nothing from them.

Layers (each cites the passage it follows; the paper is arXiv 1707.05647):
  * screen_oracle.c  -- exact uint64 tables and the per-candidate screening loop
                        (Sec. 3 Eq. T_1 / S_1 / S_sigma, Sec. 4 diamond table and
                        octagonal star, Sec. 5 Algorithm 1).
  * bounds.py        -- template feature hulls over the scale band (Sec. 5,
                        Eq. F_n) and the inclusive integer bounds, in exact
                        rationals (fractions.Fraction).
  * brute.py         -- direct pixel-set sums (no tables) used to pin the above.

Parity status: every function here is pinned by tests under tests/ against
brute-force pixel sums, numpy's cumulative sums, closed forms or the exact
rational definition; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .bounds import ScaleBounds, scale_bounds, star_geometry, template_hulls  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "screen_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C part with gcc (OpenMP over rows)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_square_half.argtypes = [ctypes.c_int]
            L.orc_square_half.restype = ctypes.c_int
            L.orc_upright.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, u64p, u64p]
            L.orc_cone.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, u64p, u64p]
            L.orc_features_at.argtypes = [u64p, u64p, u64p, u64p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int64, i32p, i32p, i64p]
            L.orc_screen.argtypes = [u64p, u64p, u64p, u64p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, i32p, i64p, ctypes.c_uint, u32p, u64p,
                                     ctypes.c_int64]
            L.orc_screen.restype = ctypes.c_int64
            L.orc_threads.argtypes = [ctypes.c_int]
            L.orc_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def threads(n: int = 0) -> int:
    """Set the screening loop's OpenMP thread count (n > 0); returns the count in effect."""
    return int(lib().orc_threads(int(n)))


def square_half(R: int) -> int:
    return int(lib().orc_square_half(int(R)))


def upright_tables(img: np.ndarray):
    """(L1, L2): exact uint64 (H+1) x (W+1) tables of I and I^2 (Sec. 3, Eq. T_1)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    L1 = np.empty((H + 1, W + 1), np.uint64)
    L2 = np.empty((H + 1, W + 1), np.uint64)
    lib().orc_upright(_p(img, ctypes.c_uint8), H, W, W, _p(L1, ctypes.c_uint64),
                      _p(L2, ctypes.c_uint64))
    return L1, L2


def cone_tables(img: np.ndarray):
    """(T1, T2): exact uint64 (H+1) x (W+2) cone tables, T[a][b] = cone(a-1, b-1) (Sec. 4)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    T1 = np.empty((H + 1, W + 2), np.uint64)
    T2 = np.empty((H + 1, W + 2), np.uint64)
    lib().orc_cone(_p(img, ctypes.c_uint8), H, W, W, _p(T1, ctypes.c_uint64),
                   _p(T2, ctypes.c_uint64))
    return T1, T2


class Tables:
    """The four exact tables of one image."""

    def __init__(self, img: np.ndarray):
        self.img = np.ascontiguousarray(img, dtype=np.uint8)
        self.H, self.W = self.img.shape
        self.L1, self.L2 = upright_tables(self.img)
        self.T1, self.T2 = cone_tables(self.img)

    def _args(self):
        u = ctypes.c_uint64
        return (_p(self.L1, u), _p(self.L2, u), _p(self.T1, u), _p(self.T2, u), self.H, self.W)

    def features_at(self, R: int, ys, xs) -> np.ndarray:
        """Rows of (S, Q, S_in, V, N, valid) for candidates (ys[i], xs[i]) at radius R."""
        ys = np.ascontiguousarray(ys, dtype=np.int32)
        xs = np.ascontiguousarray(xs, dtype=np.int32)
        out = np.zeros((len(ys), 6), np.int64)
        lib().orc_features_at(*self._args(), int(R), len(ys), _p(ys, ctypes.c_int32),
                              _p(xs, ctypes.c_int32), _p(out, ctypes.c_int64))
        return out

    def screen(self, radii, bounds: np.ndarray, features: int, cap: int | None = None):
        """Mask words (S, H, ceil(W/32)) uint32, key list, survivor count (Algorithm 1)."""
        radii = np.ascontiguousarray(radii, dtype=np.int32)
        bounds = np.ascontiguousarray(bounds, dtype=np.int64).reshape(len(radii), 6)
        S = len(radii)
        Ww = (self.W + 31) // 32
        mask = np.zeros((S, self.H, Ww), np.uint32)
        if cap is None:
            cap = S * self.H * self.W
        lst = np.zeros(max(1, min(cap, S * self.H * self.W)), np.uint64)
        cnt = lib().orc_screen(*self._args(), S, _p(radii, ctypes.c_int32),
                               _p(bounds, ctypes.c_int64), int(features),
                               _p(mask, ctypes.c_uint32), _p(lst, ctypes.c_uint64), len(lst))
        return mask, lst[:min(cnt, len(lst))].copy(), int(cnt)


def template_sums(tmpl: np.ndarray, r: int, t_min: int):
    """Per central radius t in [t_min, r]: (t, S_t, Q_t, S_in_t) of the template's
    central star at (r, r) (Sec. 5: features of the central areas)."""
    tb = Tables(tmpl)
    out = []
    for t in range(t_min, r + 1):
        f = tb.features_at(t, [r], [r])[0]
        assert f[5] == 1, "template star must lie inside the template"
        out.append((t, int(f[0]), int(f[1]), int(f[2])))
    return out


def screen_workload(img, tmpl, r, t_min, radii, features, tol, tables: Tables | None = None):
    """Whole oracle pipeline: template hulls -> per-scale bounds -> mask and list."""
    sums = template_sums(tmpl, r, t_min)
    hulls = template_hulls(sums, features)
    bnds = [scale_bounds(hulls, R, tol, features) for R in radii]
    barr = np.array([b.as_row() for b in bnds], np.int64)
    tb = tables if tables is not None else Tables(img)
    mask, lst, cnt = tb.screen(radii, barr, features)
    return dict(mask=mask, list=lst, count=cnt, bounds=barr, hulls=hulls, sums=sums, tables=tb)
