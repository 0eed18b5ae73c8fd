"""Python binding of libscreen.so -- argument marshalling only.

Every function here has the name of the C-ABI entry point it calls (see
include/screen.h); all computation happens in the library's CUDA kernels.
PyTorch supplies device memory (tensors) and streams.  There is no CPU
fallback: importing works without a GPU, but every call that needs the device
raises ScreenError when the library or the device is unavailable.
"""
from __future__ import annotations

import ctypes
import os
from fractions import Fraction

import numpy as np

from . import _build

F_MEAN, F_VAR, F_GRAD, F_PREWITT = 1, 2, 4, 8
SCR_OK, SCR_EINVAL, SCR_ENOMEM, SCR_EBUDGET, SCR_ECUDA, SCR_ETIMEOUT, SCR_EOVERFLOW = 0, -1, -2, -3, -4, -5, -6
SCR_EEVICTED, SCR_EUNSUPPORTED = -7, -8
SERVE_BATCHED, SERVE_PLAIN = 0, 1
MAX_SCALES = 32


class ScreenError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class _Rat(ctypes.Structure):
    _fields_ = [("num", ctypes.c_int64), ("den", ctypes.c_int64)]


class _Params(ctypes.Structure):
    _fields_ = [("n_scales", ctypes.c_int32), ("radii", ctypes.POINTER(ctypes.c_int32)),
                ("features", ctypes.c_uint32), ("mean_rel", _Rat), ("std_rel", _Rat),
                ("grad_rel", _Rat), ("grad_abs", _Rat), ("prewitt_rel", _Rat), ("prewitt_abs", _Rat)]


class _Bounds(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("S_lo", "S_hi", "V_lo", "V_hi", "N_lo", "N_hi")]


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("kernel_launches", "bytes_in_use", "bytes_peak", "budget")]


class _Pair(ctypes.Structure):
    _fields_ = [("image", ctypes.c_int32), ("tmpl", ctypes.c_int32)]


class _Tuning(ctypes.Structure):
    _fields_ = [("words_per_warp", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int64), ("n_records", ctypes.c_int64), ("n_units", ctypes.c_int64),
                ("candidates", ctypes.c_uint64), ("words_per_warp", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("union_words", ctypes.c_uint64),
                ("sort_passes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None

class _Joint(ctypes.Structure):
    _fields_ = [("n_areas", ctypes.c_int32), ("area_radii", ctypes.POINTER(ctypes.c_int32)),
                ("band", (ctypes.c_int32 * 2) * 3), ("q", _Rat * 3)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("table_budget_bytes", ctypes.c_uint64), ("sum_bits", ctypes.c_int32), ("sq_bits", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("start_held", ctypes.c_int32),
                ("small_log2", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("count", ctypes.c_uint64),
                ("arrival_ns", ctypes.c_int64), ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("batch", ctypes.c_uint64), ("batch_size", ctypes.c_int32), ("built", ctypes.c_int32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "requests", "batches", "uploads", "screens", "builds", "rebuilds", "evictions", "resident_images",
        "resident_bytes", "peak_resident_bytes", "mask_bytes", "launches", "build_ns", "build_copy_ns", "build_alloc_ns", "build_run_ns", "build_gpu_ns", "screen_ns", "plan_ns",
        "wait_ns", "copy_ns")]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libscreen.so (building it first if asked and stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ScreenError(SCR_ECUDA, f"libscreen.so missing at {_build.LIB}; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    vp, i32, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "screen_init": ([pp, ctypes.c_int, u64], ctypes.c_int),
        "screen_shutdown": ([vp], None),
        "screen_last_error": ([], ctypes.c_char_p),
        "screen_stats": ([vp, ctypes.POINTER(_Stats)], ctypes.c_int),
        "build_tables": ([vp, vp, i32, i32, i64, i32, i32, vp, pp], ctypes.c_int),
        "screen_set_filter": ([vp, i32, vp], ctypes.c_int),
        "screen_filter_windows": ([vp, ctypes.POINTER(_Params), i32, vp, ctypes.POINTER(i32)], ctypes.c_int),
        "screen_filter_plan": ([vp, vp, ctypes.POINTER(_Params), vp], ctypes.c_int),
        "tables_view": ([vp, ctypes.c_int, pp] + [ctypes.POINTER(i64)] * 5 + [ctypes.POINTER(i32)], ctypes.c_int),
        "tables_copy_to_host": ([vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "build_moment_tables": ([vp, vp, i32, i32, i64, vp, vp], ctypes.c_int),
        "tables_release": ([vp, vp], None),
        "template_features": ([vp, vp, i32, i32, i32, u32, pp], ctypes.c_int),
        "template_sums": ([vp, i32, ctypes.POINTER(i64)], ctypes.c_int),
        "template_release": ([vp, vp], None),
        "screen_bounds": ([vp, ctypes.POINTER(_Params), ctypes.POINTER(_Bounds)], ctypes.c_int),
        "screen_features": ([vp, vp, vp, ctypes.POINTER(_Params), vp, u64, vp], ctypes.c_int),
        "screen_joint": ([vp, vp, vp, ctypes.POINTER(_Params), ctypes.POINTER(_Joint), vp, u64, vp], ctypes.c_int),
        "compact_mask": ([vp, vp, i32, i32, i32, vp, u64, vp, vp], ctypes.c_int),
        "compact_mask_noalloc": ([vp, i32, i32, i32, vp, u64, vp, vp], ctypes.c_int),
        "compact_mask_noalloc_error": ([], ctypes.c_char_p),
        "screen_positions": ([vp, vp, vp, ctypes.POINTER(_Params), vp, u64, vp, u64, ctypes.POINTER(u64), vp],
                             ctypes.c_int),
        "screen_positions_async": ([vp, vp, vp, ctypes.POINTER(_Params), vp, u64, vp, u64, vp, vp], ctypes.c_int),
        "screen_host": ([vp, vp, i32, i32, i64, i32, i32, vp, ctypes.POINTER(_Params), vp, u64,
                         ctypes.POINTER(u64), vp], ctypes.c_int),
        "frames_create": ([vp, i32, i32, i32, i32, vp, ctypes.POINTER(_Params), u64, i32, pp], ctypes.c_int),
        "frames_submit": ([vp, vp, i64, vp, ctypes.POINTER(i64)], ctypes.c_int),
        "frames_wait": ([vp, i64, ctypes.POINTER(u64)], ctypes.c_int),
        "frames_destroy": ([vp], None),
        "screen_batch_create": ([vp, vp, i32, vp, ctypes.POINTER(_Params), i32, ctypes.POINTER(_Pair), i32,
                                 vp, vp, vp, vp, u64, vp, ctypes.POINTER(_Tuning), vp, pp], ctypes.c_int),
        "screen_batch_run": ([vp, vp], ctypes.c_int),
        "screen_batch_info": ([vp, ctypes.POINTER(_BatchInfo)], ctypes.c_int),
        "screen_batch_release": ([vp, vp], None),
        "server_clock_ns": ([], i64),
        "server_create": ([vp, ctypes.POINTER(_ServerConfig), pp], ctypes.c_int),
        "server_upload": ([vp, vp, i32, i32, i64, i32, i64, ctypes.POINTER(i64), ctypes.POINTER(u64)], ctypes.c_int),
        "server_screen": ([vp, i64, vp, ctypes.POINTER(_Params), vp, u64, i64, ctypes.POINTER(u64)], ctypes.c_int),
        "server_evict": ([vp, i64, ctypes.POINTER(u64)], ctypes.c_int),
        "server_forget": ([vp, i64], ctypes.c_int),
        "server_wait": ([vp, u64, i64, ctypes.POINTER(_RequestResult)], ctypes.c_int),
        "server_next": ([vp, i64, ctypes.POINTER(u64), ctypes.POINTER(_RequestResult)], ctypes.c_int),
        "server_hold": ([vp, i32], ctypes.c_int),
        "server_resident": ([vp, i64, ctypes.POINTER(i32)], ctypes.c_int),
        "server_stats": ([vp, ctypes.POINTER(_ServerStats)], ctypes.c_int),
        "server_destroy": ([vp], None),
        "server_lru_victims": ([vp, vp, vp, i32, u64, u64, u64, vp, ctypes.POINTER(i32)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def exported_symbols():
    return ["screen_init", "screen_shutdown", "screen_last_error", "screen_stats", "build_tables",
            "screen_set_filter", "screen_filter_windows", "screen_filter_plan",
            "tables_view", "tables_copy_to_host", "build_moment_tables", "tables_release", "template_features",
            "template_sums",
            "template_release", "screen_bounds", "screen_features", "screen_joint", "compact_mask",
            "compact_mask_noalloc",
            "compact_mask_noalloc_error", "screen_positions",
            "screen_positions_async", "screen_host", "frames_create", "frames_submit", "frames_wait",
            "frames_destroy", "screen_batch_create", "screen_batch_run",
            "screen_batch_info", "screen_batch_release", "server_clock_ns", "server_create", "server_upload",
            "server_screen", "server_evict", "server_forget", "server_wait", "server_next", "server_hold", "server_resident",
            "server_stats", "server_destroy", "server_lru_victims"]


def _check(rc: int, allow=()):
    if rc != SCR_OK and rc not in allow:
        msg = load().screen_last_error()
        raise ScreenError(rc, msg.decode() if msg else "")
    return rc


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


def _rat(v) -> _Rat:
    f = Fraction(v)
    return _Rat(f.numerator, f.denominator)


class Params:
    """scr_params: radii per scale, feature bits and the four tolerances."""

    def __init__(self, radii, features, mean_rel=Fraction(1, 20), std_rel=Fraction(1, 10),
                 grad_rel=Fraction(1, 10), grad_abs=Fraction(4), prewitt_rel=Fraction(1, 10),
                 prewitt_abs=Fraction(2)):
        self.radii = np.ascontiguousarray(radii, dtype=np.int32)
        self.c = _Params(len(self.radii), self.radii.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         int(features), _rat(mean_rel), _rat(std_rel), _rat(grad_rel), _rat(grad_abs),
                         _rat(prewitt_rel), _rat(prewitt_abs))

    @property
    def n_scales(self):
        return len(self.radii)


# ---- context ----------------------------------------------------------------

def screen_init(device: int = 0, hbm_budget_bytes: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().screen_init(ctypes.byref(ctx), device, hbm_budget_bytes))
    return ctx


def screen_shutdown(ctx) -> None:
    load().screen_shutdown(ctx)


def screen_last_error() -> str:
    return load().screen_last_error().decode()


def screen_stats(ctx) -> dict:
    s = _Stats()
    _check(load().screen_stats(ctx, ctypes.byref(s)))
    return {n: int(getattr(s, n)) for n, _ in _Stats._fields_}


# ---- tables -----------------------------------------------------------------

def build_tables(ctx, img, sum_bits: int = 32, sq_bits: int = 64, stream=None, H=None, W=None, pitch=None):
    """img: 2-D uint8 CUDA tensor (row pitch from its stride)."""
    if H is None:
        H, W = img.shape
        pitch = img.stride(0)
    out = ctypes.c_void_p()
    _check(load().build_tables(ctx, _ptr(img), H, W, pitch, sum_bits, sq_bits, _stream(stream), ctypes.byref(out)))
    return out


def screen_set_filter(ctx, windows) -> None:
    """Packed filter windows [(kS, kQ), ...] (0..2 pairs) for the context's later
    single-image table builds (build_tables, screen_host, frames_create); [] turns them off."""
    arr = np.ascontiguousarray(np.array(list(windows), dtype=np.int32).reshape(-1))
    _check(load().screen_set_filter(ctx, len(arr) // 2, _ptr(arr) if len(arr) else ctypes.c_void_p(0)))


def screen_filter_windows(tm, params: "Params", max_windows: int = 2):
    """Suggested packed filter windows [(kS, kQ), ...] for template tm and params."""
    out = (ctypes.c_int32 * 4)()
    n = ctypes.c_int32()
    _check(load().screen_filter_windows(tm, ctypes.byref(params.c), max_windows, out, ctypes.byref(n)))
    return [(int(out[2 * i]), int(out[2 * i + 1])) for i in range(n.value)]


def screen_filter_plan(tables, tm, params: "Params"):
    """Per scale, the packed window a screen would use (-1: exact corners only)."""
    out = np.empty(params.n_scales, np.int32)
    _check(load().screen_filter_plan(tables, tm, ctypes.byref(params.c), _ptr(out)))
    return [int(v) for v in out]


def tables_view(tables, which: int) -> dict:
    p = ctypes.c_void_p()
    v = [ctypes.c_int64() for _ in range(5)]
    bits = ctypes.c_int32()
    _check(load().tables_view(tables, which, ctypes.byref(p), *[ctypes.byref(x) for x in v], ctypes.byref(bits)))
    return dict(ptr=p.value, rows=v[0].value, cols=v[1].value, pitch=v[2].value, offset=v[3].value,
                plane_stride=v[4].value, bits=bits.value)


def build_moment_tables(ctx, tables, img, stream=None) -> None:
    """Add the Prewitt moment tables to `tables` (img: the same 2-D uint8 CUDA tensor)."""
    H, W = img.shape
    _check(load().build_moment_tables(ctx, _ptr(img), H, W, img.stride(0), tables, _stream(stream)))


def tables_copy_to_host(ctx, tables, which: int) -> np.ndarray:
    """which 0..3: L1, L2, T1, T2; 4, 5: the moment tables Mx, My ((H+1) x (W+1));
    6 + 2w, 7 + 2w: the upright and cone packed filter planes of window w."""
    if which in (4, 5):
        v = tables_view(tables, 0)            # the upright table's (H + 1) x (W + 1)
        out = np.empty((v["rows"], v["cols"]), np.uint64)
        _check(load().tables_copy_to_host(ctx, tables, which, _ptr(out)))
        return out
    v = tables_view(tables, which)
    out = np.empty((v["rows"], v["cols"]), np.uint64)
    _check(load().tables_copy_to_host(ctx, tables, which, _ptr(out)))
    return out


def tables_release(ctx, tables) -> None:
    load().tables_release(ctx, tables)


# ---- template ---------------------------------------------------------------

def template_features(ctx, tmpl: np.ndarray, r: int, t_min: int, features: int):
    tmpl = np.ascontiguousarray(tmpl, dtype=np.uint8)
    out = ctypes.c_void_p()
    _check(load().template_features(ctx, _ptr(tmpl), tmpl.shape[0], r, t_min, features, ctypes.byref(out)))
    return out


def template_sums(tm, t: int):
    out = (ctypes.c_int64 * 3)()
    _check(load().template_sums(tm, t, out))
    return int(out[0]), int(out[1]), int(out[2])


def template_release(ctx, tm) -> None:
    load().template_release(ctx, tm)


def screen_bounds(tm, params: Params) -> np.ndarray:
    out = (_Bounds * params.n_scales)()
    _check(load().screen_bounds(tm, ctypes.byref(params.c), out))
    return np.array([[getattr(b, n) for n, _ in _Bounds._fields_] for b in out], np.int64)


# ---- screening --------------------------------------------------------------

def mask_words(n_scales: int, H: int, W: int) -> int:
    return n_scales * H * ((W + 31) // 32)


def screen_features(ctx, tables, tm, params: Params, mask, stream=None) -> None:
    _check(load().screen_features(ctx, tables, tm, ctypes.byref(params.c), _ptr(mask), mask.numel(),
                                  _stream(stream)))


def screen_joint(ctx, tables, tm, params: Params, area_radii, bands, q, mask, stream=None) -> None:
    """Joint membership screen: area_radii [n_scales][n_areas] ints, bands
    [(t_lo, t_hi)] per area, q (mean, std, contrast) quantisation factors."""
    ar = np.ascontiguousarray(area_radii, dtype=np.int32)
    n_areas = len(bands)
    assert ar.shape == (params.n_scales, n_areas)
    j = _Joint()
    j.n_areas = n_areas
    j.area_radii = ar.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    for k, (lo, hi) in enumerate(bands):
        j.band[k][0], j.band[k][1] = int(lo), int(hi)
    for k in range(3):
        j.q[k] = _rat(q[k])
    _check(load().screen_joint(ctx, tables, tm, ctypes.byref(params.c), ctypes.byref(j), _ptr(mask), mask.numel(),
                               _stream(stream)))


def compact_mask(ctx, mask, n_scales, H, W, lst, count, stream=None) -> None:
    cap = 0 if lst is None else lst.numel()
    _check(load().compact_mask(ctx, _ptr(mask), n_scales, H, W, _ptr(lst), cap, _ptr(count), _stream(stream)))


def compact_mask_noalloc(mask, n_scales, H, W, lst, count, stream=None) -> None:
    """compact_mask without device allocation: scratch is a fixed array in the
    library (callers inside stream capture or without an allocator)."""
    cap = 0 if lst is None else lst.numel()
    rc = load().compact_mask_noalloc(_ptr(mask), n_scales, H, W, _ptr(lst), cap, _ptr(count), _stream(stream))
    if rc != SCR_OK:
        raise ScreenError(rc, compact_mask_noalloc_error())


def compact_mask_noalloc_error() -> str:
    return load().compact_mask_noalloc_error().decode()


def screen_positions(ctx, tables, tm, params: Params, mask, lst, stream=None) -> tuple[int, bool]:
    """Returns (survivor count, overflowed)."""
    n = ctypes.c_uint64()
    cap = 0 if lst is None else lst.numel()
    rc = _check(load().screen_positions(ctx, tables, tm, ctypes.byref(params.c), _ptr(mask), mask.numel(),
                                        _ptr(lst), cap, ctypes.byref(n), _stream(stream)), allow=(SCR_EOVERFLOW,))
    return int(n.value), rc == SCR_EOVERFLOW


def screen_positions_async(ctx, tables, tm, params: Params, mask, lst, count, stream=None) -> None:
    cap = 0 if lst is None else lst.numel()
    _check(load().screen_positions_async(ctx, tables, tm, ctypes.byref(params.c), _ptr(mask), mask.numel(),
                                         _ptr(lst), cap, _ptr(count), _stream(stream)))


def screen_host(ctx, img: np.ndarray, sum_bits: int, sq_bits: int, tm, params: Params, lst: np.ndarray,
                stream=None) -> tuple[int, bool]:
    """img and lst are host arrays (pinned memory makes the copies asynchronous)."""
    n = ctypes.c_uint64()
    H, W = img.shape
    rc = _check(load().screen_host(ctx, _ptr(img), H, W, img.strides[0], sum_bits, sq_bits, tm,
                                   ctypes.byref(params.c), _ptr(lst), 0 if lst is None else lst.size,
                                   ctypes.byref(n), _stream(stream)), allow=(SCR_EOVERFLOW,))
    return int(n.value), rc == SCR_EOVERFLOW


# ---- a stream of same-sized host images -------------------------------------

def frames_create(ctx, H: int, W: int, sum_bits: int, sq_bits: int, tm, params: Params, list_cap: int,
                  depth: int = 2):
    out = ctypes.c_void_p()
    _check(load().frames_create(ctx, H, W, sum_bits, sq_bits, tm, ctypes.byref(params.c), list_cap, depth,
                                ctypes.byref(out)))
    return out


def frames_submit(f, img, lst) -> int:
    """img: H x W uint8 host array (pinned for an asynchronous copy); lst:
    pinned host array of at least list_cap uint64/int64 keys, or None when
    list_cap is 0.  Returns the frame's ticket."""
    t = ctypes.c_int64()
    pitch = img.strides[0] if isinstance(img, np.ndarray) else img.stride(0)
    _check(load().frames_submit(f, _ptr(img), pitch, _ptr(lst), ctypes.byref(t)))
    return int(t.value)


def frames_wait(f, ticket: int) -> tuple[int, bool]:
    n = ctypes.c_uint64()
    rc = _check(load().frames_wait(f, ticket, ctypes.byref(n)), allow=(SCR_EOVERFLOW,))
    return int(n.value), rc == SCR_EOVERFLOW


def frames_destroy(f) -> None:
    load().frames_destroy(f)


# ---- batched screening ------------------------------------------------------

def screen_batch_create(ctx, tables, tmpls, params, pairs, counts, keys, n_keys, offsets=None, union_mask=None,
                        tuning=None, stream=None):
    """tables, tmpls, params: lists (one params per template); pairs: list of
    (image, template) indices.  Output tensors are caller-owned CUDA tensors."""
    nt = len(tmpls)
    tab_arr = (ctypes.c_void_p * len(tables))(*[t.value if hasattr(t, "value") else t for t in tables])
    tm_arr = (ctypes.c_void_p * nt)(*[t.value if hasattr(t, "value") else t for t in tmpls])
    par_arr = (_Params * nt)(*[p.c for p in params])
    pr_arr = (_Pair * len(pairs))(*[_Pair(int(i), int(t)) for (i, t) in pairs])
    tun = None if tuning is None else ctypes.byref(_Tuning(int(tuning[0]), int(tuning[1])))
    out = ctypes.c_void_p()
    _check(load().screen_batch_create(ctx, tab_arr, len(tables), tm_arr, par_arr, nt, pr_arr, len(pairs),
                                      _ptr(counts), _ptr(offsets), _ptr(union_mask), _ptr(keys),
                                      0 if keys is None else keys.numel(), _ptr(n_keys), tun, _stream(stream),
                                      ctypes.byref(out)))
    return out


def screen_batch_run(b, stream=None) -> None:
    _check(load().screen_batch_run(b, _stream(stream)))


def screen_batch_info(b) -> dict:
    info = _BatchInfo()
    _check(load().screen_batch_info(b, ctypes.byref(info)))
    return {n: int(getattr(info, n)) for n, _ in _BatchInfo._fields_}


def screen_batch_release(ctx, b) -> None:
    load().screen_batch_release(ctx, b)


# ---- serving loop -------------------------------------------------------------

def server_clock_ns() -> int:
    return int(load().server_clock_ns())


def server_create(ctx, table_budget_bytes: int = 0, sum_bits: int = 32, sq_bits: int = 64, mode: int = SERVE_BATCHED,
                  max_batch: int = 0, start_held: bool = False, small_log2: int = 0, max_inflight: int = 0):
    cfg = _ServerConfig(table_budget_bytes, sum_bits, sq_bits, mode, max_batch, int(start_held), small_log2,
                        max_inflight, 0)
    s = ctypes.c_void_p()
    _check(load().server_create(ctx, ctypes.byref(cfg), ctypes.byref(s)))
    return s


def server_upload(s, img: np.ndarray, borrow: bool = False, arrival_ns: int = 0) -> tuple[int, int]:
    """Queue an upload of a uint8 H x W array; returns (image_id, request_id).
    With borrow the caller keeps img alive until the image is forgotten."""
    assert img.dtype == np.uint8 and img.ndim == 2 and img.strides[1] == 1
    iid, rid = ctypes.c_int64(), ctypes.c_uint64()
    _check(load().server_upload(s, img.ctypes.data, img.shape[0], img.shape[1], img.strides[0], int(borrow),
                                arrival_ns, ctypes.byref(iid), ctypes.byref(rid)))
    return iid.value, rid.value


def server_screen(s, image_id: int, tm, params: Params, lst: np.ndarray | None = None, arrival_ns: int = 0) -> int:
    """Queue a screen; lst (uint64 host array or None) receives the first len(lst) keys."""
    cap = 0 if lst is None else len(lst)
    ptr = None if lst is None else lst.ctypes.data
    if lst is not None:
        assert lst.dtype == np.uint64 and lst.flags.c_contiguous
    rid = ctypes.c_uint64()
    _check(load().server_screen(s, image_id, tm, ctypes.byref(params.c), ptr, cap, arrival_ns, ctypes.byref(rid)))
    return rid.value


def server_evict(s, image_id: int) -> int:
    rid = ctypes.c_uint64()
    _check(load().server_evict(s, image_id, ctypes.byref(rid)))
    return rid.value


def server_forget(s, image_id: int) -> None:
    _check(load().server_forget(s, image_id))


def server_wait(s, request_id: int, timeout_us: int = 300_000_000) -> dict:
    res = _RequestResult()
    _check(load().server_wait(s, request_id, timeout_us, ctypes.byref(res)))
    return {n: int(getattr(res, n)) for n, _ in _RequestResult._fields_}


def server_next(s, timeout_us: int = 300_000_000) -> tuple[int, dict]:
    """The next completed, uncollected request (completion order): (request_id, result)."""
    res, rid = _RequestResult(), ctypes.c_uint64()
    _check(load().server_next(s, timeout_us, ctypes.byref(rid), ctypes.byref(res)))
    return rid.value, {n: int(getattr(res, n)) for n, _ in _RequestResult._fields_}


def server_hold(s, hold: bool) -> None:
    _check(load().server_hold(s, int(hold)))


def server_resident(s, image_id: int) -> bool:
    r = ctypes.c_int32()
    _check(load().server_resident(s, image_id, ctypes.byref(r)))
    return bool(r.value)


def server_stats(s) -> dict:
    st = _ServerStats()
    _check(load().server_stats(s, ctypes.byref(st)))
    return {n: int(getattr(st, n)) for n, _ in _ServerStats._fields_}


def server_destroy(s) -> None:
    load().server_destroy(s)


def server_lru_victims(nbytes, last_use, pinned, resident: int, budget: int, need: int) -> list[int]:
    """The serving loop's eviction choice (pure host code); raises ScreenError(SCR_EBUDGET) when nothing fits."""
    b = np.ascontiguousarray(nbytes, dtype=np.uint64)
    lu = np.ascontiguousarray(last_use, dtype=np.uint64)
    pn = np.ascontiguousarray(pinned, dtype=np.int32)
    n = len(b)
    out = np.zeros(max(n, 1), dtype=np.int32)
    nv = ctypes.c_int32()
    _check(load().server_lru_victims(b.ctypes.data, lu.ctypes.data, pn.ctypes.data, n, resident, budget, need,
                                     out.ctypes.data, ctypes.byref(nv)))
    return [int(v) for v in out[:nv.value]]


__all__ = [n for n in dir() if not n.startswith("_")]
