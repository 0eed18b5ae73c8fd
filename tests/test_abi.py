"""The C-ABI library builds, loads, and exports every entry point include/screen.h
declares; the Python binding marshals the same names.  No compute call is made."""
import ctypes
import os
import re

import pytest

import paper_1707_05647_gb300 as scr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "screen.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|int64_t|void|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("screen_init", "build_tables", "template_features", "screen_positions"):
        assert n in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(scr._build.build())
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    assert sorted(scr.exported_symbols()) == _declared()
    for n in _declared():
        assert callable(getattr(scr, n)), n


def test_nvcc_builds_for_sm103a_only():
    from paper_1707_05647_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(scr.ScreenError) as e:
        scr.screen_init(0, 0)
    assert e.value.code in (scr.SCR_ECUDA, scr.SCR_EINVAL)
    assert scr.screen_last_error()


def test_bad_handles_rejected_without_device():
    lib = scr.load()
    out = ctypes.c_void_p()
    assert lib.build_tables(None, None, 4, 4, 4, 32, 32, None, ctypes.byref(out)) == scr.SCR_EINVAL
    assert lib.template_sums(None, 3, (ctypes.c_int64 * 3)()) == scr.SCR_EINVAL
    p = scr.Params([5, 6], 7)
    assert lib.screen_bounds(None, ctypes.byref(p.c), None) == scr.SCR_EINVAL
