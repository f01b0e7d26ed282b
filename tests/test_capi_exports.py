"""The C-ABI library loads and exports every function include/clipverify.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "clipverify.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cv_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("cv_net_create", "cv_cache_build", "cv_cache_create", "cv_bound_batch", "cv_bound_batch_workspace"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2512_11087_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2512_11087_gb300 import capi
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError):
        capi.load()


def test_null_arguments_are_refused_without_a_launch():
    # host-side validation runs before any CUDA call, so this needs no GPU (raw calls, NULL stream)
    from paper_2512_11087_gb300 import capi
    lib = capi.load()
    opt = capi.cv_options_default()
    bi = capi.make_batch_in(4, None, None, 1, None, None)
    bo = capi.cv_batch_out()
    assert lib.cv_bound_batch(None, None, ctypes.byref(bi), ctypes.byref(bo), ctypes.byref(opt), None, 0,
                              None) == capi.CV_EINVAL
    code = ctypes.c_int(-1)
    assert lib.cv_batch_check(None, None, ctypes.byref(bi), ctypes.byref(code), None) == capi.CV_EINVAL
    assert code.value == 0
    bad = capi.cv_options_default()
    bad.relaxed = 7
    n = ctypes.c_size_t()
    assert lib.cv_bound_batch_workspace(None, None, ctypes.byref(bi), ctypes.byref(bad), ctypes.byref(n)) == \
        capi.CV_EINVAL
    assert lib.cv_last_error()
