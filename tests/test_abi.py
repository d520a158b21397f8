"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
symbol include/fkt.h declares, and rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2106_04487_gb300 import build, fkt

    build.build()
    return fkt.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "fkt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fkt_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fkt_plan", "fkt_mvm", "fkt_mvm_host", "fkt_destroy", "fkt_error_string"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_lists_every_export():
    from paper_2106_04487_gb300 import fkt

    assert sorted(fkt.EXPORTS) == sorted(_declared())


def test_error_strings(L):
    from paper_2106_04487_gb300 import fkt

    assert fkt.fkt_error_string(0) == "ok"
    assert "invalid" in fkt.fkt_error_string(1)
    assert fkt.fkt_error_string(99) == "unknown status"


def test_invalid_arguments_rejected_on_host(L):
    from paper_2106_04487_gb300 import fkt

    h = ctypes.c_void_p()
    k = fkt.make_kernel("gaussian", 0.1)
    dummy = ctypes.c_void_p(0x1000)
    # N = 0, d = 2, p too large, theta out of range, leaf_size 0, null output, bad kernel
    assert L.fkt_plan(dummy, 0, 3, k, 4, 64, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_plan(dummy, 10, 2, k, 4, 64, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_plan(dummy, 10, 3, k, 11, 64, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_plan(dummy, 10, 4, k, 9, 64, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_plan(dummy, 10, 3, k, 4, 64, 1.0, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_plan(dummy, 10, 3, k, 4, 0, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_plan(dummy, 10, 3, k, 4, 64, 0.5, None, None) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_plan(None, 10, 3, k, 4, 64, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    bad = fkt.make_kernel("gaussian", -1.0)
    assert L.fkt_plan(dummy, 10, 3, bad, 4, 64, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    bad = fkt.fkt_kernel(42, 1.0, 1.0, 1.0)
    assert L.fkt_plan(dummy, 10, 3, bad, 4, 64, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    rq = fkt.make_kernel("ratquad", 0.2, alpha=0.0)
    assert L.fkt_plan(dummy, 10, 3, rq, 4, 64, 0.5, None, ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    # calls on a null plan
    assert L.fkt_mvm(None, dummy, dummy, 1) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_mvm_host(None, dummy, dummy, 1) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_dense_mvm(None, dummy, dummy, 1) == fkt.FKT_ERR_INVALID_ARG
    assert L.fkt_set_option(None, b"timing", b"1") == fkt.FKT_ERR_INVALID_ARG
    st = fkt.fkt_stats()
    assert L.fkt_plan_stats(None, ctypes.byref(st)) == fkt.FKT_ERR_INVALID_ARG
    L.fkt_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2106_04487_gb300 import fkt

    monkeypatch.setattr(fkt, "_LIB", None)
    monkeypatch.setattr(fkt, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        fkt.lib()
