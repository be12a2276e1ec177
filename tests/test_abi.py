"""The C-ABI library builds, loads and exports every symbol include/ov.h declares (CPU only;
no compute calls)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    txt = (ROOT / "include" / "ov.h").read_text()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ov_[a-z0-9_A-Z]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def so_path():
    from paper_2204_01583_gb300.build import build

    return build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ov_set_gauge", "ov_apply_HW", "ov_sgn_HW_apply", "ov_overlap_apply", "ov_overlap_vjp"):
        assert must in names


def test_library_exports_every_declared_symbol(so_path):
    lib = ctypes.CDLL(str(so_path))
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol(so_path):
    from paper_2204_01583_gb300 import lib as binding

    assert sorted(binding.EXPORTS) == _declared()


def test_version_string(so_path):
    lib = ctypes.CDLL(str(so_path))
    lib.ov_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.ov_version()


def test_null_context_is_rejected_without_a_gpu(so_path):
    lib = ctypes.CDLL(str(so_path))
    lib.ov_destroy.argtypes = [ctypes.c_void_p]
    assert lib.ov_destroy(None) == 0
    lib.ov_set_contour_ellipse.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int]
    assert lib.ov_set_contour_ellipse(None, 8, 1.0, 1.0, 0.3, 0) == 1
