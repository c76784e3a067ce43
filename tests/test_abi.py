"""The C-ABI library loads and exports every entry point include/nh.h declares,
and the Python binding covers exactly those names (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nh.h")
LIB = os.path.join(ROOT, "paper_2204_01722_b300", "libnh.so")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:nh_status|const char\s*\*|int64_t)\s+(nh_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = declared()
    for n in ["nh_create", "nh_space_box", "nh_op_create", "nh_qdata_setup", "nh_residual",
              "nh_jacobian_apply", "nh_jacobian_diagonal", "nh_prolong", "nh_restrict", "nh_dot"]:
        assert n in names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2204_01722_b300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header(lib):
    from paper_2204_01722_b300 import nh
    assert sorted(nh.SIGNATURES) == declared()


def test_argument_errors_need_no_device(lib):
    """Null handles are rejected before any CUDA call."""
    from paper_2204_01722_b300 import nh
    assert nh.lib.nh_create(None, 0, None) == nh.NH_ERR_ARG
    assert nh.lib.nh_jacobian_apply(None, 0, None, None) == nh.NH_ERR_ARG
    assert nh.lib.nh_space_box(None, 1, 1, 1, None, 2, 3, None, None, None) == nh.NH_ERR_ARG
    assert nh.lib.nh_last_error(None) == b"null context"
