"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point declared in include/aqmp.h, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_09190_gb300 import aqmp, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return aqmp.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "aqmp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aqmp_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(aqmp.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_defaults(lib):
    assert "sm_103a" in aqmp.aqmp_version()
    p = aqmp.default_params()
    assert (p.rmse_tol, p.cap_num, p.cap_den, p.min_block, p.max_block, p.dict_id) == (2.0, 1, 4, 4, 64, 0)


@pytest.mark.parametrize("b,d,m", [(4, 0, 32), (8, 1, 64), (16, 2, 256), (64, 0, 8192)])
def test_num_atoms(lib, b, d, m):
    assert aqmp.aqmp_num_atoms(b, d) == m


def test_num_atoms_rejects_bad_side(lib):
    assert lib.aqmp_num_atoms(12, 0) == -1


def _encode_rc(lib, params, planes):
    arr = (aqmp.aqmp_plane * len(planes))(*planes)
    out = ctypes.c_void_p()
    rc = lib.aqmp_encode_planes(ctypes.byref(params), arr, len(planes), None, ctypes.byref(out))
    return rc, out.value


@pytest.mark.parametrize("field,value,code", [
    ("min_block", 3, -1), ("max_block", 48, -1), ("min_block", 128, -1),
    ("cap_den", 0, -1), ("cap_num", 5, -1), ("rmse_tol", -1.0, -1),
    ("dict_id", 7, -3), ("max_block", 256, -8), ("precision", 9, -8)])
def test_bad_parameters_are_rejected_before_any_device_work(lib, field, value, code):
    img = np.zeros((64, 64), np.uint8)
    p = aqmp.default_params()
    setattr(p, field, value)
    rc, out = _encode_rc(lib, p, [aqmp.aqmp_plane(img.ctypes.data, 64, 64, 64, -1.0)])
    assert rc == code and not out
    assert lib.aqmp_last_error()


def test_shape_not_multiple_of_root_is_rejected(lib):
    img = np.zeros((64, 96), np.uint8)
    rc, out = _encode_rc(lib, aqmp.default_params(), [aqmp.aqmp_plane(img.ctypes.data, 64, 96, 96, -1.0)])
    assert rc == -2 and not out
    assert b"multiple of max_block" in lib.aqmp_last_error()


def test_null_and_empty_inputs_are_rejected(lib):
    p = aqmp.default_params()
    rc, _ = _encode_rc(lib, p, [aqmp.aqmp_plane(None, 64, 64, 64, -1.0)])
    assert rc == -1
    out = ctypes.c_void_p()
    assert lib.aqmp_encode_planes(ctypes.byref(p), None, 0, None, ctypes.byref(out)) == -1
    assert lib.aqmp_correlate(12, 0, None, 4, None, 0, None) == -1
    assert lib.aqmp_correlate(8, 5, None, 4, None, 0, None) == -3
    assert lib.aqmp_correlate(64, 0, None, 0, None, 7, None) == -1      # no such mode
    assert lib.aqmp_last_device_ms(None) == -1
    assert lib.aqmp_correlate(32, 0, None, 0, None, 6, None) == -8      # tensor cores for every family: side 64 only
