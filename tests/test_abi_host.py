"""The C ABI library builds, loads and exports every symbol include/pointsht.h
declares; argument errors are reported on the host without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2312_12285_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pointsht.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pointsht_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS)


def test_version(lib):
    assert lib.pointsht_version().decode().count(".") == 2


def test_plan_create_rejects_bad_lmax_before_any_cuda_call(lib):
    h = ctypes.c_void_p()
    assert lib.pointsht_plan_create(0, ctypes.byref(h)) == _lib.EINVAL
    assert "lmax" in _lib.last_error()
    assert lib.pointsht_plan_create(100000, ctypes.byref(h)) == _lib.EINVAL
    assert lib.pointsht_plan_create(10, None) == _lib.EINVAL


def test_null_plan_and_bad_arguments(lib):
    arr, n = _lib.catalog_array([])
    assert lib.pointsht_alm(None, arr, 0, 1, _lib.FP32, None, None, 0, None) == _lib.EINVAL
    assert "plan" in _lib.last_error()
    assert lib.pointsht_workspace_size(None, arr, 0, 1, _lib.FP32) == 0
    assert lib.pointsht_plan_lmax(None) == -1
    assert lib.pointsht_plan_check(None) == _lib.EINVAL
    lib.pointsht_plan_destroy(None)
    assert lib.pointsht_cl(-1, None, 1, None, None, None) == _lib.EINVAL
    assert lib.pointsht_cl_backward(4, None, 1, None, None, None, None) == _lib.EINVAL
    assert lib.pointsht_bin(4, None, 1, None, 2, None, None) == _lib.EINVAL
    assert lib.pointsht_bin_backward(4, None, 1, None, 2, None, None) == _lib.EINVAL
    assert lib.pointsht_combine(4, None, 1, None, 1, None, None, None, None) == _lib.EINVAL
    assert lib.pointsht_shot_noise(arr, 0, 0, _lib.FP32, None, None, 0, None) == _lib.EINVAL
    assert lib.pointsht_alm_backward(None, arr, 0, 1, _lib.FP32, None, None, None, None, 0, None) == _lib.EINVAL


def test_catalog_struct_layout_matches_header():
    # x, phi, w pointers; int64 n; int32 field; int32 pad; double coeff -> 48 bytes
    assert ctypes.sizeof(_lib.Catalog) == 48
    assert _lib.Catalog.coeff.offset == 40 and _lib.Catalog.field.offset == 32


def test_ops_fail_loudly_without_cuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2312_12285_gb300 import ops
    with pytest.raises(Exception):
        ops.Plan(16)
