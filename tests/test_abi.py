"""The C ABI library builds, loads and exports every function include/sdf.h declares (CPU only:
no call here touches a GPU).  Also checks the argument validation that returns before any
device work, and that the product package never imports the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sdf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1903_00353_gb300 as pkg
    return pkg.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code in range(0, 10):
        s = lib.sdf_status_string(code)
        assert s and s != b"unknown status"
    assert lib.sdf_status_string(99) == b"unknown status"


def test_argument_validation_without_device(lib):
    out = ctypes.c_void_p(1234)
    assert lib.sdf_build_features(None, 10, 0, None, ctypes.byref(out)) == 1
    assert out.value is None
    assert lib.sdf_build_features(ctypes.c_void_p(16), 0, 0, None, ctypes.byref(out)) == 1
    assert lib.sdf_build_features(ctypes.c_void_p(16), 1 << 28, 0, None, ctypes.byref(out)) == 5
    assert lib.sdf_narrow_band(None, None, None, 1, None, None, 0, None) == 1
    assert lib.sdf_features_info(None, None, None) == 1
    lib.sdf_features_destroy(None)
    batch = ctypes.c_void_p(1234)
    assert lib.sdf_batch_create(None, None, None, 1, None, None, 0, None, ctypes.byref(batch)) == 1
    assert batch.value is None
    assert lib.sdf_batch_run(None, None) == 1
    assert lib.sdf_batch_status(None, None, None) == 1
    assert lib.sdf_batch_info(None, None, None) == 1
    assert lib.sdf_batch_timing(None, None) == 1
    lib.sdf_batch_destroy(None)
    assert lib.sdf_band_l2_loss(None, None, 0, None, None, None, None) == 1
    assert lib.sdf_narrow_band_list(None, None, 0.1, None, None, None, 0, None, 0, None) == 1
    assert lib.sdf_narrow_band_lists(None, None, None, 1, None, None, None, None, None, 0, None) == 1
    assert lib.sdf_band_list_backward(None, None, None, 0, None, None, None, 0, None) == 1
    assert lib.sdf_band_list_l2(None, None, None, 0, None, None, None, None, None, None, 0, None) == 1
    ops = ctypes.c_int64(0)
    assert lib.sdf_probe_rate(0, None, 1 << 20, 1, ctypes.byref(ops), None) == 1
    assert lib.sdf_probe_rate(1, ctypes.c_void_p(256), 1 << 20, 0, ctypes.byref(ops), None) == 1


def test_product_package_does_not_import_oracle():
    pkg_dir = os.path.join(ROOT, "paper_1903_00353_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "oracle." not in text.replace("the oracle", ""), f
