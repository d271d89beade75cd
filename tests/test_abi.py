"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without a
GPU, and exports every function include/hive.h declares; host-side argument
validation needs no device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hive(?:32)?_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2510_15095_gb300 import build as B
    path = B.build()
    from paper_2510_15095_gb300 import hive
    return hive.load_library(path)


def test_exports_match_header(lib):
    declared = _declared()
    assert {"hive_create", "hive_insert", "hive_find", "hive_erase", "hive_size",
            "hive_destroy"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_lists_every_export(lib):
    from paper_2510_15095_gb300 import hive
    assert set(hive.EXPORTS) == _declared()


def test_host_validation_without_gpu(lib):
    from paper_2510_15095_gb300 import hive
    cfg = hive.Config()
    lib.hive_config_default(C.byref(cfg))
    assert cfg.bucket_slots == 32 and cfg.grow_num == 9 and cfg.grow_den == 10
    # NULL table / NULL pointers are rejected before any CUDA call
    assert lib.hive_insert(None, None, None, 5, None, None) == 1
    assert lib.hive_find(None, None, 0, None, None, None) == 1
    assert b"NULL" in lib.hive_last_error()
    bad = hive.Config()
    lib.hive_config_default(C.byref(bad))
    bad.bucket_slots = 24
    h = C.c_void_p()
    assert lib.hive_create(C.byref(bad), None, C.byref(h)) == 1
    bad.bucket_slots = 32
    bad.shrink_num, bad.shrink_den = 9, 10
    assert lib.hive_create(C.byref(bad), None, C.byref(h)) == 1
    assert lib.hive_destroy(None) == 0
