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


def test_host_validation_of_later_entry_points(lib):
    """Argument checks of the single-kernel batch, the on-demand mapping flag
    and the 32-bit-entry tables, all before any CUDA call."""
    from paper_2510_15095_gb300 import hive
    assert lib.hive_execute_fused(None, None, None, None, 4, None, None, None) == 1
    cfg = hive.Config()
    lib.hive_config_default(C.byref(cfg))
    assert cfg.map_on_demand == 0
    cfg.resizable = 1
    cfg.map_on_demand = 2
    h = C.c_void_p()
    assert lib.hive_create(C.byref(cfg), None, C.byref(h)) == 1
    c32 = hive.Config32()
    lib.hive32_config_default(C.byref(c32))
    assert c32.layout == hive.KEY16_VAL16 and c32.max_evictions == 16
    for field, bad in (("layout", 7), ("slots", 16), ("max_evictions", 0), ("lock_spin_limit", 0),
                       ("stash_permille", 1001)):
        b = hive.Config32()
        lib.hive32_config_default(C.byref(b))
        setattr(b, field, bad)
        assert lib.hive32_create(C.byref(b), None, C.byref(h)) == 1, field
    assert lib.hive32_insert(None, None, None, 3, None, None) == 1
    assert lib.hive32_find(None, None, 3, None, None, None) == 1
    assert lib.hive32_destroy(None) == 0


def test_host_validation_of_tuning_fields(lib):
    """The block shape and the L2-window flag are checked before any CUDA
    call; their defaults are 0 (256 threads, no window)."""
    from paper_2510_15095_gb300 import hive
    cfg = hive.Config()
    lib.hive_config_default(C.byref(cfg))
    assert cfg.block_threads == 0 and cfg.l2_persist == 0 and cfg.stage_wait_limit == 0
    h = C.c_void_p()
    for field, bad in (("block_threads", 100), ("block_threads", 1024), ("block_threads", 64),
                       ("l2_persist", 2)):
        b = hive.Config()
        lib.hive_config_default(C.byref(b))
        setattr(b, field, bad)
        assert lib.hive_create(C.byref(b), None, C.byref(h)) == 1, (field, bad)
        assert b"block_threads" in lib.hive_last_error()
