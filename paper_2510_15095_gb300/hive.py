"""Python binding of the Hive hash table C ABI (include/hive.h).

Argument marshalling only: every step of every operation runs in the CUDA
kernels of ``libhive_gb300.so``.  Tensors are PyTorch CUDA tensors (PyTorch is
used for device memory and streams); keys and values are 32-bit (``torch.int32``
or ``torch.uint32`` storage, reinterpreted as unsigned), per-op codes and
statuses are ``torch.uint8``.  There is no CPU fallback: if the library is not
built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhive_gb300.so")

# Status codes (include/hive.h)
HIVE_OK = 0
ERRORS = {1: "INVALID_ARG", 2: "RESERVED_KEY", 3: "OOM", 4: "FULL", 5: "TIMEOUT", 6: "CUDA",
          7: "CONTRACT"}
INSERTED, REPLACED, ERASED, NOT_FOUND, FOUND, FULL, RESERVED_KEY = range(7)
OP_INSERT, OP_FIND, OP_ERASE = 0, 1, 2
PLACE_BALANCED, PLACE_FIRST = 0, 1
MULTI_GRAPH, MULTI_ASYNC = 1, 2

EXPORTS = ["hive_config_default", "hive_create", "hive_destroy", "hive_insert", "hive_find",
           "hive_erase", "hive_execute", "hive_execute_fused", "hive_size", "hive_capacity", "hive_clear", "hive_check",
           "hive_stats", "hive_dump", "hive_profile_enable", "hive_profile_read",
           "hive_insert_noalloc", "hive_multi_create", "hive_multi_execute",
           "hive_multi_destroy", "hive_multi_bounds", "hive_insert_host", "hive_find_host", "hive_execute_host",
           "hive_reserve", "hive_memory", "hive_check_batch", "hive_last_error",
           "hive32_config_default", "hive32_create", "hive32_destroy", "hive32_insert",
           "hive32_find", "hive32_erase", "hive32_execute", "hive32_size", "hive32_clear",
           "hive32_check",
           "hive32_stats", "hive32_dump", "hive_debug_fail_alloc", "hive_debug_hold_lock", "hive_hash",
           "hive_host_direct_access", "hive_debug_set_versions"]
KERNEL_KINDS = ["find", "insert", "erase", "mixed", "evict", "maint", "split", "merge", "count",
                "fused", "claim"]


class HiveError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hive error {ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("initial_slots", C.c_uint64), ("max_slots", C.c_uint64),
                ("bucket_slots", C.c_uint32), ("max_evictions", C.c_uint32),
                ("resize_batch", C.c_uint32), ("stash_permille", C.c_uint32),
                ("grow_num", C.c_uint32), ("grow_den", C.c_uint32),
                ("shrink_num", C.c_uint32), ("shrink_den", C.c_uint32),
                ("resizable", C.c_uint32), ("placement", C.c_uint32),
                ("lock_spin_limit", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("map_on_demand", C.c_uint32), ("l2_persist", C.c_uint32),
                ("stage_wait_limit", C.c_uint32), ("block_threads", C.c_uint32)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "replaced", "claimed_fast", "overflowed", "claimed_slow", "evict_rounds", "lock_acquired",
        "lock_timeouts", "stashed", "pending", "stash_reinserted", "splits", "merges", "probes",
        "stash_lookups", "fused_retries")]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 16), ("launches", C.c_uint64 * 16)]


class Segment(C.Structure):
    _fields_ = [("table", C.c_uint32), ("reserved0", C.c_uint32), ("n", C.c_uint64),
                ("n_insert", C.c_uint64), ("ops", C.c_void_p), ("keys", C.c_void_p),
                ("vals", C.c_void_p), ("vals_out", C.c_void_p), ("status", C.c_void_p)]


class Config32(C.Structure):
    _fields_ = [("slots", C.c_uint64), ("layout", C.c_uint32), ("max_evictions", C.c_uint32),
                ("stash_permille", C.c_uint32), ("lock_spin_limit", C.c_uint32)]


class Image32(C.Structure):
    _fields_ = [("nb", C.c_uint64), ("M", C.c_uint32), ("p", C.c_uint32), ("layout", C.c_uint32),
                ("buckets", C.c_void_p), ("masks", C.c_void_p), ("locks", C.c_void_p),
                ("stash", C.c_void_p), ("stash_n", C.c_uint64), ("stash_cap", C.c_uint64),
                ("size", C.c_uint64), ("pending", C.c_uint64)]


class Image(C.Structure):
    _fields_ = [("nb", C.c_uint64), ("S", C.c_uint32), ("M", C.c_uint32), ("p", C.c_uint32),
                ("reserved0", C.c_uint32), ("stash_n", C.c_uint64), ("stash_cap", C.c_uint64),
                ("size", C.c_uint64), ("pending", C.c_uint64),
                ("buckets", C.c_void_p), ("masks", C.c_void_p), ("locks", C.c_void_p),
                ("stash", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libhive_gb300.so and declare its signatures.  Raises if missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run __graft_entry__.build() "
                               "(the CUDA library is required, there is no fallback)")
        L = C.CDLL(path)
        vp, u64, i32 = C.c_void_p, C.c_uint64, C.c_int
        L.hive_config_default.argtypes = [C.POINTER(Config)]
        L.hive_config_default.restype = None
        L.hive_create.argtypes = [C.POINTER(Config), vp, C.POINTER(vp)]
        L.hive_destroy.argtypes = [vp]
        L.hive_insert.argtypes = [vp, vp, vp, u64, vp, vp]
        L.hive_find.argtypes = [vp, vp, u64, vp, vp, vp]
        L.hive_erase.argtypes = [vp, vp, u64, vp, vp]
        L.hive_execute.argtypes = [vp, vp, vp, vp, u64, vp, vp, vp]
        L.hive_execute_fused.argtypes = [vp, vp, vp, vp, u64, vp, vp, vp]
        L.hive_size.argtypes = [vp, C.POINTER(u64), vp]
        L.hive_capacity.argtypes = [vp, C.POINTER(u64)]
        L.hive_reserve.argtypes = [vp, u64, vp]
        L.hive_memory.argtypes = [vp, C.POINTER(u64), C.POINTER(u64)]
        L.hive_clear.argtypes = [vp, vp]
        L.hive_check.argtypes = [vp, vp]
        L.hive_stats.argtypes = [vp, C.POINTER(Stats), vp]
        L.hive_dump.argtypes = [vp, C.POINTER(Image), vp]
        L.hive_insert_noalloc.argtypes = [vp, vp, vp, u64, vp, vp]
        L.hive_insert_host.argtypes = [vp, vp, vp, u64, vp, vp]
        L.hive_find_host.argtypes = [vp, vp, u64, vp, vp, vp]
        L.hive_execute_host.argtypes = [vp, vp, vp, vp, u64, vp, vp, vp]
        L.hive_multi_create.argtypes = [C.POINTER(vp), C.c_uint32, C.c_uint32, u64, i32, vp,
                                        C.POINTER(vp)]
        L.hive_multi_execute.argtypes = [vp, C.POINTER(Segment), C.c_uint32, vp]
        L.hive_multi_destroy.argtypes = [vp]
        L.hive_multi_bounds.argtypes = [vp, C.POINTER(u64), C.c_uint32]
        L.hive_profile_enable.argtypes = [vp, i32]
        L.hive_profile_read.argtypes = [vp, C.POINTER(Profile)]
        L.hive32_config_default.argtypes = [C.POINTER(Config32)]
        L.hive32_config_default.restype = None
        L.hive32_create.argtypes = [C.POINTER(Config32), vp, C.POINTER(vp)]
        L.hive32_destroy.argtypes = [vp]
        L.hive32_insert.argtypes = [vp, vp, vp, u64, vp, vp]
        L.hive32_find.argtypes = [vp, vp, u64, vp, vp, vp]
        L.hive32_erase.argtypes = [vp, vp, u64, vp, vp]
        L.hive32_execute.argtypes = [vp, vp, vp, vp, u64, vp, vp, vp]
        L.hive32_size.argtypes = [vp, C.POINTER(u64), vp]
        L.hive32_check.argtypes = [vp, vp]
        L.hive32_clear.argtypes = [vp, vp]
        L.hive32_stats.argtypes = [vp, C.POINTER(Stats), vp]
        L.hive32_dump.argtypes = [vp, C.POINTER(Image32), vp]
        L.hive_check_batch.argtypes = [vp, C.c_uint32, vp, u64, C.c_uint32, C.POINTER(u64)]
        L.hive_debug_fail_alloc.argtypes = [C.c_uint32]
        L.hive_hash.argtypes = [vp, u64, vp, vp, vp]
        L.hive_debug_hold_lock.argtypes = [vp, u64, i32, vp]
        L.hive_host_direct_access.argtypes = [vp]
        L.hive_debug_set_versions.argtypes = [vp, C.c_uint32, vp]
        L.hive_last_error.argtypes = []
        L.hive_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("hive_config_default", "hive_last_error", "hive32_config_default"):
                getattr(L, name).restype = i32
        _lib = L
        return L


def _raise(L, code):
    if code != HIVE_OK:
        raise HiveError(code, L.hive_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _sptr(t, itemsize: int, n: int, name: str):
    """Pointer of a segment array: a contiguous CUDA tensor, or a pinned CPU
    tensor, which the kernels read and write in place through the
    CPU-GPU link (at near device speed where host_direct_access() holds)."""
    if t is not None and not t.is_cuda:
        if not t.is_pinned():
            raise ValueError(f"{name} must be a CUDA tensor or a pinned CPU tensor")
        if not t.is_contiguous() or t.element_size() != itemsize or t.numel() < n:
            raise ValueError(f"{name} must be contiguous with >= {n} {itemsize}-byte items")
        return t.data_ptr()
    return _dptr(t, itemsize, n, name)


def _dptr(t, itemsize: int, n: int, name: str):
    """Device pointer of a contiguous CUDA tensor with >= n items of itemsize."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.element_size() != itemsize:
        raise ValueError(f"{name} must have {itemsize}-byte elements")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, need {n}")
    return t.data_ptr()


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class HiveTable:
    """One Hive table on the current CUDA device (see include/hive.h)."""

    def __init__(self, initial_slots: int = 1 << 20, *, max_slots: int | None = None,
                 resizable: bool = False, max_evictions: int = 16, resize_batch: int = 1024,
                 stash_permille: int = 10, grow=(9, 10), shrink=(2, 5),
                 placement: int = PLACE_BALANCED, lock_spin_limit: int | None = None,
                 blocks_per_sm: int = 0, bucket_slots: int = 32, map_on_demand: bool = False,
                 l2_persist: bool = False, stage_wait_limit: int = 0, block_threads: int = 0,
                 stream=None):
        self._L = load_library()
        cfg = Config()
        self._L.hive_config_default(C.byref(cfg))
        cfg.initial_slots = int(initial_slots)
        cfg.bucket_slots = int(bucket_slots)
        cfg.max_slots = int(max_slots if max_slots is not None else initial_slots)
        cfg.max_evictions = int(max_evictions)
        cfg.resize_batch = int(resize_batch)
        cfg.stash_permille = int(stash_permille)
        cfg.grow_num, cfg.grow_den = map(int, grow)
        cfg.shrink_num, cfg.shrink_den = map(int, shrink)
        cfg.resizable = 1 if resizable else 0
        cfg.placement = int(placement)
        if lock_spin_limit is not None:
            cfg.lock_spin_limit = int(lock_spin_limit)
        cfg.blocks_per_sm = int(blocks_per_sm)
        cfg.map_on_demand = 1 if map_on_demand else 0
        cfg.l2_persist = 1 if l2_persist else 0
        cfg.stage_wait_limit = int(stage_wait_limit)
        cfg.block_threads = int(block_threads)
        self.config = cfg
        h = C.c_void_p()
        _raise(self._L, self._L.hive_create(C.byref(cfg), _stream_ptr(stream), C.byref(h)))
        self._h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._L.hive_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- operations -------------------------------------------------------
    def insert(self, keys, vals, status=True, stream=None):
        """Insert/Replace.  Returns the per-op status tensor (uint8) or None."""
        torch = _torch()
        n = keys.numel()
        st = None
        if status is True:
            st = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is not None and status is not False:
            st = status
        _raise(self._L, self._L.hive_insert(
            self._h, _dptr(keys, 4, n, "keys"), _dptr(vals, 4, n, "vals"), n,
            _dptr(st, 1, n, "status"), _stream_ptr(stream)))
        return st

    def insert_noalloc(self, keys, vals, status=True, stream=None):
        """hive_insert_noalloc: the fixed-table insert that allocates nothing
        (for callers that must not call cudaMalloc); at most 2^18 ops."""
        torch = _torch()
        n = keys.numel()
        st = None
        if status is True:
            st = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is not None and status is not False:
            st = status
        _raise(self._L, self._L.hive_insert_noalloc(
            self._h, _dptr(keys, 4, n, "keys"), _dptr(vals, 4, n, "vals"), n,
            _dptr(st, 1, n, "status"), _stream_ptr(stream)))
        return st

    def find(self, keys, vals_out=None, found=True, stream=None):
        """Search.  Returns (values, found-flags or None); values are 0 on a miss."""
        torch = _torch()
        n = keys.numel()
        if vals_out is None:
            vals_out = torch.empty(n, dtype=keys.dtype, device=keys.device)
        fo = None
        if found is True:
            fo = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif found is not None and found is not False:
            fo = found
        _raise(self._L, self._L.hive_find(
            self._h, _dptr(keys, 4, n, "keys"), n, _dptr(vals_out, 4, n, "vals_out"),
            _dptr(fo, 1, n, "found"), _stream_ptr(stream)))
        return vals_out, fo

    def erase(self, keys, status=True, stream=None):
        torch = _torch()
        n = keys.numel()
        st = None
        if status is True:
            st = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is not None and status is not False:
            st = status
        _raise(self._L, self._L.hive_erase(
            self._h, _dptr(keys, 4, n, "keys"), n, _dptr(st, 1, n, "status"), _stream_ptr(stream)))
        return st

    def execute(self, ops, keys, vals=None, stream=None, fused=False):
        """Mixed batch.  Returns (values, status).  fused=True runs it as one
        concurrent kernel (hive_execute_fused) instead of the phased launches."""
        torch = _torch()
        n = keys.numel()
        vo = torch.empty(n, dtype=keys.dtype, device=keys.device)
        st = torch.empty(n, dtype=torch.uint8, device=keys.device)
        fn = self._L.hive_execute_fused if fused else self._L.hive_execute
        _raise(self._L, fn(
            self._h, _dptr(ops, 1, n, "ops"), _dptr(keys, 4, n, "keys"),
            _dptr(vals, 4, n, "vals") if vals is not None else None, n,
            _dptr(vo, 4, n, "vals_out"), _dptr(st, 1, n, "status"), _stream_ptr(stream)))
        return vo, st

    # -- host-buffer calls (pinned CPU tensors for overlap) ----------------
    @staticmethod
    def _hptr(t, itemsize, n, name):
        if t is None:
            return None
        if t.is_cuda or not t.is_contiguous() or t.element_size() != itemsize or t.numel() < n:
            raise ValueError(f"{name} must be a contiguous CPU tensor of {n} {itemsize}-byte items")
        return t.data_ptr()

    def insert_host(self, keys, vals, status=None, stream=None):
        """hive_insert_host: keys/vals (and status, if given) are CPU tensors.
        Pinned tensors run in place where host_direct_access() holds; pageable
        ones stream through device staging."""
        n = keys.numel()
        _raise(self._L, self._L.hive_insert_host(
            self._h, self._hptr(keys, 4, n, "keys"), self._hptr(vals, 4, n, "vals"), n,
            self._hptr(status, 1, n, "status"), _stream_ptr(stream)))
        return status

    def find_host(self, keys, vals_out, found=None, stream=None):
        n = keys.numel()
        _raise(self._L, self._L.hive_find_host(
            self._h, self._hptr(keys, 4, n, "keys"), n, self._hptr(vals_out, 4, n, "vals_out"),
            self._hptr(found, 1, n, "found"), _stream_ptr(stream)))
        return vals_out, found

    def execute_host(self, ops, keys, vals, vals_out=None, status=None, stream=None):
        n = keys.numel()
        _raise(self._L, self._L.hive_execute_host(
            self._h, self._hptr(ops, 1, n, "ops"), self._hptr(keys, 4, n, "keys"),
            self._hptr(vals, 4, n, "vals"), n, self._hptr(vals_out, 4, n, "vals_out"),
            self._hptr(status, 1, n, "status"), _stream_ptr(stream)))
        return vals_out, status

    # -- state ------------------------------------------------------------
    def size(self, stream=None) -> int:
        out = C.c_uint64()
        _raise(self._L, self._L.hive_size(self._h, C.byref(out), _stream_ptr(stream)))
        return int(out.value)

    def reserve(self, slots: int, stream=None):
        """Grow (resizable tables) to at least `slots` slots ahead of time."""
        _raise(self._L, self._L.hive_reserve(self._h, int(slots), _stream_ptr(stream)))

    def memory(self) -> tuple:
        """(committed, reserved) device bytes of the table."""
        a, b = C.c_uint64(), C.c_uint64()
        _raise(self._L, self._L.hive_memory(self._h, C.byref(a), C.byref(b)))
        return int(a.value), int(b.value)

    def capacity(self) -> int:
        out = C.c_uint64()
        _raise(self._L, self._L.hive_capacity(self._h, C.byref(out)))
        return int(out.value)

    def clear(self, stream=None):
        _raise(self._L, self._L.hive_clear(self._h, _stream_ptr(stream)))

    def check(self, stream=None) -> int:
        """Sticky device error (0 = none); clears it."""
        return int(self._L.hive_check(self._h, _stream_ptr(stream)))

    def stats(self, stream=None) -> dict:
        s = Stats()
        _raise(self._L, self._L.hive_stats(self._h, C.byref(s), _stream_ptr(stream)))
        return {f: int(getattr(s, f)) for f, _ in Stats._fields_}

    def profile(self, enable: bool):
        """Turn per-kernel event timing on or off (see hive_profile_enable)."""
        _raise(self._L, self._L.hive_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kind: (ms, launches)} for kernels timed since the last read."""
        p = Profile()
        _raise(self._L, self._L.hive_profile_read(self._h, C.byref(p)))
        return {k: (float(p.ms[i]), int(p.launches[i])) for i, k in enumerate(KERNEL_KINDS)
                if p.launches[i]}

    def debug_hold_lock(self, bucket: int | None, held: bool, stream=None):
        """hive_debug_hold_lock: hold or free one bucket lock (None: every
        bucket in use), so that a test can make eviction waits give up."""
        b = 0xFFFFFFFFFFFFFFFF if bucket is None else int(bucket)
        _raise(self._L, self._L.hive_debug_hold_lock(self._h, b, 1 if held else 0,
                                                     _stream_ptr(stream)))

    def debug_set_versions(self, value: int, stream=None):
        """hive_debug_set_versions: set every bucket version word (bits 16..31,
        the count of finished moves), so that a test can start the
        single-kernel batch next to the count's wrap."""
        _raise(self._L, self._L.hive_debug_set_versions(self._h, int(value) & 0xFFFFFFFF,
                                                        _stream_ptr(stream)))

    def dump(self, stream=None) -> dict:
        """Host image of the table (numpy arrays) for checks and checkpoints."""
        img = Image()
        _raise(self._L, self._L.hive_dump(self._h, C.byref(img), _stream_ptr(stream)))
        nb, S = int(img.nb), int(img.S)
        b = np.empty(nb * S, np.uint64)
        m = np.empty(nb, np.uint32)
        lk = np.empty(nb, np.uint32)
        st = np.empty(max(int(img.stash_n), 1), np.uint64)
        img.buckets = b.ctypes.data
        img.masks = m.ctypes.data
        img.locks = lk.ctypes.data
        img.stash = st.ctypes.data
        _raise(self._L, self._L.hive_dump(self._h, C.byref(img), _stream_ptr(stream)))
        return {"nb": nb, "S": S, "M": int(img.M), "p": int(img.p), "buckets": b, "masks": m,
                "locks": lk, "stash": st[: int(img.stash_n)], "stash_cap": int(img.stash_cap),
                "size": int(img.size), "pending": int(img.pending)}


KEY16_VAL16, KEY_ONLY = 0, 1


class Hive32Table:
    """A fixed-capacity table with 32-bit entries (hive32_*): a 16-bit key with
    a 16-bit value (layout KEY16_VAL16) or a set of 32-bit keys (KEY_ONLY);
    32 slots of 4 bytes per 128-byte bucket."""

    def __init__(self, slots: int = 1 << 20, layout: int = KEY16_VAL16, *, max_evictions: int = 16,
                 stash_permille: int = 10, lock_spin_limit: int | None = None, stream=None):
        self._L = load_library()
        cfg = Config32()
        self._L.hive32_config_default(C.byref(cfg))
        cfg.slots = int(slots)
        cfg.layout = int(layout)
        cfg.max_evictions = int(max_evictions)
        cfg.stash_permille = int(stash_permille)
        if lock_spin_limit is not None:
            cfg.lock_spin_limit = int(lock_spin_limit)
        self.config = cfg
        h = C.c_void_p()
        _raise(self._L, self._L.hive32_create(C.byref(cfg), _stream_ptr(stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.hive32_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def insert(self, keys, vals=None, status=True, stream=None):
        torch = _torch()
        n = keys.numel()
        st = torch.empty(n, dtype=torch.uint8, device=keys.device) if status is True else (
            status if status is not None and status is not False else None)
        _raise(self._L, self._L.hive32_insert(
            self._h, _dptr(keys, 4, n, "keys"), _dptr(vals, 4, n, "vals"), n,
            _dptr(st, 1, n, "status"), _stream_ptr(stream)))
        return st

    def find(self, keys, vals_out=None, found=True, stream=None):
        torch = _torch()
        n = keys.numel()
        if vals_out is None:
            vals_out = torch.empty(n, dtype=keys.dtype, device=keys.device)
        fo = torch.empty(n, dtype=torch.uint8, device=keys.device) if found is True else (
            found if found is not None and found is not False else None)
        _raise(self._L, self._L.hive32_find(
            self._h, _dptr(keys, 4, n, "keys"), n, _dptr(vals_out, 4, n, "vals_out"),
            _dptr(fo, 1, n, "found"), _stream_ptr(stream)))
        return vals_out, fo

    def erase(self, keys, status=True, stream=None):
        torch = _torch()
        n = keys.numel()
        st = torch.empty(n, dtype=torch.uint8, device=keys.device) if status is True else (
            status if status is not None and status is not False else None)
        _raise(self._L, self._L.hive32_erase(
            self._h, _dptr(keys, 4, n, "keys"), n, _dptr(st, 1, n, "status"), _stream_ptr(stream)))
        return st

    def execute(self, ops, keys, vals=None, stream=None):
        torch = _torch()
        n = keys.numel()
        vo = torch.empty(n, dtype=keys.dtype, device=keys.device)
        st = torch.empty(n, dtype=torch.uint8, device=keys.device)
        _raise(self._L, self._L.hive32_execute(
            self._h, _dptr(ops, 1, n, "ops"), _dptr(keys, 4, n, "keys"),
            _dptr(vals, 4, n, "vals") if vals is not None else None, n,
            _dptr(vo, 4, n, "vals_out"), _dptr(st, 1, n, "status"), _stream_ptr(stream)))
        return vo, st

    def size(self, stream=None) -> int:
        out = C.c_uint64()
        _raise(self._L, self._L.hive32_size(self._h, C.byref(out), _stream_ptr(stream)))
        return int(out.value)

    def check(self, stream=None) -> int:
        return int(self._L.hive32_check(self._h, _stream_ptr(stream)))

    def clear(self, stream=None):
        _raise(self._L, self._L.hive32_clear(self._h, _stream_ptr(stream)))

    def stats(self, stream=None) -> dict:
        s = Stats()
        _raise(self._L, self._L.hive32_stats(self._h, C.byref(s), _stream_ptr(stream)))
        return {f: int(getattr(s, f)) for f, _ in Stats._fields_}

    def dump(self, stream=None) -> dict:
        img = Image32()
        _raise(self._L, self._L.hive32_dump(self._h, C.byref(img), _stream_ptr(stream)))
        nb = int(img.nb)
        b = np.empty(nb * 32, np.uint32)
        m = np.empty(nb, np.uint32)
        lk = np.empty(nb, np.uint32)
        st = np.empty(max(int(img.stash_n), 1), np.uint32)
        img.buckets = b.ctypes.data
        img.masks = m.ctypes.data
        img.locks = lk.ctypes.data
        img.stash = st.ctypes.data
        _raise(self._L, self._L.hive32_dump(self._h, C.byref(img), _stream_ptr(stream)))
        return {"nb": nb, "S": 32, "M": int(img.M), "p": int(img.p), "layout": int(img.layout),
                "buckets": b, "masks": m, "locks": lk, "stash": st[: int(img.stash_n)],
                "stash_cap": int(img.stash_cap), "size": int(img.size),
                "pending": int(img.pending)}


class HiveMulti:
    """A group of tables serviced by one launch per phase (hive_multi_*)."""

    def __init__(self, tables, max_segments: int, max_ops: int, use_graph: bool = True,
                 asynchronous: bool = False, stream=None):
        self._L = load_library()
        self.tables = list(tables)
        arr = (C.c_void_p * len(self.tables))(*[t._h.value for t in self.tables])
        h = C.c_void_p()
        flags = (MULTI_GRAPH if use_graph else 0) | (MULTI_ASYNC if asynchronous else 0)
        _raise(self._L, self._L.hive_multi_create(arr, len(self.tables), int(max_segments),
                                                  int(max_ops), flags,
                                                  _stream_ptr(stream), C.byref(h)))
        self._h = h

    def execute(self, segments, stream=None):
        """segments: iterable of dicts with keys table, ops, keys and optionally
        vals, vals_out, status (CUDA tensors, or pinned CPU tensors that the
        kernels use in place) and n_insert (int)."""
        segs = list(segments)
        arr = (Segment * max(len(segs), 1))()
        for i, g in enumerate(segs):
            n = g["keys"].numel()
            arr[i].table = int(g["table"])
            arr[i].n = n
            arr[i].n_insert = int(g.get("n_insert", n))
            arr[i].ops = _sptr(g["ops"], 1, n, "ops")
            arr[i].keys = _sptr(g["keys"], 4, n, "keys")
            arr[i].vals = _sptr(g.get("vals"), 4, n, "vals")
            arr[i].vals_out = _sptr(g.get("vals_out"), 4, n, "vals_out")
            arr[i].status = _sptr(g.get("status"), 1, n, "status")
        _raise(self._L, self._L.hive_multi_execute(self._h, arr, len(segs), _stream_ptr(stream)))

    def bounds(self) -> list:
        """hive_multi_bounds: upper bounds of the tables' live sizes (host
        side; never waits)."""
        n = len(self.tables)
        out = (C.c_uint64 * max(n, 1))()
        _raise(self._L, self._L.hive_multi_bounds(self._h, out, n))
        return [int(out[i]) for i in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            self._L.hive_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hash_keys(keys, stream=None):
    """hive_hash: (BitHash1, BitHash2) of every key of a CUDA tensor with
    32-bit elements, as int32 tensors holding the unsigned mixes."""
    torch = _torch()
    L = load_library()
    n = keys.numel()
    h1 = torch.empty(n, dtype=torch.int32, device=keys.device)
    h2 = torch.empty(n, dtype=torch.int32, device=keys.device)
    _raise(L, L.hive_hash(_dptr(keys, 4, n, "keys"), n, _dptr(h1, 4, n, "h1"),
                          _dptr(h2, 4, n, "h2"), _stream_ptr(stream)))
    return h1, h2


def host_direct_access() -> bool:
    """hive_host_direct_access: whether the current device reaches host memory
    coherently, so that host-buffer calls on pinned arrays run in place."""
    L = load_library()
    out = C.c_int(0)
    _raise(L, L.hive_host_direct_access(C.byref(out)))
    return bool(out.value)


def debug_fail_alloc(n: int):
    """hive_debug_fail_alloc: the n-th device allocation of the library from
    now on fails as out of memory (0 cancels)."""
    L = load_library()
    _raise(L, L.hive_debug_fail_alloc(int(n)))


def check_batch(keys, ops=None, op: int = OP_INSERT, key_limit: int = 0xFFFFFFFE):
    """Host-side batch-contract check (hive_check_batch): None when the batch
    keeps the contract, else the index of the first op that breaks it.
    `keys` (and `ops`, for a mixed batch) are host arrays (numpy or CPU
    tensors); with ops None every op is `op`.  Needs no GPU."""
    L = load_library()
    a = np.asarray(keys)
    # 32-bit integer storage is taken as unsigned bits; anything else is converted
    k = np.ascontiguousarray(a.view(np.uint32) if a.dtype.kind in "iu" and a.dtype.itemsize == 4
                             else a.astype(np.uint32))
    o = None if ops is None else np.ascontiguousarray(np.asarray(ops, dtype=np.uint8))
    if o is not None and o.size != k.size:
        raise ValueError("ops and keys differ in length")
    bad = C.c_uint64()
    code = L.hive_check_batch(None if o is None else o.ctypes.data, op, k.ctypes.data, k.size,
                              key_limit, C.byref(bad))
    if code == HIVE_OK:
        return None
    if code != 1 or bad.value >= k.size:
        _raise(L, code)
    return int(bad.value)


def to_device_u32(a: np.ndarray, device="cuda"):
    """numpy uint32 -> CUDA tensor holding the same 32-bit words (int32 storage)."""
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(device)


def to_host_u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)
