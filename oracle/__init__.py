"""CPU oracle for the Hive hash table.  TEST INFRASTRUCTURE, NOT THE PRODUCT.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never imports it and shares no code with it.

The oracle is a plain single-threaded dictionary (``std::unordered_map``)
applied op by op (Section III-D of the paper), the paper's two hash mixes
(Section III-C, Listing 1), the linear-hashing address and resize policy
(Section IV-C) and a checker of the table's structural invariants.  See
``hive_oracle.cpp`` for the passage each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hive_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libhive_oracle.so")
_lock = threading.Lock()
_lib = None

# per-op result codes and op codes (same numbers as the library's interface)
INSERTED, REPLACED, ERASED, NOT_FOUND, FOUND, FULL, RESERVED = range(7)
OP_INSERT, OP_FIND, OP_ERASE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no GPU code involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC,
                               "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


class LHState(C.Structure):
    _fields_ = [("nb", C.c_uint64), ("nb_init", C.c_uint64), ("nb_max", C.c_uint64),
                ("M", C.c_uint32), ("p", C.c_uint32), ("S", C.c_uint32), ("K", C.c_uint32),
                ("grow_num", C.c_uint32), ("grow_den", C.c_uint32),
                ("shrink_num", C.c_uint32), ("shrink_den", C.c_uint32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, u64, u32, u8p = C.c_void_p, C.c_uint64, C.c_uint32, C.c_void_p
            L.orc_new.restype = vp
            L.orc_free.argtypes = [vp]
            L.orc_size.argtypes = [vp]
            L.orc_size.restype = u64
            L.orc_clear.argtypes = [vp]
            L.orc_insert.argtypes = [vp, vp, vp, u64, u8p]
            L.orc_find.argtypes = [vp, vp, u64, vp, u8p]
            L.orc_erase.argtypes = [vp, vp, u64, u8p]
            L.orc_execute.argtypes = [vp, vp, vp, vp, u64, vp, u8p]
            L.orc_dump.argtypes = [vp, vp, vp]
            L.orc_sharded_step.argtypes = [C.c_int, vp, vp, u64, u8p, vp, u64, vp, u8p, vp, vp, vp,
                                           u64, vp, u8p]
            L.orc_sharded_step.restype = C.c_double
            L.orc_bithash1.argtypes = [u32]
            L.orc_bithash1.restype = u32
            L.orc_bithash2.argtypes = [u32]
            L.orc_bithash2.restype = u32
            L.orc_lh_address.argtypes = [u32, u32, u32]
            L.orc_lh_address.restype = u32
            L.orc_bithash_many.argtypes = [C.c_int, vp, vp, u64]
            L.orc_bithash_checksum.argtypes = [u64, u64]
            L.orc_bithash_checksum.restype = u64
            L.orc_lh_address_many.argtypes = [vp, vp, u64, u32, u32]
            P = C.POINTER(LHState)
            L.orc_lh_init.argtypes = [P, u64, u64, u32, u32, u32, u32, u32, u32]
            L.orc_lh_split_step.argtypes = [P]
            L.orc_lh_split_step.restype = u32
            L.orc_lh_merge_step.argtypes = [P, u32]
            L.orc_lh_merge_step.restype = u32
            L.orc_lh_grow.argtypes = [P, u64, u64]
            L.orc_lh_grow.restype = u32
            L.orc_lh_shrink.argtypes = [P, u64]
            L.orc_lh_shrink.restype = u32
            L.orc_check_image.argtypes = [vp, vp, vp, u64, u32, u32, u32, vp, u64, u64, u64,
                                          u64, vp, vp, C.POINTER(C.c_uint64)]
            L.orc_check_image.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


class Dict:
    """The dictionary of Section III-D, applied op by op in array order."""

    def __init__(self):
        self._L = lib()
        self._h = self._L.orc_new()

    def close(self):
        if self._h:
            self._L.orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return int(self._L.orc_size(self._h))

    @property
    def handle(self):
        return self._h

    def clear(self):
        self._L.orc_clear(self._h)

    def insert(self, keys, vals):
        keys, vals = _u32(keys), _u32(vals)
        st = np.empty(keys.size, np.uint8)
        self._L.orc_insert(self._h, _ptr(keys), _ptr(vals), keys.size, _ptr(st))
        return st

    def find(self, keys):
        keys = _u32(keys)
        v = np.empty(keys.size, np.uint32)
        f = np.empty(keys.size, np.uint8)
        self._L.orc_find(self._h, _ptr(keys), keys.size, _ptr(v), _ptr(f))
        return v, f

    def erase(self, keys):
        keys = _u32(keys)
        st = np.empty(keys.size, np.uint8)
        self._L.orc_erase(self._h, _ptr(keys), keys.size, _ptr(st))
        return st

    def execute(self, ops, keys, vals):
        ops = np.ascontiguousarray(ops, dtype=np.uint8)
        keys, vals = _u32(keys), _u32(vals)
        v = np.empty(keys.size, np.uint32)
        st = np.empty(keys.size, np.uint8)
        self._L.orc_execute(self._h, _ptr(ops), _ptr(keys), _ptr(vals), keys.size, _ptr(v), _ptr(st))
        return v, st

    def dump(self):
        n = len(self)
        k = np.empty(n, np.uint32)
        v = np.empty(n, np.uint32)
        self._L.orc_dump(self._h, _ptr(k), _ptr(v))
        return k, v


def bithash1(x: int) -> int:
    return int(lib().orc_bithash1(int(x) & 0xFFFFFFFF))


def bithash2(x: int) -> int:
    return int(lib().orc_bithash2(int(x) & 0xFFFFFFFF))


def lh_address(h: int, M: int, p: int) -> int:
    return int(lib().orc_lh_address(int(h) & 0xFFFFFFFF, M, p))


def bithash_many(which: int, keys) -> np.ndarray:
    """BitHash1 (which=1) or BitHash2 (which=2) of every key."""
    k = _u32(keys)
    out = np.empty(k.size, np.uint32)
    lib().orc_bithash_many(which, _ptr(k), _ptr(out), k.size)
    return out


def bithash_checksum(lo: int, hi: int) -> int:
    """Sum over keys lo..hi-1 of (BitHash1(k) + 2^32 BitHash2(k)) * (2k + 1)
    modulo 2^64 (see orc_bithash_checksum)."""
    return int(lib().orc_bithash_checksum(int(lo), int(hi)))


def sharded_step(threads: int, ins_keys, ins_vals, find_keys, mix_ops, mix_keys, mix_vals):
    """A parallel CPU baseline (orc_sharded_step): inserts, then finds, then a
    mixed batch, on `threads` host threads over key-sharded maps.  Returns
    (seconds, insert statuses, find values, find flags, mixed values, mixed
    statuses); the results equal Dict's applied in the same order."""
    ik, iv, fk = _u32(ins_keys), _u32(ins_vals), _u32(find_keys)
    mo = np.ascontiguousarray(mix_ops, dtype=np.uint8)
    mk, mv = _u32(mix_keys), _u32(mix_vals)
    ist = np.empty(ik.size, np.uint8)
    fv, ff = np.empty(fk.size, np.uint32), np.empty(fk.size, np.uint8)
    mvo, mst = np.empty(mk.size, np.uint32), np.empty(mk.size, np.uint8)
    sec = lib().orc_sharded_step(int(threads), _ptr(ik), _ptr(iv), ik.size, _ptr(ist), _ptr(fk),
                                 fk.size, _ptr(fv), _ptr(ff), _ptr(mo), _ptr(mk), _ptr(mv),
                                 mk.size, _ptr(mvo), _ptr(mst))
    return float(sec), ist, fv, ff, mvo, mst


def lh_address_many(h, M: int, p: int) -> np.ndarray:
    hh = _u32(h)
    out = np.empty(hh.size, np.uint32)
    lib().orc_lh_address_many(_ptr(hh), _ptr(out), hh.size, M, p)
    return out


class Policy:
    """Linear-hashing capacity model (Section IV-C) under the load-factor policy."""

    def __init__(self, nb_init, nb_max, S=32, K=1024, grow=(9, 10), shrink=(2, 5)):
        self.s = LHState()
        lib().orc_lh_init(C.byref(self.s), nb_init, nb_max, S, K, grow[0], grow[1],
                          shrink[0], shrink[1])

    @property
    def state(self):
        return (int(self.s.nb), int(self.s.M), int(self.s.p))

    def split_step(self):
        return int(lib().orc_lh_split_step(C.byref(self.s)))

    def merge_step(self, max_step=0xFFFFFFFF):
        return int(lib().orc_lh_merge_step(C.byref(self.s), max_step))

    def grow(self, size, n_ins):
        return int(lib().orc_lh_grow(C.byref(self.s), size, n_ins))

    def shrink(self, size):
        return int(lib().orc_lh_shrink(C.byref(self.s), size))


def check_image(img: dict, S: int, dict_: Dict | None = None, policy: Policy | None = None):
    """Run invariants 1-7 over a host image of the table.  Returns (code, where)."""
    where = C.c_uint64(0)
    b = np.ascontiguousarray(img["buckets"], dtype=np.uint64)
    m = np.ascontiguousarray(img["masks"], dtype=np.uint32)
    lk = np.ascontiguousarray(img["locks"], dtype=np.uint32)
    st = np.ascontiguousarray(img["stash"], dtype=np.uint64)
    code = lib().orc_check_image(
        _ptr(b), _ptr(m), _ptr(lk), int(img["nb"]), S, int(img["M"]), int(img["p"]),
        _ptr(st) if st.size else None, st.size, int(img["stash_cap"]), int(img["size"]),
        int(img.get("pending", 0)), dict_.handle if dict_ is not None else None,
        C.byref(policy.s) if policy is not None else None, C.byref(where))
    return int(code), int(where.value)
