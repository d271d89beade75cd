// Hive table with 32-bit entries (Section III-B: with 32-bit entries -- a
// key-only set, or a 16-bit key with a 16-bit value -- a 32-slot bucket is
// 128 bytes, one cache line, half the bytes of a probe of the 64-bit table).
//
// Same algorithm as the 64-bit table, fixed capacity:
//   k32_ops<MODE, LAYOUT>  bulk find / insert (steps 1-2) / erase / mixed.
//                          Every probe round is staged: the op buckets are
//                          copied into the warp's shared-memory buffer
//                          (16-byte cp.async, eight lanes per bucket) and each
//                          lane scans its op's bucket(s) itself, 16 bytes (four
//                          slots) per read.
//   k32_overflow<LAYOUT>   steps 3-4: bounded cuckoo eviction under the
//                          bucket lock, warp per item (one slot per lane),
//                          then the stash.
//   k32_maint<LAYOUT>      stash maintenance: reinsert, sort by key, compact.
// The empty word is all ones; its key (0xFFFF or 0xFFFFFFFF) is reserved.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hive_device.cuh"
#include "hive_internal.h"

namespace hive {
namespace {

constexpr int kS32 = 32;                   // slots per bucket
constexpr uint32_t kEmpty32 = 0xFFFFFFFFu;  // empty slot
constexpr int kOps32Threads = 256;
constexpr int kStage32Words = 2048;         // 8 KB per warp: 64 buckets of 128 B
// A paired insert round fills the 8 KB; a single-bucket round needs 32
// buckets (4 KB), which lets four blocks share an SM.
__host__ __device__ constexpr int stage32_words(int mode) {
  return mode == kModeInsert ? kStage32Words : kStage32Words / 2;
}
__host__ __device__ constexpr size_t stage32_smem(int mode) {
  return static_cast<size_t>(kOps32Threads / 32) * (4u * stage32_words(mode) + 16u);
}
constexpr uint32_t kMbarSpin32 = 1u << 22;
constexpr int kMaint32Threads = 1024;
#ifndef HIVE32_STAGE_LSU
// Staged rounds copy buckets with cp.async through the load/store path (1)
// or with one bulk copy (TMA) per bucket (0).
#define HIVE32_STAGE_LSU 1
#endif
constexpr unsigned kMaint32SmemWords = 16384;  // 64 KB of words sorted in shared memory

// Entry layouts.
template <int LAYOUT>
struct E32;
template <>
struct E32<HIVE32_KEY16_VAL16> {  // value << 16 | key
  static __device__ __forceinline__ uint32_t key(uint32_t w) { return w & 0xFFFFu; }
  static __device__ __forceinline__ uint32_t val(uint32_t w) { return w >> 16; }
  static __device__ __forceinline__ uint32_t pack(uint32_t k, uint32_t v) { return (v << 16) | k; }
  // keys 0xFFFE and 0xFFFF are reserved; keys and values must fit 16 bits
  static __device__ __forceinline__ bool reserved(uint32_t k, uint32_t v) {
    return k >= 0xFFFEu || v > 0xFFFFu;
  }
};
template <>
struct E32<HIVE32_KEY_ONLY> {  // the key itself
  static __device__ __forceinline__ uint32_t key(uint32_t w) { return w; }
  static __device__ __forceinline__ uint32_t val(uint32_t) { return 0u; }
  static __device__ __forceinline__ uint32_t pack(uint32_t k, uint32_t) { return k; }
  static __device__ __forceinline__ bool reserved(uint32_t k, uint32_t) { return k >= 0xFFFFFFFEu; }
};

__device__ __forceinline__ void st_relaxed32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void lds_frag4(const uint32_t* p, uint32_t& a, uint32_t& b,
                                          uint32_t& c, uint32_t& d) {
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
               : "r"(smem_u32(p)));
}

struct Counters32 {
  int size_delta = 0;
  unsigned replaced = 0, claimed = 0, overflowed = 0, probes = 0;
  bool reserved = false, contract = false;
};

__device__ __forceinline__ void flush32(const View32& v, Counters32& c, int lane) {
  const int sd = __reduce_add_sync(kFull, static_cast<unsigned>(c.size_delta));
  const unsigned rp = __reduce_add_sync(kFull, c.replaced);
  const unsigned cl = __reduce_add_sync(kFull, c.claimed);
  const unsigned of = __reduce_add_sync(kFull, c.overflowed);
  const unsigned rs = __ballot_sync(kFull, c.reserved);
  const unsigned ct = __ballot_sync(kFull, c.contract);
  if (lane == 0) {
    if (c.probes) atomicAdd(&v.ctrl->stats[kStProbes], static_cast<unsigned long long>(c.probes));
    if (sd) atomicAdd(&v.ctrl->size, static_cast<unsigned long long>(static_cast<long long>(sd)));
    if (rp) atomicAdd(&v.ctrl->stats[kStReplaced], static_cast<unsigned long long>(rp));
    if (cl) atomicAdd(&v.ctrl->stats[kStClaimedFast], static_cast<unsigned long long>(cl));
    if (of) atomicAdd(&v.ctrl->stats[kStOverflowed], static_cast<unsigned long long>(of));
    if (rs) atomicOr(&v.ctrl->err, kErrReserved);
    if (ct) atomicOr(&v.ctrl->err, kErrContract);
  }
  c = Counters32();
}

// ---- staging -------------------------------------------------------------

struct Stage32 {
  uint64_t* bar;
  uint32_t* buf;  // kStage32Words words, 16-byte aligned
  uint32_t phase;
  bool dead;
};

__device__ __forceinline__ Stage32 stage32_init(uint64_t* smem, int warp_in_block, int lane,
                                                int words) {
  Stage32 sg;
  uint64_t* base = smem + static_cast<size_t>(warp_in_block) * (words / 2 + 2);
  sg.bar = base;
  sg.buf = reinterpret_cast<uint32_t*>(base + 2);
  sg.phase = 0;
  sg.dead = false;
  if (lane == 0) mbar_init(sg.bar, 1);
  __syncwarp();
  return sg;
}

__device__ __forceinline__ void stage32_drain(Stage32& sg) {
  if (!sg.dead) return;
  bool ok = false;
  for (uint32_t it = 0; it < kMbarSpin32 && !ok; ++it) ok = mbar_try_wait(sg.bar, sg.phase ^ 1u);
}

// Copies, for every op j with bit j of `need`, its bucket x1 (and with PAIR
// its bucket x2) into buffer bucket j (PAIR: 2j and 2j + 1), then waits
// (warp-wide, bounded).  Returns false with the stage dead if the wait gave up.
template <bool PAIR>
__device__ __forceinline__ bool stage32_round(const View32& v, Stage32& sg, unsigned need,
                                              uint32_t x1, uint32_t x2, int lane) {
  constexpr uint32_t kBucketBytes = kS32 * 4u;
  if (HIVE32_STAGE_LSU) {
    // cp.async through the load/store path: eight lanes copy one 128-byte
    // bucket, 16 bytes each, so one warp instruction moves four buckets
    constexpr int NB = PAIR ? 64 : 32;
    const int q = lane >> 3, ql = lane & 7;
    __syncwarp();
#pragma unroll 4
    for (int r = 0; r < NB / 4; ++r) {
      const int bi = 4 * r + q;
      const int op = PAIR ? (bi >> 1) : bi;
      const uint32_t y1 = __shfl_sync(kFull, x1, op);
      const uint32_t y2 = PAIR ? __shfl_sync(kFull, x2, op) : 0u;
      const uint32_t b = (PAIR && (bi & 1)) ? y2 : y1;
      if ((need >> op) & 1u)
        cp_async16(sg.buf + bi * kS32 + 4 * ql, v.buckets + static_cast<uint64_t>(b) * kS32 + 4 * ql);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();
    return true;
  }
  fence_proxy_async();
  __syncwarp();
  if (lane == 0) mbar_arrive_expect_tx(sg.bar, __popc(need) * (PAIR ? 2u : 1u) * kBucketBytes);
  __syncwarp();
  if ((need >> lane) & 1u) {
    if (PAIR) {
      bulk_g2s(sg.buf + 2 * lane * kS32, v.buckets + static_cast<uint64_t>(x1) * kS32,
               kBucketBytes, sg.bar);
      bulk_g2s(sg.buf + (2 * lane + 1) * kS32, v.buckets + static_cast<uint64_t>(x2) * kS32,
               kBucketBytes, sg.bar);
    } else {
      bulk_g2s(sg.buf + lane * kS32, v.buckets + static_cast<uint64_t>(x1) * kS32, kBucketBytes,
               sg.bar);
    }
  }
  bool ok = false;
  for (uint32_t it = 0; it < kMbarSpin32 && !ok; ++it) ok = mbar_try_wait(sg.bar, sg.phase);
  sg.phase ^= 1u;
  if (__any_sync(kFull, !ok)) {  // never expected
    sg.dead = true;
    if (lane == 0) atomicOr(&v.ctrl->err, kErrTimeout);
    return false;
  }
  return true;
}

// Slot of `key` in a bucket staged in shared memory, or -1.  Reads 16 bytes
// (four slots) at a time, starting at fragment (lane mod 8) so the lanes of a
// wavefront hit different banks.  scan32_global is the same search on a
// bucket in global memory (the fallback when a staged wait gave up).
template <int LAYOUT>
__device__ __forceinline__ int scan32(const uint32_t* B, uint32_t key, int lane) {
  using E = E32<LAYOUT>;
  int ms = -1;
#pragma unroll
  for (int k = 0; k < kS32 / 4; ++k) {
    const int f = (k + lane) & (kS32 / 4 - 1);
    uint32_t a, b, c, d;
    lds_frag4(B + 4 * f, a, b, c, d);
    if (E::key(a) == key) ms = 4 * f;
    if (E::key(b) == key) ms = 4 * f + 1;
    if (E::key(c) == key) ms = 4 * f + 2;
    if (E::key(d) == key) ms = 4 * f + 3;
  }
  return ms;
}
template <int LAYOUT>
__device__ __forceinline__ int scan32_global(const uint32_t* B, uint32_t key) {
  using E = E32<LAYOUT>;
  int ms = -1;
  for (int k = 0; k < kS32; ++k) {
    const uint32_t w = ld_relaxed32(B + k);
    if (w != kEmpty32 && E::key(w) == key) ms = k;
  }
  return ms;
}

// Claim step 2 in bucket b, first trying slot s (the fetch_and result is the
// authority), and publish the word.
__device__ __forceinline__ bool claim32(const View32& v, uint32_t b, uint32_t s, uint32_t word) {
  for (int t = 0; t <= kS32 && s < kS32; ++t) {
    const uint32_t bit = 1u << s;
    const uint32_t old = atomicAnd(v.masks + b, ~bit);
    if (old & bit) {
      st_relaxed32(v.buckets + static_cast<uint64_t>(b) * kS32 + s, word);
      return true;
    }
    s = old ? static_cast<uint32_t>(__ffs(old) - 1) : kS32;
  }
  return false;
}
// Claim publishing with CAS(EMPTY -> word) (the eviction kernel, where an
// exchange may land on a claimed, unpublished slot).
__device__ __forceinline__ bool claim32_cas(const View32& v, uint32_t b, uint32_t word,
                                            uint32_t hint = 0) {
  uint32_t fm = hint ? hint : ld_relaxed32(v.masks + b);
  for (int t = 0; t <= 2 * kS32 && fm; ++t) {
    const uint32_t s = __ffs(fm) - 1;
    const uint32_t bit = 1u << s;
    const uint32_t old = atomicAnd(v.masks + b, ~bit);
    if (old & bit) {
      if (atomicCAS(v.buckets + static_cast<uint64_t>(b) * kS32 + s, kEmpty32, word) == kEmpty32)
        return true;
      fm = ld_relaxed32(v.masks + b);
    } else {
      fm = old;
    }
  }
  return false;
}

__device__ __forceinline__ bool stash32_find(const View32& v, uint32_t stash_n, uint32_t key,
                                             uint32_t& pos) {
  uint32_t lo = 0, hi = stash_n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(v.stash_keys + mid) < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  pos = lo;
  return lo < stash_n && __ldg(v.stash_keys + lo) == key;
}

// Acts on a found word `cur` in slot sp of bucket b (or in the stash when
// b == kNoOp): find, erase or replace.
template <int LAYOUT>
__device__ __forceinline__ void act32(const View32& v, uint32_t opk, uint32_t* sp, uint32_t b,
                                      uint32_t slot, uint32_t cur, uint32_t key, uint32_t val,
                                      uint8_t& st, uint32_t& outv, Counters32& cnt) {
  using E = E32<LAYOUT>;
  if (opk == OP_FIND) {
    outv = E::val(cur);
    st = ST_FOUND;
  } else if (opk == OP_ERASE) {
    st = ST_ERASED;
    if (atomicCAS(sp, cur, kEmpty32) == cur) {
      if (b != kNoOp)
        atomicOr(v.masks + b, 1u << slot);
      else
        atomicExch(&v.ctrl->stash_dirty, 1u);
      cnt.size_delta -= 1;
    } else {
      cnt.contract = true;
    }
  } else {
    st = ST_REPLACED;
    const uint32_t nw = E::pack(key, val);
    if (nw == cur || atomicCAS(sp, cur, nw) == cur)
      cnt.replaced += 1;
    else
      cnt.contract = true;
  }
}

// Ops [32c, 32c + 32) of a batch.
template <int MODE, int LAYOUT>
__device__ __forceinline__ void run_chunk32(const View32& v, uint32_t stash_n, const Ops32 a,
                                            uint32_t c, uint64_t n, const List32 ovf,
                                            Counters32& cnt, Stage32& sg, int lane) {
  using E = E32<LAYOUT>;
  constexpr bool kIns = (MODE == kModeInsert || MODE == kModeMixed);
  const uint32_t i = (c << 5) + lane;
  const bool valid = i < n;
  uint32_t op = MODE == kModeMixed ? (valid ? static_cast<uint32_t>(__ldcs(a.ops + i)) : OP_FIND)
                                   : (MODE == kModeFind    ? OP_FIND
                                      : MODE == kModeErase ? OP_ERASE
                                                           : OP_INSERT);
  if (op > OP_ERASE) op = OP_FIND;
  const uint32_t key = valid ? __ldcs(a.keys + i) : 0u;
  uint32_t val = 0;
  if (kIns && valid && op == OP_INSERT && a.vals) val = __ldcs(a.vals + i);
  const bool reserved = valid && E::reserved(key, op == OP_INSERT ? val : 0u);
  const bool live = valid && !reserved;
  cnt.reserved |= reserved;
  const uint32_t b1 = lh_bucket(bithash1(key), v.M, v.p);
  const uint32_t b2 = lh_bucket(bithash2(key), v.M, v.p);
  bool done = !live;
  uint8_t st = reserved ? ST_RESERVED : ST_NOT_FOUND;
  uint32_t outv = 0;
  uint32_t m1 = 0, m2 = 0;

  unsigned need = __ballot_sync(kFull, !done);
  if (need) {
    const bool mine = !done;
    if (kIns && mine && op == OP_INSERT) {
      m1 = ld_relaxed32(v.masks + b1);
      m2 = ld_relaxed32(v.masks + b2);
    }
    if (MODE == kModeInsert) {
      // both buckets of every op in one staged round
      cnt.probes += 2 * __popc(need);
      if (!sg.dead && stage32_round<true>(v, sg, need, b1, b2, lane)) {
        if (mine) {
          // buffer buckets 2 lane (BitHash1) and 2 lane + 1 (BitHash2)
          int ms = scan32<LAYOUT>(sg.buf + 2 * lane * kS32, key, lane);
          if (ms < 0) {
            const int m2 = scan32<LAYOUT>(sg.buf + (2 * lane + 1) * kS32, key, lane);
            if (m2 >= 0) ms = kS32 + m2;
          }
          if (ms >= 0) {
            done = true;
            const uint32_t b = ms < kS32 ? b1 : b2;
            const uint32_t slot = ms & (kS32 - 1);
            act32<LAYOUT>(v, OP_INSERT, v.buckets + static_cast<uint64_t>(b) * kS32 + slot, b,
                          slot, sg.buf[2 * lane * kS32 + ms], key, val, st, outv, cnt);
          }
        }
      } else if (mine) {
        for (int w = 0; w < 2 && !done; ++w) {
          const uint32_t b = w ? b2 : b1;
          const uint32_t* B = v.buckets + static_cast<uint64_t>(b) * kS32;
          const int ms = scan32_global<LAYOUT>(B, key);
          if (ms >= 0) {
            done = true;
            act32<LAYOUT>(v, OP_INSERT, const_cast<uint32_t*>(B) + ms, b, ms,
                          ld_relaxed32(B + ms), key, val, st, outv, cnt);
          }
        }
      }
    } else {
      // BitHash1 bucket, then the BitHash2 bucket of the ops still open
#pragma unroll 1
      for (int w = 0; w < 2; ++w) {
        const uint32_t myb = w ? b2 : b1;
        need = __ballot_sync(kFull, !done);
        if (!need) break;
        cnt.probes += __popc(need);
        const bool open = !done;
        int ms = -1;
        uint32_t cur = 0;
        if (!sg.dead && stage32_round<false>(v, sg, need, myb, 0, lane)) {
          if (open) {
            ms = scan32<LAYOUT>(sg.buf + lane * kS32, key, lane);
            if (ms >= 0) cur = sg.buf[lane * kS32 + ms];
          }
        } else if (open) {
          const uint32_t* B = v.buckets + static_cast<uint64_t>(myb) * kS32;
          ms = scan32_global<LAYOUT>(B, key);
          if (ms >= 0) cur = ld_relaxed32(B + ms);
        }
        if (open && ms >= 0) {
          done = true;
          act32<LAYOUT>(v, op, v.buckets + static_cast<uint64_t>(myb) * kS32 + ms, myb, ms, cur,
                        key, val, st, outv, cnt);
        }
      }
    }
  }

  // the stash (step 4) holds keys that found no bucket room
  if (!done && stash_n) {
    uint32_t pos;
    if (stash32_find(v, stash_n, key, pos)) {
      const uint32_t w = ld_relaxed32(v.stash_kv + pos);
      if (w != kEmpty32 && E::key(w) == key) {
        done = true;
        act32<LAYOUT>(v, op, v.stash_kv + pos, kNoOp, 0, w, key, val, st, outv, cnt);
      }
    }
  }

  // step 2: claim for absent keys, the bucket with more free slots first
  bool to_ovf = false;
  if (kIns && !done && op == OP_INSERT) {
    const uint32_t word = E::pack(key, val);
    const uint32_t f1 = __popc(m1), f2 = __popc(m2);
    const bool first1 = f1 >= f2;
    const uint32_t tb = first1 ? b1 : b2, tm = first1 ? m1 : m2;
    const uint32_t ob = first1 ? b2 : b1, om = first1 ? m2 : m1;
    bool placed = false;
    if (tm) placed = claim32(v, tb, __ffs(tm) - 1, word);
    if (!placed && om && ob != tb) placed = claim32(v, ob, __ffs(om) - 1, word);
    if (placed) {
      st = ST_INSERTED;
      cnt.size_delta += 1;
      cnt.claimed += 1;
    } else {
      to_ovf = true;
      cnt.overflowed += 1;
    }
  }
  if (kIns) {
    const unsigned om = __ballot_sync(kFull, to_ovf);
    if (om) {
      const int leader = __ffs(om) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(ovf.count, static_cast<unsigned>(__popc(om)));
      base = __shfl_sync(kFull, base, leader);
      if (to_ovf) {
        const unsigned r = base + __popc(om & ((1u << lane) - 1u));
        ovf.words[r] = E::pack(key, val);
        ovf.idx[r] = i;
      }
    }
  }
  if (valid) {
    if (MODE == kModeFind) {
      if (a.vals_out) __stcs(a.vals_out + i, outv);
      if (a.found) a.found[i] = st == ST_FOUND ? 1 : 0;
    } else {
      if (a.status && !to_ovf) a.status[i] = st;
      if (MODE == kModeMixed && a.vals_out) __stcs(a.vals_out + i, outv);
    }
  }
}

template <int MODE, int LAYOUT>
__global__ void __launch_bounds__(kOps32Threads, MODE == kModeInsert ? 3 : 4)
    k32_ops(View32 v, Ops32 a, uint64_t n, List32 ovf) {
  extern __shared__ __align__(16) uint64_t smem32[];
  const int lane = threadIdx.x & 31;
  const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t nchunks = static_cast<uint32_t>((n + 31) >> 5);
  const uint32_t stash_n = v.ctrl->stash_n;
  Stage32 sg = stage32_init(smem32, threadIdx.x >> 5, lane, stage32_words(MODE));
  Counters32 cnt;
  for (uint32_t c = warp0; c < nchunks; c += nwarps)
    run_chunk32<MODE, LAYOUT>(v, stash_n, a, c, n, ovf, cnt, sg, lane);
  stage32_drain(sg);
  flush32(v, cnt, lane);
}

// ---- steps 3-4 -------------------------------------------------------------

struct Ovf32 {
  unsigned claim = 0, rounds = 0, locks = 0, to = 0, stash = 0, pend = 0, added = 0;
  bool reserved = false;
};

__device__ __forceinline__ bool lock32(const View32& v, uint32_t b) {
  for (uint32_t t = 0; t < v.lock_spin_limit; ++t) {
    if (atomicCAS(v.locks + b, 0u, 1u) == 0u) return true;
    __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ bool stash32_reserve(const View32& v) {
  const uint32_t limit = v.lock_spin_limit * 4u;
  for (uint32_t t = 0; t < limit; ++t) {
    const unsigned c = atomicAdd(&v.ctrl->stash_claims, 1u);
    if (c < v.stash_cap) return true;
    atomicSub(&v.ctrl->stash_claims, 1u);
    if (ld_relaxed32(&v.ctrl->stash_tail) >= v.stash_cap) return false;
    __nanosleep(256);
  }
  return false;
}

// One overflowing insert, warp-wide (lane i holds slot i of the bucket in
// hand).  Mirrors the 64-bit eviction kernel: claim, else a bounded chain of
// locked exchanges with a lookahead victim, else the stash, else FULL.
template <int LAYOUT>
__device__ __forceinline__ void overflow32_item(const View32& v, uint32_t word0, uint32_t idx,
                                                uint8_t* status, Ovf32& oc, int lane) {
  using E = E32<LAYOUT>;
  const uint32_t key0 = E::key(word0);
  const uint32_t b1 = lh_bucket(bithash1(key0), v.M, v.p);
  const uint32_t b2 = lh_bucket(bithash2(key0), v.M, v.p);
  int outcome = 0;  // 0: evict, 1: placed, 2: stashed, 3: no room
  if (lane == 0) {
    const uint32_t m1 = ld_relaxed32(v.masks + b1);
    const uint32_t m2 = ld_relaxed32(v.masks + b2);
    if ((m1 && claim32_cas(v, b1, word0)) || (b2 != b1 && m2 && claim32_cas(v, b2, word0))) {
      outcome = 1;
      ++oc.claim;
    } else {
      if (!oc.reserved) oc.reserved = stash32_reserve(v);
      if (!oc.reserved) outcome = 3;
    }
  }
  outcome = __shfl_sync(kFull, outcome, 0);
  if (outcome == 0) {
    uint32_t cur = word0, b = b1;
    bool placed = false;
    for (uint32_t r = 0; r < v.max_evictions; ++r) {
      const uint32_t w = ld_relaxed32(v.buckets + static_cast<uint64_t>(b) * kS32 + lane);
      uint32_t am = 0;
      if (w != kEmpty32) {
        const uint32_t k = E::key(w);
        const uint32_t a1 = lh_bucket(bithash1(k), v.M, v.p);
        const uint32_t a2 = lh_bucket(bithash2(k), v.M, v.p);
        const uint32_t alt = (a1 == b) ? a2 : a1;
        if (alt != b) am = ld_relaxed32(v.masks + alt);
      }
      const unsigned gm = __ballot_sync(kFull, am != 0u);
      const bool has_empty = __ballot_sync(kFull, w == kEmpty32) != 0u;
      const uint32_t vs = gm ? static_cast<uint32_t>(__ffs(gm) - 1)
                             : ((bithash2(E::key(cur)) + r) & (kS32 - 1));
      const uint32_t vmask = __shfl_sync(kFull, am, vs);
      int res = 0;
      uint32_t victim = kEmpty32;
      if (lane == 0) {
        ++oc.rounds;
        if (!lock32(v, b)) {
          res = 2;
          ++oc.to;
        } else {
          ++oc.locks;
          if (has_empty && claim32_cas(v, b, cur)) {
            res = 1;
          } else {
            victim = atomicExch(v.buckets + static_cast<uint64_t>(b) * kS32 + vs, cur);
            res = (victim == kEmpty32) ? 1 : 0;
          }
          atomicExch(v.locks + b, 0u);
        }
      }
      res = __shfl_sync(kFull, res, 0);
      victim = __shfl_sync(kFull, victim, 0);
      if (res == 1) {
        placed = true;
        break;
      }
      if (res == 2) break;
      cur = victim;
      const uint32_t kc = E::key(cur);
      const uint32_t a1 = lh_bucket(bithash1(kc), v.M, v.p);
      const uint32_t a2 = lh_bucket(bithash2(kc), v.M, v.p);
      const uint32_t nb = (a1 == b) ? a2 : a1;
      if (nb == b) break;
      b = nb;
      int ok = 0;
      if (lane == 0) ok = claim32_cas(v, b, cur, vmask);
      if (__shfl_sync(kFull, ok, 0)) {
        placed = true;
        break;
      }
    }
    if (lane == 0) {
      if (placed && oc.reserved && ld_relaxed32(&v.ctrl->stash_claims) >= v.stash_cap) {
        atomicSub(&v.ctrl->stash_claims, 1u);
        oc.reserved = false;
      }
      if (!placed) {
        oc.reserved = false;
        const unsigned pos = atomicAdd(&v.ctrl->stash_tail, 1u);
        st_relaxed32(v.stash_kv + pos, cur);
        ++oc.stash;
      }
    }
    outcome = placed ? 1 : 2;
  }
  if (lane == 0) {
    if (outcome == 3) {
      ++oc.pend;
      atomicOr(&v.ctrl->err, kErrFull);
      if (status) status[idx] = ST_FULL;
    } else {
      ++oc.added;
      if (status) status[idx] = ST_INSERTED;
    }
  }
}

template <int LAYOUT>
__global__ void __launch_bounds__(256) k32_overflow(View32 v, List32 in, uint8_t* status) {
  const int lane = threadIdx.x & 31;
  const unsigned warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
  const unsigned total = *in.count;
  Ovf32 oc;
  for (unsigned it = warp0; it < total; it += nwarps)
    overflow32_item<LAYOUT>(v, in.words[it], in.idx[it], status, oc, lane);
  if (lane == 0) {
    Ctrl* c = v.ctrl;
    if (oc.reserved) atomicSub(&c->stash_claims, 1u);
    if (oc.added) atomicAdd(&c->size, static_cast<unsigned long long>(oc.added));
    if (oc.claim) atomicAdd(&c->stats[kStClaimedSlow], static_cast<unsigned long long>(oc.claim));
    if (oc.rounds) atomicAdd(&c->stats[kStEvictRounds], static_cast<unsigned long long>(oc.rounds));
    if (oc.locks) atomicAdd(&c->stats[kStLockAcquired], static_cast<unsigned long long>(oc.locks));
    if (oc.to) {
      atomicAdd(&c->stats[kStLockTimeouts], static_cast<unsigned long long>(oc.to));
      atomicOr(&c->err, kErrTimeout);
    }
    if (oc.stash) atomicAdd(&c->stats[kStStashed], static_cast<unsigned long long>(oc.stash));
    if (oc.pend) atomicAdd(&c->stats[kStPending], static_cast<unsigned long long>(oc.pend));
  }
}

// ---- stash maintenance (single CTA) -----------------------------------------

template <int LAYOUT>
__device__ __forceinline__ uint64_t sort_key32(uint32_t w) {
  // EMPTY sorts last
  return w == kEmpty32 ? ~0ull : static_cast<uint64_t>(E32<LAYOUT>::key(w));
}

template <int LAYOUT>
__device__ void bitonic32(uint32_t* a, unsigned P) {
  for (unsigned k = 2; k <= P; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      for (unsigned t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
        const unsigned low = t & (j - 1);
        const unsigned i = ((t - low) << 1) | low;
        const unsigned l = i | j;
        const uint32_t x = a[i], y = a[l];
        const bool up = (i & k) == 0;
        if ((sort_key32<LAYOUT>(x) > sort_key32<LAYOUT>(y)) == up) {
          a[i] = y;
          a[l] = x;
        }
      }
      __syncthreads();
    }
  }
}

template <int LAYOUT>
__global__ void __launch_bounds__(kMaint32Threads) k32_maint(View32 v) {
  extern __shared__ uint32_t smem_m32[];
  using E = E32<LAYOUT>;
  __shared__ unsigned s_reins, s_live;
  Ctrl* c = v.ctrl;
  const unsigned tail = c->stash_tail;
  const unsigned sorted = c->stash_n;
  const unsigned dirty = c->stash_dirty;
  if (threadIdx.x == 0) {
    s_reins = 0;
    s_live = 0;
    c->ovf_n = 0;
  }
  __syncthreads();
  if (tail == sorted && !dirty) return;
  unsigned reins = 0;
  for (unsigned j = threadIdx.x; j < tail; j += blockDim.x) {
    const uint32_t w = v.stash_kv[j];
    if (w == kEmpty32) continue;
    const uint32_t k = E::key(w);
    const uint32_t b1 = lh_bucket(bithash1(k), v.M, v.p);
    const uint32_t b2 = lh_bucket(bithash2(k), v.M, v.p);
    const uint32_t m1 = ld_relaxed32(v.masks + b1);
    bool ok = m1 && claim32(v, b1, __ffs(m1) - 1, w);
    if (!ok) {
      const uint32_t m2 = ld_relaxed32(v.masks + b2);
      ok = m2 && claim32(v, b2, __ffs(m2) - 1, w);
    }
    if (ok) {
      v.stash_kv[j] = kEmpty32;
      ++reins;
    }
  }
  if (reins) atomicAdd(&s_reins, reins);
  __syncthreads();
  unsigned P = 1;
  while (P < tail) P <<= 1;
  if (P <= kMaint32SmemWords) {
    for (unsigned j = threadIdx.x; j < P; j += blockDim.x)
      smem_m32[j] = j < tail ? v.stash_kv[j] : kEmpty32;
    __syncthreads();
    bitonic32<LAYOUT>(smem_m32, P);
    for (unsigned j = threadIdx.x; j < P; j += blockDim.x) v.stash_kv[j] = smem_m32[j];
  } else {
    bitonic32<LAYOUT>(v.stash_kv, P);  // [tail, P) is EMPTY by construction
  }
  __syncthreads();
  unsigned live = 0;
  for (unsigned j = threadIdx.x; j < P; j += blockDim.x) {
    const uint32_t w = v.stash_kv[j];
    if (w != kEmpty32) {
      v.stash_keys[j] = E::key(w);
      ++live;
    }
  }
  if (live) atomicAdd(&s_live, live);
  __syncthreads();
  if (threadIdx.x == 0) {
    c->stash_n = s_live;
    c->stash_tail = s_live;
    c->stash_claims = s_live;
    c->stash_dirty = 0;
    if (s_reins) c->stats[kStStashReinserted] += s_reins;
  }
}

// Resident blocks per SM of each bulk kernel, per layout and mode (set once
// per process by setup32; every GPU of the machine is the same model).
int g_occ32[2][4] = {{1, 1, 1, 1}, {1, 1, 1, 1}};

template <int MODE, int LAYOUT>
cudaError_t launch32_t(const View32& v, const Ops32& a, uint64_t n, const List32& ovf,
                       int num_sms, cudaStream_t s) {
  const uint64_t chunks = (n + 31) / 32;
  uint64_t blocks = (chunks + (kOps32Threads / 32) - 1) / (kOps32Threads / 32);
  const uint64_t cap = static_cast<uint64_t>(num_sms) * g_occ32[LAYOUT][MODE];
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  k32_ops<MODE, LAYOUT><<<static_cast<unsigned>(blocks), kOps32Threads, stage32_smem(MODE), s>>>(
      v, a, n, ovf);
  return cudaGetLastError();
}

template <int LAYOUT>
cudaError_t launch32_l(int mode, const View32& v, const Ops32& a, uint64_t n, const List32& ovf,
                       int num_sms, cudaStream_t s) {
  switch (mode) {
    case kModeFind:
      return launch32_t<kModeFind, LAYOUT>(v, a, n, ovf, num_sms, s);
    case kModeInsert:
      return launch32_t<kModeInsert, LAYOUT>(v, a, n, ovf, num_sms, s);
    case kModeErase:
      return launch32_t<kModeErase, LAYOUT>(v, a, n, ovf, num_sms, s);
    default:
      return launch32_t<kModeMixed, LAYOUT>(v, a, n, ovf, num_sms, s);
  }
}

template <int MODE, int LAYOUT>
cudaError_t setup32_mode() {
  const int smem = static_cast<int>(stage32_smem(MODE));
  cudaError_t e = cudaFuncSetAttribute(k32_ops<MODE, LAYOUT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int b = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k32_ops<MODE, LAYOUT>, kOps32Threads,
                                                      stage32_smem(MODE));
  g_occ32[LAYOUT][MODE] = b > 0 ? b : 1;
  return e;
}

template <int LAYOUT>
cudaError_t setup32_l(int* blocks_per_sm) {
  cudaError_t e = setup32_mode<kModeFind, LAYOUT>();
  if (e == cudaSuccess) e = setup32_mode<kModeInsert, LAYOUT>();
  if (e == cudaSuccess) e = setup32_mode<kModeErase, LAYOUT>();
  if (e == cudaSuccess) e = setup32_mode<kModeMixed, LAYOUT>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k32_maint<LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kMaint32SmemWords * 4));
  *blocks_per_sm = g_occ32[LAYOUT][kModeInsert];
  return e;
}

}  // namespace

cudaError_t launch32_ops(int mode, const View32& v, const Ops32& a, uint64_t n, const List32& ovf,
                         int num_sms, cudaStream_t s) {
  return v.layout == HIVE32_KEY_ONLY
             ? launch32_l<HIVE32_KEY_ONLY>(mode, v, a, n, ovf, num_sms, s)
             : launch32_l<HIVE32_KEY16_VAL16>(mode, v, a, n, ovf, num_sms, s);
}

cudaError_t launch32_overflow(const View32& v, const List32& in, uint8_t* status, int blocks,
                              cudaStream_t s) {
  if (v.layout == HIVE32_KEY_ONLY)
    k32_overflow<HIVE32_KEY_ONLY><<<blocks, 256, 0, s>>>(v, in, status);
  else
    k32_overflow<HIVE32_KEY16_VAL16><<<blocks, 256, 0, s>>>(v, in, status);
  return cudaGetLastError();
}

cudaError_t launch32_maint(const View32& v, cudaStream_t s) {
  const size_t smem = kMaint32SmemWords * 4;
  if (v.layout == HIVE32_KEY_ONLY)
    k32_maint<HIVE32_KEY_ONLY><<<1, kMaint32Threads, smem, s>>>(v);
  else
    k32_maint<HIVE32_KEY16_VAL16><<<1, kMaint32Threads, smem, s>>>(v);
  return cudaGetLastError();
}

cudaError_t setup32(int layout, int* blocks_per_sm) {
  return layout == HIVE32_KEY_ONLY ? setup32_l<HIVE32_KEY_ONLY>(blocks_per_sm)
                                   : setup32_l<HIVE32_KEY16_VAL16>(blocks_per_sm);
}

}  // namespace hive
