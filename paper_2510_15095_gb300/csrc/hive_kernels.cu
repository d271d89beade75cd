// Hive hash table kernels for GB300 (sm_103a).
//
// Layout (Section III-A/B of the paper): a bucket is S packed 64-bit words
// (value << 32 | key), S = 32 (256 bytes) or 16 (128 bytes), aligned to its
// size; a 32-bit free mask per bucket (bit i set = slot i free); a 32-bit lock
// per bucket used only by eviction; an overflow stash of packed words.  The
// empty word is all ones (key 0xFFFFFFFF).
//
// Kernels:
//   k_ops<MODE,S>  bulk find / insert (steps 1-2) / erase / mixed batch.  A
//                  warp takes 32 ops.  Staged: each probe round copies the
//                  buckets of all 32 ops into the warp's shared-memory buffer
//                  (cp.async for 128-byte buckets, one bulk copy per 256-byte
//                  bucket) and each lane scans its own op's buckets.  Direct:
//                  L = S/2 lanes read a bucket as 16-byte fragments, and
//                  match-and-elect (WCME, Section III-F) is a ballot over the
//                  fragments.  New keys claim a slot with one atomicAnd on the
//                  free mask (WABC, Section III-E), the free slot predicted from
//                  the probe round.
//   k_overflow<S>  steps 3-4 for inserts whose two buckets were full: warp per
//                  item, bounded cuckoo eviction under the bucket lock
//                  (Algorithm 3), then the stash.
//   k_maint<S>     stash maintenance: reinsert stash words into buckets that
//                  have room, compact, sort by key (lookups binary-search it).
//   k_split<S>     linear-hashing expansion, warp per bucket pair (Section IV-C1).
//   k_merge<S>     linear-hashing contraction, warp per bucket pair (IV-C2).
//   k_fused<S>     a mixed batch as one concurrent kernel (bucket versions make
//                  lookups safe against eviction chains in flight).
//   k_multi_*      the same phases over many tables in one launch each.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hive_internal.h"
#include "hive_device.cuh"

namespace hive {
namespace {

constexpr int kOpsThreads = 256;
#ifndef HIVE_MULTI_MIN_BLOCKS
#define HIVE_MULTI_MIN_BLOCKS 3  // the multi-table bulk kernel also holds a table view per warp
#endif
// Bulk-kernel modes (bit kModeFind, kModeInsert, ...) whose probes are staged
// in shared memory, per bucket width; the others load
// fragments straight from global memory with the warp-wide match-and-elect.
// Measured on the 2^26-slot, 95%-load bench workload, staging wins for
// every mode at both widths (with the copy path chosen below per width).
#ifndef HIVE_STAGED_MODES_S16
#define HIVE_STAGED_MODES_S16 0xF
#endif
#ifndef HIVE_STAGED_MODES_S32
#define HIVE_STAGED_MODES_S32 0xF
#endif
// How a staged round copies its buckets, per bucket width: 1 = cp.async
// through the load/store path (16 bytes per lane, coalesced per bucket),
// 0 = one bulk copy (TMA) per bucket.  Measured on the bench workload, the
// load/store path wins for 128-byte buckets (S = 16 finds 30.1 against 27.7
// Gops/s) and bulk copies win for 256-byte buckets (S = 32 inserts 11.7
// against 11.0).
#ifndef HIVE_STAGE_LSU_S16
#define HIVE_STAGE_LSU_S16 1
#endif
#ifndef HIVE_STAGE_LSU_S32
#define HIVE_STAGE_LSU_S32 0
#endif
// Where the paired insert round takes the free slots that steer its claims:
// 1 = the EMPTY words of the staged buckets (no mask reads), 0 = the two
// free masks, read while the copies are in flight.
#ifndef HIVE_FREE_FROM_STAGE
#define HIVE_FREE_FROM_STAGE 1
#endif
#ifndef HIVE_STAGED_SMALL_MIN_BLOCKS
#define HIVE_STAGED_SMALL_MIN_BLOCKS 4  // 32 KB of staging per block (S = 16 single rounds)
#endif
#ifndef HIVE_STAGED_MIN_BLOCKS
#define HIVE_STAGED_MIN_BLOCKS 3  // 64 KB of staging per block: three blocks fit an SM
#endif
#ifndef HIVE_OPS_MIN_BLOCKS
#define HIVE_OPS_MIN_BLOCKS 4  // resident 256-thread blocks per SM the bulk kernel is built for
#endif
constexpr int kOvfThreads = 256;
__host__ __device__ constexpr bool staged_mode(int mode, int S) {
  return ((S == 16 ? HIVE_STAGED_MODES_S16 : HIVE_STAGED_MODES_S32) >> mode) & 1;
}
constexpr int kMaintThreads = 1024;
constexpr unsigned kMaintSmemWords = 8192;  // 64 KB of words sorted in shared memory

// ----------------------------------------------------------------------------
// Hashing and addressing
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint64_t pack(uint32_t k, uint32_t v) {
  return (static_cast<uint64_t>(v) << 32) | k;
}
__device__ __forceinline__ uint32_t key_of(uint64_t w) { return static_cast<uint32_t>(w); }
__device__ __forceinline__ uint32_t val_of(uint64_t w) { return static_cast<uint32_t>(w >> 32); }

// ----------------------------------------------------------------------------
// Memory access helpers
// ----------------------------------------------------------------------------

// 16-byte bucket fragment through the read-only path (table not written by
// the running kernel).
__device__ __forceinline__ void ld_frag_ro(const uint64_t* p, uint64_t& a, uint64_t& b) {
  asm("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}
// 16-byte bucket fragment while other warps may be writing the table.
__device__ __forceinline__ void ld_frag(const uint64_t* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.relaxed.gpu.global.L1::no_allocate.v2.u64 {%0, %1}, [%2];"
               : "=l"(a), "=l"(b)
               : "l"(p)
               : "memory");
}

// ----------------------------------------------------------------------------
// Slot claims (WABC, Section III-E / Algorithm 2)
// ----------------------------------------------------------------------------

// Claim a free slot of bucket b starting from the predicted slot `s`, then
// publish `word` with a plain store.  Used where no eviction runs concurrently
// (the bulk kernel and maintenance).  Algorithm 2 restores the bit with
// fetch_or when the fetch_and finds it already clear; that would free a slot
// another warp owns, so here a failed claim retries on the returned mask.
template <int S>
__device__ __forceinline__ bool claim_store(const View& v, uint32_t b, uint32_t s,
                                            uint64_t word) {
  for (int t = 0; t <= S && s < S; ++t) {
    const uint32_t bit = 1u << s;
    const uint32_t old = atomicAnd(v.masks + b, ~bit);
    if (old & bit) {
      st_relaxed64(v.buckets + static_cast<uint64_t>(b) * S + s, word);
      return true;
    }
    s = old ? static_cast<uint32_t>(__ffs(old) - 1) : S;
  }
  return false;
}

// The claim of the eviction kernel and of the single-kernel batch: fetch_and
// on the free mask, then a plain store.  The bit makes the slot the
// claimer's, and nothing else writes a slot while it is EMPTY: in the
// eviction phase slots only go from EMPTY to occupied (there are no erases)
// and a chain exchanges only a slot it saw occupied; in the single-kernel
// batch every other write to a bucket word is a CAS whose expected word is
// not EMPTY (an erase's, a replace's, a chain's swap).  `hint`: a free mask
// of bucket b read moments ago, used as the first guess (the fetch_and result
// is the authority either way).
template <int S>
__device__ __forceinline__ bool claim_pub(const View& v, uint32_t b, uint64_t word,
                                          uint32_t hint = 0) {
  uint32_t fm = hint ? hint : ld_relaxed32(v.masks + b);
  for (int t = 0; t <= S && fm; ++t) {
    const uint32_t s = __ffs(fm) - 1;
    const uint32_t bit = 1u << s;
    const uint32_t old = atomicAnd(v.masks + b, ~bit);
    if (old & bit) {
      st_relaxed64(v.buckets + static_cast<uint64_t>(b) * S + s, word);
      return true;
    }
    fm = old;
  }
  return false;
}

// The bucket lock serialises evictors of one bucket (Algorithm 3).  Every
// access it protects is an L2 atomic whose result has returned before the
// unlock issues, so neither side needs a fence.
__device__ __forceinline__ bool lock_bucket(const View& v, uint32_t b) {
  for (uint32_t t = 0; t < v.lock_spin_limit; ++t) {
    if (atomicCAS(v.locks + b, 0u, 1u) == 0u) return true;
    __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void unlock_bucket(const View& v, uint32_t b) {
  atomicExch(v.locks + b, 0u);
}

// Stash binary search over the sorted key prefix.
__device__ __forceinline__ bool stash_find(const View& v, uint32_t stash_n, uint32_t key,
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

// ----------------------------------------------------------------------------
// Bulk op kernel
// ----------------------------------------------------------------------------

struct LaneCounters {
  int size_delta = 0;
  unsigned replaced = 0, claimed = 0, overflowed = 0, stash_lookups = 0;
  unsigned probes = 0;  // warp-uniform: buckets probed by this warp
  bool reserved = false, contract = false;
};

// Lane geometry of a bucket of S slots read as 16-byte fragments: L lanes per
// bucket, Q buckets per load instruction.
template <int S>
struct Geo {
  static constexpr int L = S / 2;
  static constexpr int Q = 32 / L;
  static constexpr unsigned LM = (L >= 32) ? 0xFFFFFFFFu : ((1u << L) - 1u);
};

// ---- Shared-memory staging of bucket reads ----
//
// A kernel that stages its probes gives each warp one mbarrier and a buffer
// (stage_words() below): every bucket a probe round needs -- the 32 ops'
// buckets of a single-bucket round, or both candidate buckets of 32 (S = 16)
// or 16 (S = 32) ops of a paired round -- is copied in before any compare, so
// the warp has all of them in flight at once without holding registers.
// 128-byte buckets are copied with 16-byte cp.async through the load/store
// path (stage_issue_lsu); 256-byte buckets with one bulk copy (TMA) each,
// counted by the barrier (stage_issue).  Each lane then scans its own op's
// buckets in shared memory.  A barrier wait that does not end within
// View::stage_spin_limit tries raises the table's sticky TIMEOUT error, marks
// the stage dead and redoes the round from global memory; before the warp
// exits it waits up to kMbarSpinLimit tries for the copies still in flight.
constexpr int kStageWords = 1024;
// Staging words of a paired insert round: both buckets of kPairWords / (2 S)
// ops per round (32 ops at S = 16 and 8 KB; fewer words split a chunk into
// more rounds and leave more of the SM's on-chip memory to L1)
#ifndef HIVE_PAIR_WORDS
#define HIVE_PAIR_WORDS 1024
#endif
constexpr int kPairWords = HIVE_PAIR_WORDS;
constexpr uint32_t kMbarSpinLimit = 1u << 22;

// Staging words a warp of mode MODE needs: a paired insert round fills the
// whole 8 KB; a single-bucket round holds 32 buckets (4 KB at S = 16), which
// lets four 256-thread blocks share an SM.
__host__ __device__ constexpr int stage_words(int mode, int S) {
  return mode == kModeInsert ? kPairWords : 32 * S;
}
// Shared-memory words per warp: its barrier, then its staging words.  (The
// 64 KB of a paired round's block keeps three blocks within a 196 KB
// shared-memory carveout, which leaves the L1 that the cp.async.ca copies go
// through 60 KB; three blocks of 68 KB need the largest carveout, and the
// insert kernel then ran at two-thirds speed.)
__host__ __device__ constexpr int warp_smem_words(int mode, int S) {
  return 2 + stage_words(mode, S);
}
__host__ __device__ constexpr size_t stage_smem(int mode, int S, int threads = kOpsThreads) {
  return static_cast<size_t>(threads / 32) * 8u * warp_smem_words(mode, S);
}
__host__ __device__ constexpr int staged_min_blocks(int mode, int S) {
  return (mode != kModeInsert && stage_words(mode, S) < kStageWords) ? HIVE_STAGED_SMALL_MIN_BLOCKS
                                                                     : HIVE_STAGED_MIN_BLOCKS;
}

struct Stage {
  uint64_t* bar;   // mbarrier
  uint64_t* buf;   // kStageWords words, 16-byte aligned
  uint32_t phase;  // parity of the barrier's current phase
  bool dead;       // a wait gave up: copies may still land, the buffer is not reused
};

// Sets up the calling warp's stage in the kernel's dynamic shared memory
// (`stride` words per warp: its barrier, then its staging words).
__device__ __forceinline__ Stage stage_init(uint64_t* smem, int warp_in_block, int lane,
                                            int stride = kStageWords + 2) {
  Stage sg;
  uint64_t* base = smem + static_cast<size_t>(warp_in_block) * stride;
  sg.bar = base;
  sg.buf = base + 2;
  sg.phase = 0;
  sg.dead = false;
  if (lane == 0) mbar_init(sg.bar, 1);
  __syncwarp();
  return sg;
}

// Before a warp exits: a stage whose wait gave up may still receive bytes;
// wait (bounded) for them so that no copy lands after the block has left.
__device__ __forceinline__ void stage_drain(Stage& sg) {
  if (!sg.dead) return;
  bool ok = false;
  for (uint32_t it = 0; it < kMbarSpinLimit && !ok; ++it) ok = mbar_try_wait(sg.bar, sg.phase ^ 1u);
}

// Issues the copies of one staged round and waits for them (warp-wide).
// PAIR = false: op j (bit j of `need`, j < 32) copies bucket x1 of lane j to
// buffer bucket j.  PAIR = true: ops [o0, o0 + 512 / S) copy buckets x1 and x2
// of their lanes to buffer buckets 2 (j - o0) and 2 (j - o0) + 1.  Returns
// false, with the stage marked dead and the error raised, if the wait gave up.
template <int S, bool PAIR>
__device__ __forceinline__ void stage_issue(const View& v, Stage& sg, unsigned need, int o0,
                                            uint32_t x1, uint32_t x2, int lane) {
  constexpr uint32_t kBucketBytes = S * 8u;
  fence_proxy_async();  // earlier fragment reads of the buffer come before the new copies
  __syncwarp();
  if (lane == 0) mbar_arrive_expect_tx(sg.bar, __popc(need) * (PAIR ? 2u : 1u) * kBucketBytes);
  __syncwarp();
  if (!PAIR) {
    if ((need >> lane) & 1u)
      bulk_g2s(sg.buf + lane * S, v.buckets + static_cast<uint64_t>(x1) * S, kBucketBytes, sg.bar);
  } else {
    constexpr int BO = kPairWords / (2 * S);
#pragma unroll
    for (int k = 0; k < (2 * BO + 31) / 32; ++k) {
      const int bi = lane + 32 * k;
      const int op = o0 + ((bi >> 1) & (BO - 1));
      const uint32_t y1 = __shfl_sync(kFull, x1, op & 31);
      const uint32_t y2 = __shfl_sync(kFull, x2, op & 31);
      if (bi < 2 * BO && ((need >> op) & 1u))
        bulk_g2s(sg.buf + bi * S, v.buckets + static_cast<uint64_t>((bi & 1) ? y2 : y1) * S,
                 kBucketBytes, sg.bar);
    }
  }
}

// Waits (bounded, warp-wide) for the copies of the round issued last.
// A limit below 16 polls without suspending (mbarrier.test_wait), so that a
// test can make the wait give up while the copies are certainly in flight.
__device__ __forceinline__ bool stage_wait(const View& v, Stage& sg, int lane) {
  bool ok = false;
  if (v.stage_spin_limit < 16) {
    for (uint32_t it = 0; it < v.stage_spin_limit && !ok; ++it) ok = mbar_test_wait(sg.bar, sg.phase);
  } else {
    for (uint32_t it = 0; it < v.stage_spin_limit && !ok; ++it) ok = mbar_try_wait(sg.bar, sg.phase);
  }
  sg.phase ^= 1u;
  if (__any_sync(kFull, !ok)) {  // never expected
    sg.dead = true;
    if (lane == 0) atomicOr(&v.ctrl->err, kErrTimeout);
    return false;
  }
  return true;
}

// The same round through the load/store path: the lanes of a group of L = S/2
// copy one bucket with 16-byte cp.async each, so one warp instruction moves
// 32 / L whole buckets, coalesced exactly as the direct probe loads them.
// stage_wait_lsu() then waits for the warp's copies (cp.async.wait_group)
// and syncs the warp.  No registers hold the data and no spin loop waits.
template <int S, bool PAIR>
__device__ __forceinline__ void stage_issue_lsu(const View& v, Stage& sg, unsigned need, int o0,
                                                uint32_t x1, uint32_t x2, int lane) {
  constexpr int L = Geo<S>::L, Q = Geo<S>::Q;  // lanes per bucket, buckets per instruction
  constexpr int NB = PAIR ? 2 * (kPairWords / (2 * S)) : 32;  // buckets per round
  const int q = lane / L, ql = lane % L;
  __syncwarp();  // earlier reads of the buffer by any lane come first
#pragma unroll 4
  for (int r = 0; r < NB / Q; ++r) {
    const int bi = Q * r + q;                  // buffer bucket of this lane group
    const int op = PAIR ? o0 + (bi >> 1) : bi;  // its op
    const uint32_t y1 = __shfl_sync(kFull, x1, op & 31);
    const uint32_t y2 = PAIR ? __shfl_sync(kFull, x2, op & 31) : 0u;
    const uint32_t b = (PAIR && (bi & 1)) ? y2 : y1;
    if ((need >> op) & 1u)
      cp_async16(sg.buf + bi * S + 2 * ql, v.buckets + static_cast<uint64_t>(b) * S + 2 * ql);
  }
  cp_async_commit();
}
__device__ __forceinline__ void stage_wait_lsu() {
  cp_async_wait_all();
  __syncwarp();
}

// A staged round in two halves, so that a caller can do other work while the
// copies are in flight: stage_begin() issues them on the path chosen for the
// bucket width, stage_end() waits (false: the wait gave up, see stage_wait).
template <int S, bool PAIR>
__device__ __forceinline__ void stage_begin(const View& v, Stage& sg, unsigned need, int o0,
                                            uint32_t x1, uint32_t x2, int lane) {
  if (S == 16 ? HIVE_STAGE_LSU_S16 : HIVE_STAGE_LSU_S32)
    stage_issue_lsu<S, PAIR>(v, sg, need, o0, x1, x2, lane);
  else
    stage_issue<S, PAIR>(v, sg, need, o0, x1, x2, lane);
}
template <int S>
__device__ __forceinline__ bool stage_end(const View& v, Stage& sg, int lane) {
  if (S == 16 ? HIVE_STAGE_LSU_S16 : HIVE_STAGE_LSU_S32) {
    stage_wait_lsu();
    return true;
  }
  return stage_wait(v, sg, lane);
}

template <int S, bool PAIR>
__device__ __forceinline__ bool stage_round(const View& v, Stage& sg, unsigned need, int o0,
                                            uint32_t x1, uint32_t x2, int lane) {
  stage_begin<S, PAIR>(v, sg, need, o0, x1, x2, lane);
  return stage_end<S>(v, sg, lane);
}

// One probe round over the 32 ops of a warp.  `need` has bit j set when op j
// (held by lane j, its home lane) must read bucket `myb` this round.  Load u
// (u = 0..3) of lane group q (L lanes) reads the bucket of op Q*u + q of the
// current group of 4Q ops, 16 bytes (two slots) per lane, so each load
// instruction probes Q buckets.  Match-and-elect (Section III-F) is a ballot per load: the lowest
// matching lane of a group is the winner, and one shuffle per load hands the
// matched value to every home lane, which then reads its own op's outcome out
// of the warp-uniform ballots.  A home lane that must update the matched slot
// (erase, replace) does the single CAS itself: the expected word is
// (value << 32 | key), both of which it now holds.
template <int MODE, int S>
__device__ __forceinline__ void probe(const View& v, unsigned need, uint32_t myb, uint32_t key,
                                      uint32_t val, uint32_t op, int lane, bool& done,
                                      uint8_t& st, uint32_t& outv, uint32_t& fcnt,
                                      uint32_t& fslot, LaneCounters& cnt) {
  constexpr bool kIns = (MODE == kModeInsert || MODE == kModeMixed);
  constexpr int L = Geo<S>::L, Q = Geo<S>::Q;
  constexpr unsigned LM = Geo<S>::LM;
  constexpr int G = 4 * Q;   // ops per group
  constexpr int NG = 32 / G; // groups per warp
  constexpr unsigned GM = (G >= 32) ? 0xFFFFFFFFu : ((1u << G) - 1u);
  const int q = lane / L;
  const int ql = lane % L;
  const int my_g = lane / G, my_j = lane % G, my_u = my_j / Q, my_q = my_j % Q;
#pragma unroll 1
  for (int g = 0; g < NG; ++g) {
    const unsigned gneed = (need >> (G * g)) & GM;
    if (!gneed) continue;
    uint64_t wa[4], wb[4];
    uint32_t kq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int src = G * g + Q * u + q;
      const uint32_t bq = __shfl_sync(kFull, myb, src);
      kq[u] = __shfl_sync(kFull, key, src);
      if ((gneed >> (Q * u + q)) & 1u) {
        const uint64_t* p = v.buckets + static_cast<uint64_t>(bq) * S + 2 * ql;
        if (MODE == kModeFind)
          ld_frag_ro(p, wa[u], wb[u]);
        else
          ld_frag(p, wa[u], wb[u]);
      } else {
        wa[u] = kEmptyWord;
        wb[u] = kEmptyWord;
      }
    }
    unsigned my_m = 0, my_mh = 0, my_el = 0, my_eh = 0;
    uint32_t got = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool lo = key_of(wa[u]) == kq[u];
      const bool hi = key_of(wb[u]) == kq[u];
      const unsigned m = __ballot_sync(kFull, lo || hi);
      const unsigned mh = (MODE != kModeFind) ? __ballot_sync(kFull, hi) : 0u;
      const unsigned el = kIns ? __ballot_sync(kFull, wa[u] == kEmptyWord) : 0u;
      const unsigned eh = kIns ? __ballot_sync(kFull, wb[u] == kEmptyWord) : 0u;
      const uint32_t cv = lo ? val_of(wa[u]) : val_of(wb[u]);
      const unsigned hm = (m >> (L * my_q)) & LM;
      const uint32_t x = __shfl_sync(kFull, cv, L * my_q + (hm ? __ffs(hm) - 1 : 0));
      if (u == my_u) {
        my_m = m;
        my_mh = mh;
        my_el = el;
        my_eh = eh;
        got = x;
      }
    }
    if (my_g == g && ((gneed >> my_j) & 1u)) {
      const unsigned hm = (my_m >> (L * my_q)) & LM;
      if (hm) {
        done = true;
        const uint32_t opk = MODE == kModeMixed
                                 ? op
                                 : (MODE == kModeFind ? OP_FIND
                                                      : (MODE == kModeErase ? OP_ERASE : OP_INSERT));
        if (opk == OP_FIND) {
          outv = got;
          st = ST_FOUND;
          done = true;
        } else {
          const uint32_t w = __ffs(hm) - 1;
          const uint32_t slot = 2 * w + ((my_mh >> (L * my_q + w)) & 1u);
          uint64_t* sp = v.buckets + static_cast<uint64_t>(myb) * S + slot;
          const uint64_t cur = pack(key, got);
          if (opk == OP_ERASE) {
            // Algorithm 4: CAS the slot to EMPTY, then publish the free bit.
            // The atomicOr issues only after the CAS has returned, so a
            // claimer that sees the bit finds the slot already EMPTY.
            if (atomicCAS(ull(sp), cur, kEmptyWord) == cur) {
              atomicOr(v.masks + myb, 1u << slot);
              cnt.size_delta -= 1;
              st = ST_ERASED;
            } else {
              st = ST_ERASED;
              cnt.contract = true;
            }
          } else {
            // Algorithm 1: CAS the cached word to the new pair.
            if (atomicCAS(ull(sp), cur, pack(key, val)) == cur) {
              cnt.replaced += 1;
              st = ST_REPLACED;
            } else {
              st = ST_REPLACED;
              cnt.contract = true;
            }
          }
        }
      } else if (kIns) {
        const unsigned ev = (my_el >> (L * my_q)) & LM;
        const unsigned od = (my_eh >> (L * my_q)) & LM;
        fcnt = __popc(ev) + __popc(od);
        const uint32_t se = ev ? 2u * (__ffs(ev) - 1) : S;
        const uint32_t so = od ? 2u * (__ffs(od) - 1) + 1u : S;
        fslot = se < so ? se : so;
      }
    }
  }
}

// Insert batches probe both candidate buckets of an op in one round: the two
// lane groups of a pair read the BitHash1 and the BitHash2 bucket of one op,
// P = Q / 2 ops per load instruction.  An insert of a new key needs both
// buckets anyway (step 1 must rule the key out of both before step 2 claims),
// so this halves the dependent probe rounds of the find-shaped probe() above.
// Covers the op groups of ops [o0, o1).  On a match the home lane replaces the value with one CAS
// (Algorithm 1); otherwise it records each bucket's free count and first
// free slot.
template <int S>
__device__ __forceinline__ void probe_pair(const View& v, unsigned need, uint32_t b1,
                                           uint32_t b2, uint32_t key, uint32_t val, int lane,
                                           bool& done, uint8_t& st, uint32_t& f1, uint32_t& s1,
                                           uint32_t& f2, uint32_t& s2, LaneCounters& cnt, int o0,
                                           int o1) {
  constexpr int L = Geo<S>::L, Q = Geo<S>::Q;
  constexpr unsigned LM = Geo<S>::LM;
  constexpr int P = Q / 2;    // ops per load instruction
  constexpr int G = 4 * P;    // ops per group
  constexpr unsigned GM = (1u << G) - 1u;
  constexpr unsigned PM = (2 * L >= 32) ? 0xFFFFFFFFu : ((1u << (2 * L)) - 1u);
  const int q = lane / L;
  const int ql = lane % L;
  const int my_g = lane / G, my_j = lane % G, my_u = my_j / P, my_p = my_j % P;
#pragma unroll 1
  for (int g = o0 / G; g < o1 / G; ++g) {
    const unsigned gneed = (need >> (G * g)) & GM;
    if (!gneed) continue;
    uint64_t wa[4], wb[4];
    uint32_t kq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int src = G * g + P * u + (q >> 1);
      const uint32_t q1 = __shfl_sync(kFull, b1, src);
      const uint32_t q2 = __shfl_sync(kFull, b2, src);
      kq[u] = __shfl_sync(kFull, key, src);
      if ((gneed >> (P * u + (q >> 1))) & 1u) {
        const uint64_t* p = v.buckets + static_cast<uint64_t>((q & 1) ? q2 : q1) * S + 2 * ql;
        ld_frag(p, wa[u], wb[u]);
      } else {
        wa[u] = kEmptyWord;
        wb[u] = kEmptyWord;
      }
    }
    unsigned my_m = 0, my_mh = 0, my_el = 0, my_eh = 0;
    uint32_t got = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool lo = key_of(wa[u]) == kq[u];
      const bool hi = key_of(wb[u]) == kq[u];
      const unsigned m = __ballot_sync(kFull, lo || hi);
      const unsigned mh = __ballot_sync(kFull, hi);
      const unsigned el = __ballot_sync(kFull, wa[u] == kEmptyWord);
      const unsigned eh = __ballot_sync(kFull, wb[u] == kEmptyWord);
      const uint32_t cv = lo ? val_of(wa[u]) : val_of(wb[u]);
      const unsigned pm = (m >> (2 * L * my_p)) & PM;
      const uint32_t x = __shfl_sync(kFull, cv, 2 * L * my_p + (pm ? __ffs(pm) - 1 : 0));
      if (u == my_u) {
        my_m = m;
        my_mh = mh;
        my_el = el;
        my_eh = eh;
        got = x;
      }
    }
    if (my_g == g && ((gneed >> my_j) & 1u)) {
      const int base = 2 * L * my_p;
      const unsigned pm = (my_m >> base) & PM;
      if (pm) {
        // the lowest matching lane: the BitHash1 group wins when both match
        done = true;
        st = ST_REPLACED;
        const uint32_t w = __ffs(pm) - 1;
        const uint32_t slot = 2 * (w % L) + ((my_mh >> (base + w)) & 1u);
        const uint32_t b = w < static_cast<uint32_t>(L) ? b1 : b2;
        uint64_t* sp = v.buckets + static_cast<uint64_t>(b) * S + slot;
        const uint64_t cur = pack(key, got);
        if (atomicCAS(ull(sp), cur, pack(key, val)) == cur)
          cnt.replaced += 1;
        else
          cnt.contract = true;
      } else {
        const unsigned e0 = (my_el >> base) & LM, o_0 = (my_eh >> base) & LM;
        const unsigned e1 = (my_el >> (base + L)) & LM, o_1 = (my_eh >> (base + L)) & LM;
        f1 = __popc(e0) + __popc(o_0);
        f2 = __popc(e1) + __popc(o_1);
        const uint32_t a0 = e0 ? 2u * (__ffs(e0) - 1) : S;
        const uint32_t a1 = o_0 ? 2u * (__ffs(o_0) - 1) + 1u : S;
        const uint32_t c0 = e1 ? 2u * (__ffs(e1) - 1) : S;
        const uint32_t c1 = o_1 ? 2u * (__ffs(o_1) - 1) + 1u : S;
        s1 = a0 < a1 ? a0 : a1;
        s2 = c0 < c1 ? c0 : c1;
      }
    }
  }
}

// An erase or replace CAS issued by a staged probe round, checked only at the
// end of the chunk, so that its round trip overlaps the rounds and claims
// after it (an op updates at most one slot, so one record per lane).
struct PendCas {
  uint64_t cur, old;
  uint32_t b, slot, kind;  // kind: 0 none, 1 erase, 2 replace
};

__device__ __forceinline__ void resolve_cas(const View& v, const PendCas& pc, LaneCounters& cnt) {
  if (pc.kind == 0) return;
  const bool ok = pc.old == pc.cur;
  if (pc.kind == 1) {
    // Algorithm 4: the free bit is published once the CAS has emptied the slot
    if (ok) {
      atomicOr(v.masks + pc.b, 1u << pc.slot);
      cnt.size_delta -= 1;
    } else {
      cnt.contract = true;
    }
  } else {
    if (ok)
      cnt.replaced += 1;
    else
      cnt.contract = true;
  }
}

// A single-bucket probe round on staged buckets, one op per lane: lane j
// scans buffer bucket j (its op's bucket this round) with swizzled 16-byte
// reads, as scan_staged_pair() below does for both buckets, and acts on a
// match exactly as probe() does.  `mask` is the bucket's free mask, read while
// the copies were in flight (insert-capable modes), for the claim.
template <int MODE, int S>
__device__ __forceinline__ void scan_staged_one(const View& v, const uint64_t* sbuf, int lane,
                                                uint32_t myb, uint32_t key, uint32_t val,
                                                uint32_t op, uint32_t mask, bool& done,
                                                uint8_t& st, uint32_t& outv, uint32_t& fcnt,
                                                uint32_t& fslot, PendCas& pc) {
  constexpr bool kIns = (MODE == kModeInsert || MODE == kModeMixed);
  constexpr int NP = S / 2;
  const uint64_t* B = sbuf + lane * S;
  int ms = -1;
#pragma unroll 8
  for (int k = 0; k < NP; ++k) {
    const int f = (k + lane) & (NP - 1);
    uint64_t a, b;
    lds_frag(B + 2 * f, a, b);
    if (key_of(a) == key) ms = 2 * f;
    if (key_of(b) == key) ms = 2 * f + 1;
  }
  if (ms >= 0) {
    done = true;
    const uint64_t cur = B[ms];
    const uint32_t opk = MODE == kModeMixed
                             ? op
                             : (MODE == kModeFind ? OP_FIND
                                                  : (MODE == kModeErase ? OP_ERASE : OP_INSERT));
    if (opk == OP_FIND) {
      outv = val_of(cur);
      st = ST_FOUND;
    } else {
      uint64_t* sp = v.buckets + static_cast<uint64_t>(myb) * S + ms;
      st = opk == OP_ERASE ? ST_ERASED : ST_REPLACED;
      pc.old = atomicCAS(ull(sp), cur, opk == OP_ERASE ? kEmptyWord : pack(key, val));
      pc.cur = cur;
      pc.b = myb;
      pc.slot = ms;
      pc.kind = opk == OP_ERASE ? 1u : 2u;
    }
  } else if (kIns) {
    fcnt = __popc(mask);
    fslot = mask ? __ffs(mask) - 1 : S;
  }
}

// A single-bucket probe round, staged when the warp has a live stage.
// CLAIM: the op may claim a slot in this kernel, so the round also reads the
// bucket's free mask.
template <int MODE, int S, bool CLAIM>
__device__ __forceinline__ void probe_round(const View& v, unsigned need, uint32_t myb,
                                            uint32_t key, uint32_t val, uint32_t op, int lane,
                                            bool& done, uint8_t& st, uint32_t& outv,
                                            uint32_t& fcnt, uint32_t& fslot, LaneCounters& cnt,
                                            Stage* sg, PendCas& pc) {
  if (sg && !sg->dead) {
    const bool mine = (need >> lane) & 1u;
    const uint32_t m = (CLAIM && mine && op == OP_INSERT) ? ld_relaxed32(v.masks + myb) : 0u;
    if (stage_round<S, false>(v, *sg, need, 0, myb, 0, lane)) {
      if (mine)
        scan_staged_one<MODE, S>(v, sg->buf, lane, myb, key, val, op, m, done, st, outv, fcnt,
                                 fslot, pc);
      return;
    }
  }
  probe<MODE, S>(v, need, myb, key, val, op, lane, done, st, outv, fcnt, fslot, cnt);
}

// The paired insert round on staged buckets, one op per lane.  With both
// candidate buckets of its op in shared memory, a lane scans them itself:
// S / 2 16-byte fragment reads per bucket, starting at fragment (op mod S / 2)
// so that the eight lanes of a shared-memory wavefront read eight different
// bank groups, and one compare per slot against the op's key (a key sits in
// at most one slot of the table).  Free counts and first free slots come from
// the EMPTY words of the staged buckets (HIVE_FREE_FROM_STAGE), or from the
// free masks read while the copies are in flight: either way they only steer
// the claim, whose fetch_and result is the authority (a slot claimed and not
// yet written still reads EMPTY; the claim then retries on the returned mask).  This
// takes a few instructions per slot where the warp-wide match-and-elect takes
// several ballots per 16-byte fragment, and the staged kernel is bound by
// instruction issue, not by memory.
template <int S>
__device__ __forceinline__ void scan_staged_pair(const View& v, const uint64_t* sbuf, int jj,
                                                 uint32_t b1, uint32_t b2, uint32_t key,
                                                 uint32_t val, uint32_t m1, uint32_t m2,
                                                 bool& done, uint8_t& st, uint32_t& f1,
                                                 uint32_t& s1, uint32_t& f2, uint32_t& s2,
                                                 LaneCounters& cnt) {
  constexpr int NP = S / 2;  // 16-byte fragments per bucket
  const uint64_t* B = sbuf + 2 * jj * S;
  int ms = -1;  // matched word in [0, 2S): bucket ms / S, slot ms % S
  uint32_t em[2] = {0u, 0u};  // EMPTY slots of each bucket
#pragma unroll
  for (int which = 0; which < 2; ++which) {
#pragma unroll 8
    for (int k = 0; k < NP; ++k) {
      const int f = (k + jj) & (NP - 1);
      uint64_t a, b;
      lds_frag(B + which * S + 2 * f, a, b);
      if (key_of(a) == key) ms = which * S + 2 * f;
      if (key_of(b) == key) ms = which * S + 2 * f + 1;
      if (HIVE_FREE_FROM_STAGE)
        em[which] |= ((key_of(a) == kEmptyKey ? 1u : 0u) | (key_of(b) == kEmptyKey ? 2u : 0u))
                     << (2 * f);
    }
  }
  if (HIVE_FREE_FROM_STAGE) {
    m1 = em[0];
    m2 = em[1];
  }
  if (ms >= 0) {
    done = true;
    st = ST_REPLACED;
    const uint64_t cur = B[ms];
    const uint32_t b = ms < S ? b1 : b2;
    uint64_t* sp = v.buckets + static_cast<uint64_t>(b) * S + (ms & (S - 1));
    if (atomicCAS(ull(sp), cur, pack(key, val)) == cur)
      cnt.replaced += 1;
    else
      cnt.contract = true;
  } else {
    f1 = __popc(m1);
    f2 = __popc(m2);
    s1 = m1 ? __ffs(m1) - 1 : S;
    s2 = m2 ? __ffs(m2) - 1 : S;
  }
}

// The paired insert round, staged in batches of 512 / S ops when the warp has
// a live stage.
template <int S>
__device__ __forceinline__ void probe_pair_round(const View& v, unsigned need, uint32_t b1,
                                                 uint32_t b2, uint32_t key, uint32_t val,
                                                 int lane, bool& done, uint8_t& st, uint32_t& f1,
                                                 uint32_t& s1, uint32_t& f2, uint32_t& s2,
                                                 LaneCounters& cnt, Stage* sg) {
  constexpr int BO = kPairWords / (2 * S);
  constexpr unsigned BM = (BO >= 32) ? 0xFFFFFFFFu : ((1u << BO) - 1u);
  if (sg) {
    // free masks of both buckets, in flight beside the copies (unless the
    // staged words give the free slots)
    const bool mine = !HIVE_FREE_FROM_STAGE && ((need >> lane) & 1u);
    const uint32_t m1 = mine ? ld_relaxed32(v.masks + b1) : 0u;
    const uint32_t m2 = mine ? ld_relaxed32(v.masks + b2) : 0u;
#pragma unroll 1
    for (int o0 = 0; o0 < 32; o0 += BO) {
      const unsigned bneed = need & (BM << o0);
      if (!bneed) continue;
      if (sg->dead || !stage_round<S, true>(v, *sg, bneed, o0, b1, b2, lane)) {
        probe_pair<S>(v, need & ~((1u << o0) - 1u), b1, b2, key, val, lane, done, st, f1, s1, f2,
                      s2, cnt, o0, 32);
        return;
      }
      if ((bneed >> lane) & 1u)
        scan_staged_pair<S>(v, sg->buf, lane - o0, b1, b2, key, val, m1, m2, done, st, f1, s1,
                            f2, s2, cnt);
    }
  } else {
    probe_pair<S>(v, need, b1, b2, key, val, lane, done, st, f1, s1, f2, s2, cnt, 0, 32);
  }
}

// Op arrays of one batch, or of one segment of a multi-table batch.
struct OpPtrs {
  const uint8_t* ops;
  const uint32_t* keys;
  const uint32_t* vals;
  uint32_t* vals_out;
  uint8_t* found;
  uint8_t* status;
};

// Adds a warp's counters to the table of `v` and clears them: one atomic per
// non-zero counter.
__device__ __forceinline__ void flush_counters(const View& v, LaneCounters& cnt, int lane) {
  const int sd = __reduce_add_sync(kFull, static_cast<unsigned>(cnt.size_delta));
  const unsigned rp = __reduce_add_sync(kFull, cnt.replaced);
  const unsigned cl = __reduce_add_sync(kFull, cnt.claimed);
  const unsigned of = __reduce_add_sync(kFull, cnt.overflowed);
  const unsigned rs = __ballot_sync(kFull, cnt.reserved);
  const unsigned ct = __ballot_sync(kFull, cnt.contract);
  const unsigned sl = __reduce_add_sync(kFull, cnt.stash_lookups);
  if (lane == 0) {
    if (cnt.probes)
      atomicAdd(&v.ctrl->stats[kStProbes], static_cast<unsigned long long>(cnt.probes));
    if (sl) atomicAdd(&v.ctrl->stats[kStStashLookups], static_cast<unsigned long long>(sl));
    if (sd) atomicAdd(&v.ctrl->size, static_cast<unsigned long long>(static_cast<long long>(sd)));
    if (rp) atomicAdd(&v.ctrl->stats[kStReplaced], static_cast<unsigned long long>(rp));
    if (cl) atomicAdd(&v.ctrl->stats[kStClaimedFast], static_cast<unsigned long long>(cl));
    if (of) atomicAdd(&v.ctrl->stats[kStOverflowed], static_cast<unsigned long long>(of));
    if (rs) atomicOr(&v.ctrl->err, kErrReserved);
    if (ct) atomicOr(&v.ctrl->err, kErrContract);
  }
  cnt = LaneCounters();
}

// The same for every warp of a block at once, with one atomic per counter
// and block: the counters live in one control block, and an atomic per warp
// and counter at the end of a launch of thousands of warps queued in L2 for
// tens of microseconds.  Every thread of the block calls it; `scratch` is
// 8 free shared-memory words of the calling warp, and warp w's are at
// base + w * stride.
__device__ __forceinline__ void flush_counters_block(const View& v, LaneCounters& cnt, int lane,
                                                     uint64_t* scratch, const uint64_t* base,
                                                     int stride) {
  const int sd = __reduce_add_sync(kFull, static_cast<unsigned>(cnt.size_delta));
  const unsigned rp = __reduce_add_sync(kFull, cnt.replaced);
  const unsigned cl = __reduce_add_sync(kFull, cnt.claimed);
  const unsigned of = __reduce_add_sync(kFull, cnt.overflowed);
  const unsigned sl = __reduce_add_sync(kFull, cnt.stash_lookups);
  const unsigned rs = __ballot_sync(kFull, cnt.reserved);
  const unsigned ct = __ballot_sync(kFull, cnt.contract);
  __syncwarp();
  if (lane == 0) {
    scratch[0] = cnt.probes;
    scratch[1] = sl;
    scratch[2] = static_cast<uint64_t>(static_cast<int64_t>(sd));
    scratch[3] = rp;
    scratch[4] = cl;
    scratch[5] = of;
    scratch[6] = rs ? 1u : 0u;
    scratch[7] = ct ? 1u : 0u;
  }
  __syncthreads();
  const int f = threadIdx.x;
  if (f < 8) {
    uint64_t sum = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) sum += base[w * stride + f];
    if (sum) {
      switch (f) {
        case 0: atomicAdd(&v.ctrl->stats[kStProbes], static_cast<unsigned long long>(sum)); break;
        case 1: atomicAdd(&v.ctrl->stats[kStStashLookups], static_cast<unsigned long long>(sum)); break;
        case 2: atomicAdd(&v.ctrl->size, static_cast<unsigned long long>(sum)); break;
        case 3: atomicAdd(&v.ctrl->stats[kStReplaced], static_cast<unsigned long long>(sum)); break;
        case 4: atomicAdd(&v.ctrl->stats[kStClaimedFast], static_cast<unsigned long long>(sum)); break;
        case 5: atomicAdd(&v.ctrl->stats[kStOverflowed], static_cast<unsigned long long>(sum)); break;
        case 6: atomicOr(&v.ctrl->err, kErrReserved); break;
        default: atomicOr(&v.ctrl->err, kErrContract); break;
      }
    }
  }
  cnt = LaneCounters();
}

// One op's inputs (op code, key, value).
struct OpIn {
  uint32_t op, key, val;
};

template <int MODE>
__device__ __forceinline__ OpIn load_in(const OpPtrs& a, uint32_t c, uint64_t n, int lane) {
  constexpr bool kIns = (MODE == kModeInsert || MODE == kModeMixed);
  const uint32_t i = (c << 5) + lane;
  const bool valid = i < n;
  OpIn in;
  in.op = OP_FIND;
  if (MODE == kModeMixed)
    in.op = valid ? static_cast<uint32_t>(__ldcs(a.ops + i)) : OP_FIND;
  else if (MODE == kModeInsert)
    in.op = OP_INSERT;
  else if (MODE == kModeErase)
    in.op = OP_ERASE;
  if (in.op > OP_ERASE) in.op = OP_FIND;  // unknown op codes read only
  in.key = valid ? __ldcs(a.keys + i) : kEmptyKey;
  in.val = (kIns && valid && in.op == OP_INSERT && a.vals) ? __ldcs(a.vals + i) : 0u;
  return in;
}

// List appends at a high rate go through a per-warp shared-memory buffer: a
// warp gathers entries over several rounds and reserves list space for all it
// holds with one atomicAdd when the next round's entries would not fit.  One
// counter serves the whole list; an atomicAdd on that one word per warp round
// queued behind each other in L2 and held up every warp's memory pipeline.
// (The bulk kernel's own eviction hand-off is rare enough to append directly;
// a mixed batch's new keys go to fixed per-chunk places, see run_chunk.)
// A buffer of `cap` entries takes 2 * cap shared-memory words: cap packed
// words, then cap op indices and cap segment tags (u32).
struct OvfBuf {
  uint64_t* words;
  uint32_t* idx;
  uint32_t* seg;
  uint32_t n;       // entries held (warp-uniform)
  uint32_t cap;
};

__device__ __forceinline__ OvfBuf ovf_buf_init(uint64_t* region, uint32_t cap) {
  OvfBuf ob;
  ob.words = region;
  ob.idx = reinterpret_cast<uint32_t*>(region + cap);
  ob.seg = ob.idx + cap;
  ob.n = 0;
  ob.cap = cap;
  return ob;
}

// Moves every buffered entry to the list (warp-wide).
__device__ __forceinline__ void ovf_flush(const List& ovf, OvfBuf& ob, int lane) {
  if (!ob.n) return;
  __syncwarp();
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(ovf.count, ob.n);
  base = __shfl_sync(kFull, base, 0);
  for (uint32_t j = lane; j < ob.n; j += 32) {
    ovf.words[base + j] = ob.words[j];
    ovf.idx[base + j] = ob.idx[j];
    if (ovf.seg) ovf.seg[base + j] = ob.seg[j];
  }
  __syncwarp();
  ob.n = 0;
}

// Adds one round's entries (lanes with `put`) to the buffer, flushing first
// if they would not fit.
__device__ __forceinline__ void ovf_put(const List& ovf, OvfBuf& ob, int lane, bool put,
                                        uint64_t word, uint32_t idx, uint32_t seg) {
  const unsigned om = __ballot_sync(kFull, put);
  if (!om) return;
  if (ob.n + __popc(om) > ob.cap) ovf_flush(ovf, ob, lane);
  if (put) {
    const unsigned r = ob.n + __popc(om & ((1u << lane) - 1u));
    ob.words[r] = word;
    ob.idx[r] = idx;
    ob.seg[r] = seg;
  }
  ob.n += __popc(om);
}

// The final flush of every warp of a block at once: one atomicAdd reserves
// the list space of the whole block.  Every thread of the block calls it.
__device__ __forceinline__ void ovf_flush_block(const List& ovf, OvfBuf& ob, int lane) {
  __shared__ unsigned warp_n[32];
  __shared__ unsigned block_base;
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) warp_n[w] = ob.n;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int k = 0; k < nw; ++k) tot += warp_n[k];
    block_base = tot ? atomicAdd(ovf.count, tot) : 0u;
  }
  __syncthreads();
  unsigned base = block_base;
  for (int k = 0; k < w; ++k) base += warp_n[k];
  for (uint32_t j = lane; j < ob.n; j += 32) {
    ovf.words[base + j] = ob.words[j];
    ovf.idx[base + j] = ob.idx[j];
    if (ovf.seg) ovf.seg[base + j] = ob.seg[j];
  }
  __syncwarp();
  ob.n = 0;
}

// Ops [32c, 32c + 32) of a batch of n ops on the table of `v`.  Full-bucket
// inserts go to the overflow list, tagged with `seg` when the list keeps tags.
// `pre` holds the chunk's inputs when the caller loaded them ahead.
// DEFER (mixed batches): inserts of absent keys do not claim here.  Chunk c
// writes them to list places [32c, 32c + k) and k to ovf.chunk_cnt[c], with no
// atomic, and k_claim places them once every find, erase and replace of the
// batch has run.
template <int MODE, int S, bool DEFER = false>
__device__ __forceinline__ void run_chunk(const View& v, uint32_t stash_n, const OpPtrs a,
                                          uint32_t c, uint64_t n, const List ovf, uint32_t seg,
                                          LaneCounters& cnt, int lane, Stage* sg = nullptr,
                                          const OpIn* pre = nullptr) {
  constexpr bool kIns = (MODE == kModeInsert || MODE == kModeMixed);
  constexpr bool kClaim = kIns && !DEFER;
  const uint32_t i = (c << 5) + lane;
  const bool valid = i < n;
  const OpIn in = pre ? *pre : load_in<MODE>(a, c, n, lane);
  const uint32_t op = in.op, key = in.key, val = in.val;
  const bool reserved = valid && key >= kReservedKeyMin;
  const bool live = valid && !reserved;
  cnt.reserved |= reserved;

  const uint32_t b1 = lh_bucket(bithash1(key), v.M, v.p);
  const uint32_t b2 = lh_bucket(bithash2(key), v.M, v.p);
  bool done = !live;
  uint8_t st = reserved ? ST_RESERVED : ST_NOT_FOUND;
  uint32_t outv = 0;
  uint32_t f1 = 0, s1 = S, f2 = 0, s2 = S;
  PendCas pc{0, 0, 0, 0, 0};

  // Probe the BitHash1 bucket of every op, then the BitHash2 bucket of the
  // ops still unresolved (Section IV-B: WCME over the d = 2 candidates).
  unsigned need = __ballot_sync(kFull, !done);
  if (MODE == kModeInsert) {
    cnt.probes += 2 * __popc(need);
    if (need) probe_pair_round<S>(v, need, b1, b2, key, val, lane, done, st, f1, s1, f2, s2, cnt, sg);
  } else {
    cnt.probes += __popc(need);
    if (need)
      probe_round<MODE, S, kClaim>(v, need, b1, key, val, op, lane, done, st, outv, f1, s1, cnt,
                                   sg, pc);
    need = __ballot_sync(kFull, !done);
    cnt.probes += __popc(need);
    if (need)
      probe_round<MODE, S, kClaim>(v, need, b2, key, val, op, lane, done, st, outv, f2, s2, cnt,
                                   sg, pc);
  }

  // The stash (Section IV-A step 4) holds keys that found no bucket room.
  if (!done && stash_n) {
    uint32_t pos;
    cnt.stash_lookups += 1;
    if (stash_find(v, stash_n, key, pos)) {
      uint64_t* sp = v.stash_kv + pos;
      const uint64_t w = ld_relaxed64(sp);
      if (key_of(w) == key) {
        done = true;
        if (op == OP_FIND) {
          outv = val_of(w);
          st = ST_FOUND;
        } else if (op == OP_ERASE) {
          st = ST_ERASED;
          if (atomicCAS(ull(sp), w, kEmptyWord) == w) {
            cnt.size_delta -= 1;
            atomicExch(&v.ctrl->stash_dirty, 1u);
          } else {
            cnt.contract = true;
          }
        } else {
          st = ST_REPLACED;
          if (atomicCAS(ull(sp), w, pack(key, val)) == w) cnt.replaced += 1; else cnt.contract = true;
        }
      }
    }
  }

  // Step 2: claim-then-commit for absent keys.
  bool to_ovf = false;
  if (DEFER && kIns && !done && op == OP_INSERT) {
    to_ovf = true;  // k_claim places it
  } else if (kIns && !done && op == OP_INSERT) {
    const uint64_t word = pack(key, val);
    const bool first1 = v.placement ? (f1 > 0) : (f1 >= f2);
    const uint32_t tb = first1 ? b1 : b2, ts = first1 ? s1 : s2;
    const uint32_t ob = first1 ? b2 : b1, os = first1 ? s2 : s1;
    bool placed = false;
    if (f1 + f2 > 0) {
      placed = claim_store<S>(v, tb, ts, word);
      if (!placed && ob != tb) placed = claim_store<S>(v, ob, os, word);
    }
    if (placed) {
      done = true;
      st = ST_INSERTED;
      cnt.size_delta += 1;
      cnt.claimed += 1;
    } else {
      to_ovf = true;
      cnt.overflowed += 1;
    }
  }

  resolve_cas(v, pc, cnt);

  // Hand full-bucket inserts to the eviction kernel (steps 3-4).
  if (kIns) {
    const unsigned om = __ballot_sync(kFull, to_ovf);
    if (DEFER) {
      if (to_ovf) {
        const unsigned r = (c << 5) + __popc(om & ((1u << lane) - 1u));
        ovf.words[r] = pack(key, val);
        ovf.idx[r] = i;
      }
      if (lane == 0) ovf.chunk_cnt[c] = static_cast<uint8_t>(__popc(om));
    } else if (om) {
      const int leader = __ffs(om) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(ovf.count, static_cast<unsigned>(__popc(om)));
      base = __shfl_sync(kFull, base, leader);
      if (to_ovf) {
        const unsigned r = base + __popc(om & ((1u << lane) - 1u));
        ovf.words[r] = pack(key, val);
        ovf.idx[r] = i;
        if (ovf.seg) ovf.seg[r] = seg;
      }
    }
  }

  if (valid) {
    if (MODE == kModeFind) {
      __stcs(a.vals_out + i, outv);
      if (a.found) a.found[i] = st == ST_FOUND ? 1 : 0;
    } else {
      if (a.status && !to_ovf) a.status[i] = st;
      if (MODE == kModeMixed && a.vals_out) __stcs(a.vals_out + i, outv);
    }
  }
}

// Resident blocks of THREADS threads per SM a bulk kernel is built for: the
// warps per SM of the 256-thread shape (at least one block), which sets the
// register budget of each shape.
__host__ __device__ constexpr int ops_min_blocks(int mode, int S, int threads) {
  return ((staged_mode(mode, S) ? staged_min_blocks(mode, S) : HIVE_OPS_MIN_BLOCKS) * kOpsThreads /
              threads >
          0)
             ? (staged_mode(mode, S) ? staged_min_blocks(mode, S) : HIVE_OPS_MIN_BLOCKS) *
                   kOpsThreads / threads
             : 1;
}

// DEFER (mixed batches): the new keys are claimed by k_claim afterwards.
// THREADS: the block shape (128, 256 or 512 threads; a tuning knob).
template <int MODE, int S, bool DEFER, int THREADS>
__global__ void __launch_bounds__(THREADS, ops_min_blocks(MODE, S, THREADS))
    k_ops(View v, OpPtrs a, uint64_t n, List ovf, int prefetch_masks) {
  // claims and erases update free masks at random; a large batch first asks
  // L2 for the whole mask array in sequential pieces
  if (prefetch_masks) prefetch_l2_grid(v.masks, static_cast<uint64_t>(v.nb) * sizeof(uint32_t));
  const int lane = threadIdx.x & 31;
  // n < 2^32 per call, so chunk and op indices fit 32 bits
  const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t nchunks = static_cast<uint32_t>((n + 31) >> 5);
  const uint32_t stash_n = v.ctrl->stash_n;
  LaneCounters cnt;
  if (staged_mode(MODE, S)) {
    // bucket reads staged in shared memory
    extern __shared__ __align__(16) uint64_t ops_smem[];
    Stage sg = stage_init(ops_smem, threadIdx.x >> 5, lane, warp_smem_words(MODE, S));
    // inputs are loaded one chunk ahead, so their latency hides behind the
    // current chunk's probes and claims
    OpIn nxt{};
    if (warp0 < nchunks) nxt = load_in<MODE>(a, warp0, n, lane);
    for (uint32_t c = warp0; c < nchunks; c += nwarps) {
      const OpIn cur = nxt;
      if (c + nwarps < nchunks) nxt = load_in<MODE>(a, c + nwarps, n, lane);
      run_chunk<MODE, S, DEFER>(v, stash_n, a, c, n, ovf, 0, cnt, lane, &sg, &cur);
    }
    stage_drain(sg);
    // the staging buffers are free now (a dead stage's late copies have landed
    // or stage_drain gave up on them, and then its first words stay unused)
    if (!__syncthreads_or(sg.dead ? 1 : 0))
      flush_counters_block(v, cnt, lane, sg.buf, ops_smem + 2, warp_smem_words(MODE, S));
    else
      flush_counters(v, cnt, lane);
  } else {
    for (uint32_t c = warp0; c < nchunks; c += nwarps)
      run_chunk<MODE, S, DEFER>(v, stash_n, a, c, n, ovf, 0, cnt, lane);
    flush_counters(v, cnt, lane);
  }
}

// Step 2 for the new keys of a mixed batch (WABC, Section III-E), after the
// bulk kernel has run every find, erase and replace of the batch: the slots
// those erases freed are then visible to the claims.  The bulk kernel left
// chunk c's new keys at list places [32c, 32c + chunk_cnt[c]).  A warp takes 32
// chunks at a time, scans their counts and spreads their entries over its
// lanes, one item per lane: hash, read both free masks, claim the predicted
// slot of the emptier bucket with one atomicAnd (the other bucket next),
// store the word.  Nothing moves or erases a word meanwhile, so the claim
// publishes with a plain store.  Items whose two buckets are both full go to
// `out` for eviction (steps 3-4).
constexpr int kClaimThreads = 256;
constexpr int kClaimBuf = 256;  // entries of each warp's buffer of full-bucket items
#ifndef HIVE_CLAIM_PREFETCH_SLOT
#define HIVE_CLAIM_PREFETCH_SLOT 0
#endif
#ifndef HIVE_CLAIM_ILP
#define HIVE_CLAIM_ILP 4
#endif
constexpr int kClaimIlp = HIVE_CLAIM_ILP;  // items per lane in flight at once
template <int S>
__global__ void __launch_bounds__(kClaimThreads)
    k_claim(View v, List in, uint32_t nchunks, List out, uint8_t* __restrict__ status,
            int prefetch_masks) {
  // The claims read the free masks at random: a batch with as many new keys
  // as a fraction of the buckets is served faster from L2 after one
  // sequential fetch of the whole mask array than by a DRAM sector per read.
  if (prefetch_masks) prefetch_l2_grid(v.masks, static_cast<uint64_t>(v.nb) * sizeof(uint32_t));
  __shared__ __align__(16) uint64_t claim_smem[(kClaimThreads / 32) * 2 * kClaimBuf];
  const int lane = threadIdx.x & 31;
  OvfBuf ob = ovf_buf_init(claim_smem + (threadIdx.x >> 5) * 2 * kClaimBuf, kClaimBuf);
  LaneCounters cnt;
  const uint32_t ngroups = (nchunks + 31) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // chunk counts are loaded one group ahead
  uint32_t k_next = (g < ngroups && (g << 5) + lane < nchunks) ? in.chunk_cnt[(g << 5) + lane] : 0u;
  for (; g < ngroups; g += nwarps) {
    const uint32_t k = k_next;
    const uint32_t gn = g + nwarps;
    k_next = (gn < ngroups && (gn << 5) + lane < nchunks) ? in.chunk_cnt[(gn << 5) + lane] : 0u;
    uint32_t incl = k;  // inclusive prefix sum of the 32 counts
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += t;
    }
    const uint32_t excl = incl - k;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32 * kClaimIlp) {
      uint64_t word[kClaimIlp];
      uint32_t idx[kClaimIlp], b1[kClaimIlp], b2[kClaimIlp], m1[kClaimIlp], m2[kClaimIlp];
#pragma unroll
      for (int u = 0; u < kClaimIlp; ++u) {
        const uint32_t t = t0 + 32 * u + lane;
        // chunk j of entry t: the first j whose inclusive sum passes t
        uint32_t j = 0;
#pragma unroll
        for (uint32_t step = 16; step; step >>= 1) {
          const uint32_t e = __shfl_sync(kFull, incl, j + step - 1);
          if (e <= t) j += step;
        }
        const uint32_t ex = __shfl_sync(kFull, excl, j & 31);
        const uint32_t pos = (((g << 5) + j) << 5) + (t - ex);
        word[u] = t < total ? in.words[pos] : kEmptyWord;
        idx[u] = t < total ? in.idx[pos] : kNoOp;
      }
#pragma unroll
      for (int u = 0; u < kClaimIlp; ++u) {
        const uint32_t key = key_of(word[u]);
        b1[u] = lh_bucket(bithash1(key), v.M, v.p);
        b2[u] = lh_bucket(bithash2(key), v.M, v.p);
        const bool valid = t0 + 32 * u + lane < total;
        m1[u] = valid ? ld_relaxed32(v.masks + b1[u]) : 0u;
        m2[u] = valid ? ld_relaxed32(v.masks + b2[u]) : 0u;
      }
      // first claim attempt of every item, then the outcomes (a failed
      // attempt retries on the returned mask, then on the other bucket)
      uint32_t old[kClaimIlp], bit[kClaimIlp];
#pragma unroll
      for (int u = 0; u < kClaimIlp; ++u) {
        const uint32_t f1 = __popc(m1[u]), f2 = __popc(m2[u]);
        const bool first1 = v.placement ? (f1 > 0) : (f1 >= f2);
        if (!first1) {
          const uint32_t tb = b1[u], tm = m1[u];
          b1[u] = b2[u];
          m1[u] = m2[u];
          b2[u] = tb;
          m2[u] = tm;
        }
        bit[u] = m1[u] ? (1u << (__ffs(m1[u]) - 1)) : 0u;
#if HIVE_CLAIM_PREFETCH_SLOT
        if (bit[u])
          asm volatile("prefetch.global.L2 [%0];" ::"l"(v.buckets + static_cast<uint64_t>(b1[u]) * S +
                                                          (__ffs(bit[u]) - 1)));
#endif
        old[u] = bit[u] ? atomicAnd(v.masks + b1[u], ~bit[u]) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kClaimIlp; ++u) {
        const bool valid = t0 + 32 * u + lane < total;
        bool placed = false, to_ovf = false;
        if (valid) {
          if (old[u] & bit[u]) {
            st_relaxed64(v.buckets + static_cast<uint64_t>(b1[u]) * S + (__ffs(bit[u]) - 1),
                         word[u]);
            placed = true;
          } else {
            if (bit[u]) placed = claim_store<S>(v, b1[u], old[u] ? __ffs(old[u]) - 1 : S, word[u]);
            if (!placed && b2[u] != b1[u] && m2[u])
              placed = claim_store<S>(v, b2[u], __ffs(m2[u]) - 1, word[u]);
          }
          if (placed) {
            cnt.size_delta += 1;
            cnt.claimed += 1;
            if (status && idx[u] != kNoOp) status[idx[u]] = ST_INSERTED;
          } else {
            to_ovf = true;
            cnt.overflowed += 1;
          }
        }
        ovf_put(out, ob, lane, to_ovf, word[u], idx[u], 0);
      }
    }
  }
  ovf_flush_block(out, ob, lane);
  flush_counters_block(v, cnt, lane, ob.words, claim_smem, 2 * kClaimBuf);
}

// ----------------------------------------------------------------------------
// Steps 3-4: bounded cuckoo eviction and the overflow stash (Algorithm 3)
// ----------------------------------------------------------------------------

// A chain may end in the stash, so it first reserves a stash word; chains that
// finish in a bucket give the reservation back, so appends never pass
// stash_cap.  When every free word is reserved by running chains, wait for
// them (they end within max_evictions rounds); give up only once the stash is
// really full or after a bounded wait.
__device__ __forceinline__ bool stash_reserve(const View& v) {
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

// Counters of the eviction kernel, kept by lane 0 of a warp, and the stash
// word the warp holds in reserve.  A warp works one item at a time, so one
// reservation covers all its chains: it is kept across items that end in a
// bucket and renewed only after a chain used it for a stash append.
struct OvfCounters {
  unsigned claim = 0, rounds = 0, locks = 0, to = 0, stash = 0, pend = 0, added = 0;
  Ctrl* reserved_in = nullptr;  // control block of the table the reservation belongs to
};

// `lead`: the calling lane leads its group and holds the group's counters.
__device__ __forceinline__ void flush_ovf_counters(const View& v, OvfCounters& oc, bool lead) {
  if (lead) {
    Ctrl* c = v.ctrl;
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
  Ctrl* keep = oc.reserved_in;  // a reservation outlives the counters
  oc = OvfCounters();
  oc.reserved_in = keep;
}

// Gives back a warp's unused stash reservation.
__device__ __forceinline__ void release_reservation(OvfCounters& oc, bool lead) {
  if (lead && oc.reserved_in) atomicSub(&oc.reserved_in->stash_claims, 1u);
  oc.reserved_in = nullptr;
}

// A block's pool of stash reservations: one table-wide atomic fills it for
// the groups that will carry an item, and the groups take from it in shared
// memory.  With thousands of groups per launch, one reservation atomic each
// on the single counter serialised in L2 and cost about a fifth of the
// eviction kernel's time.  A taker succeeds only on a positive count; a
// failed take puts its decrement back.
__device__ __forceinline__ bool pool_take(int* pool) {
  if (!pool) return false;
  if (atomicSub(pool, 1) > 0) return true;
  atomicAdd(pool, 1);
  return false;
}

// Fills the pool with up to `want` reservations (thread 0 of the block).
__device__ __forceinline__ int pool_fill(const View& v, unsigned want) {
  if (!want) return 0;
  const unsigned base = atomicAdd(&v.ctrl->stash_claims, want);
  const unsigned got = base >= v.stash_cap ? 0u : min(want, v.stash_cap - base);
  if (got < want) atomicSub(&v.ctrl->stash_claims, want - got);
  return static_cast<int>(got);
}

// Steps 3-4 for one insert whose candidate buckets were full (warp-wide).
// `idx` is the caller's op index (kNoOp for a word moved by a merge); the
// outcome goes to status[idx].  With `resizable`, an insert that finds no room
// at all joins the pending list, else it is reported FULL.
// `pool` (optional): stash words the calling block reserved for its groups
// in one atomic (a shared-memory count), taken before the table-wide
// counter is asked.
template <int S>
__device__ __forceinline__ void overflow_item(const View& v, uint64_t word0, uint32_t idx,
                                              uint32_t seg, uint8_t* status, int resizable,
                                              const List& pend, OvfCounters& oc, int lane,
                                              int* pool = nullptr) {
  // The item belongs to a group of S lanes (a half-warp at S = 16, so a warp
  // carries two chains at once): group lane gl holds slot gl of the bucket in
  // hand, and group lane 0 leads.
  constexpr unsigned kGroupBits = (S >= 32) ? 0xFFFFFFFFu : ((1u << S) - 1u);
  const int gl = lane & (S - 1);
  const int gb = lane - gl;
  const unsigned gmask = kGroupBits << gb;
  auto group_ballot = [&](bool pred) { return (__ballot_sync(gmask, pred) >> gb) & kGroupBits; };
  const uint32_t key0 = key_of(word0);
  const uint32_t b1 = lh_bucket(bithash1(key0), v.M, v.p);
  const uint32_t b2 = lh_bucket(bithash2(key0), v.M, v.p);

  // 0: needs eviction, 1: placed, 2: stashed, 3: no room (pending)
  int outcome = 0;
  // the BitHash1 bucket, read now for the first eviction round: most items
  // here find both buckets still full
  const uint64_t w0 = ld_relaxed64(v.buckets + static_cast<uint64_t>(b1) * S + gl);
  if (gl == 0) {
    // both free masks in one round trip; claim where a bit is free
    const uint32_t m1 = ld_relaxed32(v.masks + b1);
    const uint32_t m2 = ld_relaxed32(v.masks + b2);
    if ((m1 && claim_pub<S>(v, b1, word0, m1)) || (b2 != b1 && m2 && claim_pub<S>(v, b2, word0, m2))) {
      outcome = 1;
      ++oc.claim;
    } else {
      if (oc.reserved_in != v.ctrl) {
        if (oc.reserved_in) atomicSub(&oc.reserved_in->stash_claims, 1u);
        oc.reserved_in = (pool_take(pool) || stash_reserve(v)) ? v.ctrl : nullptr;
      }
      if (!oc.reserved_in) outcome = 3;
    }
  }
  outcome = __shfl_sync(gmask, outcome, 0, S);

  if (outcome == 0) {
    uint64_t cur = word0;
    uint32_t b = b1;
    bool placed = false;
    for (uint32_t r = 0; r < v.max_evictions; ++r) {
      // Look ahead: each lane checks whether the word in its slot could move
      // to its other candidate bucket without a further eviction.
      const uint64_t w = r == 0 ? w0 : ld_relaxed64(v.buckets + static_cast<uint64_t>(b) * S + gl);
      uint32_t am = 0;  // free mask of this word's other candidate bucket
      if (w != kEmptyWord) {
        const uint32_t k = key_of(w);
        const uint32_t a1 = lh_bucket(bithash1(k), v.M, v.p);
        const uint32_t a2 = lh_bucket(bithash2(k), v.M, v.p);
        const uint32_t alt = (a1 == b) ? a2 : a1;
        if (alt != b) am = ld_relaxed32(v.masks + alt);
      }
      const unsigned gm = group_ballot(am != 0u);
      const unsigned occ = group_ballot(w != kEmptyWord);
      const bool has_empty = occ != kGroupBits;
      int res = 0;  // 0: evicted `victim`, 1: placed, 2: lock wait gave up, 3: redo the round
      uint64_t victim = kEmptyWord;
      // victim: an occupied slot whose word can move on at once, else an
      // occupied slot picked by rotation (never an EMPTY one, see claim_pub)
      uint32_t vs = S;
      if (gm) {
        vs = __ffs(gm) - 1;
      } else if (occ) {
        const uint32_t start = (bithash2(key_of(cur)) + r) & (S - 1);
        const unsigned rot =
            start ? (((occ >> start) | (occ << (S - start))) & kGroupBits) : occ;
        vs = (start + __ffs(rot) - 1) & (S - 1);
      }
      const uint32_t vmask = __shfl_sync(gmask, am, vs & (S - 1), S);
      if (gl == 0) {
        ++oc.rounds;
        if (!lock_bucket(v, b)) {
          res = 2;
          ++oc.to;
        } else {
          ++oc.locks;
          if (has_empty && claim_pub<S>(v, b, cur)) {
            res = 1;
          } else if (vs >= S) {
            res = 3;  // every slot claimed but not yet published: look again
          } else {
            victim = atomicExch(ull(v.buckets + static_cast<uint64_t>(b) * S + vs), cur);
            res = (victim == kEmptyWord) ? 1 : 0;
          }
          unlock_bucket(v, b);
        }
      }
      res = __shfl_sync(gmask, res, 0, S);
      victim = __shfl_sync(gmask, victim, 0, S);
      if (res == 1) {
        placed = true;
        break;
      }
      if (res == 2) break;
      if (res == 3) continue;
      // Re-route the displaced word to its alternate bucket.
      cur = victim;
      const uint32_t kc = key_of(cur);
      const uint32_t a1 = lh_bucket(bithash1(kc), v.M, v.p);
      const uint32_t a2 = lh_bucket(bithash2(kc), v.M, v.p);
      const uint32_t nb = (a1 == b) ? a2 : a1;
      if (nb == b) break;  // both candidates are this bucket: no alternative
      b = nb;
      int ok = 0;
      if (gl == 0) ok = claim_pub<S>(v, b, cur, vmask);
      if (__shfl_sync(gmask, ok, 0, S)) {
        placed = true;
        break;
      }
    }
    if (gl == 0) {
      if (placed && oc.reserved_in && ld_relaxed32(&v.ctrl->stash_claims) >= v.stash_cap) {
        // every free stash word is reserved: give this one back so that a
        // waiting group can go on
        atomicSub(&v.ctrl->stash_claims, 1u);
        oc.reserved_in = nullptr;
      }
      if (!placed) {
        oc.reserved_in = nullptr;  // this append uses the reservation
        const unsigned pos = atomicAdd(&v.ctrl->stash_tail, 1u);
        st_relaxed64(v.stash_kv + pos, cur);
        ++oc.stash;
      }
    }
    outcome = placed ? 1 : 2;
  }

  if (gl == 0) {
    if (outcome == 3) {
      ++oc.pend;
      if (resizable) {
        const unsigned pos = atomicAdd(pend.count, 1u);
        pend.words[pos] = word0;
        pend.idx[pos] = idx;
        if (pend.seg) pend.seg[pos] = seg;
      } else {
        atomicOr(&v.ctrl->err, kErrFull);
        if (status && idx != kNoOp) status[idx] = ST_FULL;
      }
    } else if (idx != kNoOp) {
      ++oc.added;
      if (status) status[idx] = ST_INSERTED;
    }
  }
}

#ifndef HIVE_OVF_MIN_BLOCKS
#define HIVE_OVF_MIN_BLOCKS 1  // resident blocks per SM the eviction kernel's registers allow
#endif
template <int S>
__global__ void __launch_bounds__(kOvfThreads, HIVE_OVF_MIN_BLOCKS)
    k_overflow(View v, List in, List pend, int resizable, uint8_t* __restrict__ status) {
  // one item per group of S lanes at a time
  const int lane = threadIdx.x & 31;
  const unsigned group0 = (blockIdx.x * blockDim.x + threadIdx.x) / S;
  const unsigned ngroups = (gridDim.x * blockDim.x) / S;
  const bool lead = (lane & (S - 1)) == 0;
  const unsigned total = *in.count;
  // one stash reservation for each group of the block that gets an item, and
  // the groups' counters summed in shared memory: a few table-wide atomics
  // per block instead of several per group
  __shared__ int pool;
  __shared__ unsigned sum[7];
  const unsigned gpb = blockDim.x / S;
  if (threadIdx.x == 0) {
    const unsigned first = blockIdx.x * gpb;
    pool = pool_fill(v, total > first ? min(total - first, gpb) : 0u);
  }
  if (threadIdx.x < 7) sum[threadIdx.x] = 0;
  __syncthreads();
  OvfCounters oc;
  for (unsigned it = group0; it < total; it += ngroups)
    overflow_item<S>(v, in.words[it], in.idx[it], 0, status, resizable, pend, oc, lane, &pool);
  if (lead) {
    if (oc.reserved_in) atomicAdd(&pool, 1);  // back to the block's pool
    oc.reserved_in = nullptr;
    const unsigned c[7] = {oc.claim, oc.rounds, oc.locks, oc.to, oc.stash, oc.pend, oc.added};
#pragma unroll
    for (int k = 0; k < 7; ++k)
      if (c[k]) atomicAdd(&sum[k], c[k]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (pool > 0) atomicSub(&v.ctrl->stash_claims, static_cast<unsigned>(pool));
    OvfCounters b;
    b.claim = sum[0];
    b.rounds = sum[1];
    b.locks = sum[2];
    b.to = sum[3];
    b.stash = sum[4];
    b.pend = sum[5];
    b.added = sum[6];
    flush_ovf_counters(v, b, true);
  }
}

// ----------------------------------------------------------------------------
// Concurrent mixed batch in one kernel (the paper's single-kernel mode)
// ----------------------------------------------------------------------------
//
// Here finds, erases, replaces, claims and eviction chains of one batch run
// at the same time, so a lookup can race with a chain that has taken a word
// out of a bucket and not yet put it down.  Each bucket has a version word:
// bits 0..15 count the chains holding, in transit, a word whose BitHash1
// bucket this is, bits 16..31 count chain steps that finished (modulo 2^16:
// the count lives as long as the table, and its carry leaves the word
// instead of reaching the transit count).  A chain raises the transit count
// of the BitHash1 bucket of the word it is about to swap out (whichever of
// its two buckets that word sits in) and lowers it (bumping the step count)
// once that word sits in its other bucket or in the stash, with a fence on
// each side.  A lookup of key k reads the version of
// k's BitHash1 bucket before probing and again after a miss: one word covers
// every move of k.  The miss stands only if no word was in transit there and
// the version did not move; otherwise the op probes again.  A hit needs no
// check: the word was observed in place.  Because erases now run beside
// chains, a chain swaps its victim with a CAS on the word it read (never
// onto an EMPTY slot); claims then own their slot by its free bit alone.
constexpr uint32_t kTransitMask = 0xFFFFu;  // words in transit
constexpr uint32_t kStep = 1u << 16;         // one finished step
constexpr uint32_t kFusedRetryLimit = 1u << 14;

__device__ __forceinline__ void transit_begin(const View& v, uint32_t b) {
  atomicAdd(v.vers + b, 1u);
  fence_acq_rel_gpu();
}
__device__ __forceinline__ void transit_end(const View& v, uint32_t b) {
  fence_acq_rel_gpu();
  atomicAdd(v.vers + b, kStep - 1u);  // one word fewer in transit, one step more
}

// Steps 3-4 for one new key whose candidate buckets had no free slot, inside
// the single-kernel batch.  One chain per lane: the lanes of a warp carry up
// to 32 chains at once, each on its own (they may diverge; a chain holds at
// most one bucket lock at a time and waits for it a bounded number of
// tries).  A chain is a run of dependent round trips, so carrying many at
// once is what keeps the step short; a warp-wide chain left 31 lanes idle
// per round trip.  The caller has already tried both free masks and holds a
// stash reservation in `oc`.  Each round reads the bucket in hand 8 words at
// a time with the free masks of those words' other buckets, and stops at the
// first word that could move on at once (the victim); if none could, the
// victim is the first occupied slot from a rotating start.  Under the bucket
// lock the chain claims a free slot of the bucket for its word, or swaps the
// victim out with a CAS on the exact word it re-read (never onto an EMPTY
// slot), marking the version of the victim's BitHash1 bucket as holding a
// word in transit until that word is down again.  Returns 1 placed, 2
// stashed.
template <int S>
__device__ int chain_lane(const View& v, uint64_t word0, uint32_t b1, OvfCounters& oc) {
  uint64_t cur = word0;
  uint32_t b = b1;
  uint32_t held = kNoOp;  // version bucket marked for the word in hand
  bool placed = false;
  for (uint32_t r = 0; r < v.max_evictions; ++r) {
    uint64_t* B = v.buckets + static_cast<uint64_t>(b) * S;
    unsigned occ = 0;
    int vs = -1;
    uint32_t vmask = 0;
#pragma unroll 1
    for (int f0 = 0; f0 < S; f0 += 8) {
      uint64_t w[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) ld_frag(B + f0 + 2 * q, w[2 * q], w[2 * q + 1]);
      uint32_t am[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        am[k] = 0;
        if (w[k] != kEmptyWord) {
          occ |= 1u << (f0 + k);
          const uint32_t kk = key_of(w[k]);
          const uint32_t a1 = lh_bucket(bithash1(kk), v.M, v.p);
          const uint32_t a2 = lh_bucket(bithash2(kk), v.M, v.p);
          const uint32_t alt = (a1 == b) ? a2 : a1;
          if (alt != b) am[k] = ld_relaxed32(v.masks + alt);
        }
      }
#pragma unroll
      for (int k = 7; k >= 0; --k)
        if (am[k]) {
          vs = f0 + k;
          vmask = am[k];
        }
      if (vs >= 0) break;
    }
    if (vs < 0 && occ) {
      const uint32_t start = (bithash2(key_of(cur)) + r) & (S - 1);
      const unsigned rot = (occ >> start) | (start ? (occ << (32 - start)) : 0u);
      vs = static_cast<int>((start + __ffs(rot) - 1) & (S - 1));
    }
    int res;  // 0: swapped, 1: placed, 2: lock wait gave up, 3: redo the round
    uint64_t wv = kEmptyWord;
    uint32_t vb = 0;  // BitHash1 bucket of the victim: its version carries the transit mark
    ++oc.rounds;
    if (!lock_bucket(v, b)) {
      res = 2;
      ++oc.to;
    } else {
      ++oc.locks;
      const uint32_t mb = ld_relaxed32(v.masks + b);
      if (mb && claim_pub<S>(v, b, cur, mb)) {
        res = 1;
      } else if (vs < 0) {
        res = 3;
      } else {
        uint64_t* sp = B + vs;
        wv = ld_relaxed64(sp);
        if (wv == kEmptyWord) {
          res = 3;  // claimed and not yet published, or erased: look again
        } else {
          vb = lh_bucket(bithash1(key_of(wv)), v.M, v.p);
          transit_begin(v, vb);
          if (atomicCAS(ull(sp), wv, cur) == wv) {
            res = 0;
          } else {
            transit_end(v, vb);
            res = 3;
          }
        }
      }
      unlock_bucket(v, b);
    }
    // the word in hand now sits in b (placed or swapped in)
    if ((res == 0 || res == 1) && held != kNoOp) transit_end(v, held);
    if (res == 1) {
      placed = true;
      held = kNoOp;
      break;
    }
    if (res == 2) break;
    if (res == 3) continue;
    held = vb;
    cur = wv;
    const uint32_t kc = key_of(cur);
    const uint32_t a1 = lh_bucket(bithash1(kc), v.M, v.p);
    const uint32_t a2 = lh_bucket(bithash2(kc), v.M, v.p);
    const uint32_t nb = (a1 == b) ? a2 : a1;
    if (nb == b) break;
    b = nb;
    if (claim_pub<S>(v, b, cur, vmask)) {
      transit_end(v, held);
      held = kNoOp;
      placed = true;
      break;
    }
  }
  if (placed && oc.reserved_in && ld_relaxed32(&v.ctrl->stash_claims) >= v.stash_cap) {
    // every free stash word is reserved: give this one back
    atomicSub(&v.ctrl->stash_claims, 1u);
    oc.reserved_in = nullptr;
  }
  if (!placed) {
    oc.reserved_in = nullptr;  // this append uses the reservation
    const unsigned pos = atomicAdd(&v.ctrl->stash_tail, 1u);
    st_relaxed64(v.stash_kv + pos, cur);
    ++oc.stash;
    if (held != kNoOp) transit_end(v, held);
  }
  return placed ? 1 : 2;
}

// A warp's queue of new keys whose two buckets were full, in shared memory:
// kFusedQ packed words, then kFusedQ op indices.  The warp runs their chains
// 32 at a time (one per lane) once 32 are waiting, and the rest before it
// exits.  `n` is warp-uniform.
constexpr uint32_t kFusedQ = 64;
struct EvictQ {
  uint64_t* words;
  uint32_t* idx;
  uint32_t n;
};

// Runs the chains of the first min(n, 32) queued keys, one per lane, and
// moves the rest to the front (warp-wide).  Each key first tries both free
// masks again (slots may have been freed since); the keys still without room
// take a stash reservation for the warp's chains with one atomic, then run
// their chains.
template <int S>
__device__ void fused_drain(const View& v, EvictQ& q, uint8_t* status, const List& pend,
                            int resizable, OvfCounters& oc, int lane) {
  __syncwarp();
  const uint32_t m = q.n < 32 ? q.n : 32u;
  const bool has = static_cast<uint32_t>(lane) < m;
  const uint64_t word = has ? q.words[lane] : kEmptyWord;
  const uint32_t idx = has ? q.idx[lane] : kNoOp;
  const uint32_t key = key_of(word);
  const uint32_t b1 = lh_bucket(bithash1(key), v.M, v.p);
  const uint32_t b2 = lh_bucket(bithash2(key), v.M, v.p);
  int out = 0;  // 1 placed, 2 stashed, 3 no room
  if (has) {
    const uint32_t m1 = ld_relaxed32(v.masks + b1);
    const uint32_t m2 = ld_relaxed32(v.masks + b2);
    if ((m1 && claim_pub<S>(v, b1, word, m1)) ||
        (b2 != b1 && m2 && claim_pub<S>(v, b2, word, m2))) {
      out = 1;
      ++oc.claim;
    }
  }
  // a chain may end in the stash, so it holds a reservation (kept by the lane
  // for its later chains unless a stash append uses it)
  const bool need_res = has && out == 0 && oc.reserved_in != v.ctrl;
  const unsigned rm = __ballot_sync(kFull, need_res);
  if (rm) {
    const int leader = __ffs(rm) - 1;
    const unsigned k = __popc(rm);
    unsigned c0 = 0;
    if (lane == leader) c0 = atomicAdd(&v.ctrl->stash_claims, k);
    c0 = __shfl_sync(kFull, c0, leader);
    const unsigned ok_n = c0 >= v.stash_cap ? 0u : min(k, v.stash_cap - c0);
    if (lane == leader && ok_n < k) atomicSub(&v.ctrl->stash_claims, k - ok_n);
    if (need_res) {
      const unsigned rank = __popc(rm & ((1u << lane) - 1u));
      oc.reserved_in = (rank < ok_n || stash_reserve(v)) ? v.ctrl : nullptr;
    }
  }
  if (has && out == 0) out = oc.reserved_in == v.ctrl ? chain_lane<S>(v, word, b1, oc) : 3;
  __syncwarp();
  if (has) {
    if (out == 3) {
      ++oc.pend;
      if (resizable) {
        // placed by the eviction kernel after the table grows; it writes the status
        const unsigned p = atomicAdd(pend.count, 1u);
        pend.words[p] = word;
        pend.idx[p] = idx;
      } else {
        atomicOr(&v.ctrl->err, kErrFull);
        if (status && idx != kNoOp) status[idx] = ST_FULL;
      }
    } else {
      ++oc.added;
      if (status && idx != kNoOp) status[idx] = ST_INSERTED;
    }
  }
  // the keys after the first 32 move to the front
  const uint32_t rest = q.n - m;
  __syncwarp();
  uint64_t mw = 0;
  uint32_t mi = 0;
  if (static_cast<uint32_t>(lane) < rest) {
    mw = q.words[32 + lane];
    mi = q.idx[32 + lane];
  }
  __syncwarp();
  if (static_cast<uint32_t>(lane) < rest) {
    q.words[lane] = mw;
    q.idx[lane] = mi;
  }
  __syncwarp();
  q.n = rest;
}

// One single-bucket probe round of the single-kernel batch: bucket `myb` of
// every op in `need` copied into the warp's staging buffer (buffer bucket j
// for op j) with 16-byte cp.async through L2 only, then waited for.  Each
// copy starts after the version read (an acquire) that precedes it in
// program order, and the wait ends before the fence ahead of the second
// version read.
template <int S>
__device__ __forceinline__ void fused_stage(const View& v, uint64_t* sbuf, unsigned need,
                                            uint32_t myb, int lane) {
  constexpr int L = Geo<S>::L, Q = Geo<S>::Q;
  const int q = lane / L, ql = lane % L;
  __syncwarp();  // earlier reads of the buffer by any lane come first
#pragma unroll 4
  for (int r = 0; r < 32 / Q; ++r) {
    const int bi = Q * r + q;
    const uint32_t y = __shfl_sync(kFull, myb, bi);
    if ((need >> bi) & 1u)
      cp_async16_cg(sbuf + bi * S + 2 * ql, v.buckets + static_cast<uint64_t>(y) * S + 2 * ql);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncwarp();
}

// Looks the op keys of the `need` lanes up in the stash words appended during
// this kernel, [from, to) (warp-wide).  A lane that finds its key gets its
// position in `pos` and returns true.
__device__ __forceinline__ bool stash_tail_find(const View& v, uint32_t from, uint32_t to,
                                                unsigned need, uint32_t key, int lane,
                                                uint32_t& pos) {
  bool hit = false;
  for (uint32_t base = from; base < to; base += 32) {
    const uint32_t j = base + lane;
    const uint64_t w = j < to ? ld_relaxed64(v.stash_kv + j) : kEmptyWord;
    for (unsigned m = need; m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      const uint32_t kj = __shfl_sync(kFull, key, src);
      const unsigned eq = __ballot_sync(kFull, w != kEmptyWord && key_of(w) == kj);
      if (lane == src && eq && !hit) {
        hit = true;
        pos = base + __ffs(eq) - 1;
      }
    }
  }
  return hit;
}

// A warp's queue of ops that take the checked probe, in shared memory:
// kFusedQ words (value << 32 | key), then kFusedQ words (op << 32 | op index).
// `n` is warp-uniform.
struct OpQ {
  uint64_t* kv;
  uint64_t* oi;
  uint32_t n;
};

// The checked probe of the first min(n, 32) queued ops, one per lane
// (warp-wide); the rest move to the front.  Each attempt reads the version of
// the BitHash1 bucket of every op still open, probes that bucket and, for the
// ops still open, the BitHash2 bucket (each round staged in shared memory),
// then the stash.  A hit is acted on at once: a find takes the staged value
// (the word was seen in place), an erase or replace CASes the word it saw and
// probes again if the CAS fails (the word moved).  A miss stands only if no
// word of that version was in transit and the version did not move;
// otherwise the op probes again.  New keys then claim a slot by its free bit;
// keys whose two buckets are full join the warp's eviction queue.
template <int S>
__device__ void fused_checked(const View& v, uint32_t stash_n, const OpPtrs& a, OpQ& rq,
                              EvictQ& q, const List& pend, int resizable, LaneCounters& cnt,
                              OvfCounters& oc, unsigned& retries, int lane, uint64_t* sbuf) {
  __syncwarp();
  const uint32_t mq = rq.n < 32 ? rq.n : 32u;
  const bool has = static_cast<uint32_t>(lane) < mq;
  const uint64_t kv = has ? rq.kv[lane] : 0u;
  const uint64_t oi = has ? rq.oi[lane] : 0u;
  {
    const uint32_t rest = rq.n - mq;
    uint64_t t0 = 0, t1 = 0;
    if (static_cast<uint32_t>(lane) < rest) {
      t0 = rq.kv[32 + lane];
      t1 = rq.oi[32 + lane];
    }
    __syncwarp();
    if (static_cast<uint32_t>(lane) < rest) {
      rq.kv[lane] = t0;
      rq.oi[lane] = t1;
    }
    __syncwarp();
    rq.n = rest;
  }
  const uint32_t op = has ? static_cast<uint32_t>(oi >> 32) : OP_FIND;
  const uint32_t key = has ? key_of(kv) : kEmptyKey;
  const uint32_t val = val_of(kv);
  const uint32_t i = static_cast<uint32_t>(oi);
  const uint32_t b1 = lh_bucket(bithash1(key), v.M, v.p);
  const uint32_t b2 = lh_bucket(bithash2(key), v.M, v.p);
  bool done = !has;
  uint8_t st = ST_NOT_FOUND;
  uint32_t outv = 0;
  uint32_t f1 = 0, s1 = S, f2 = 0, s2 = S;
  bool absent = false;  // a miss that survived the version check
  for (uint32_t attempt = 0;; ++attempt) {
    const bool active = !done && !absent;
    const unsigned need = __ballot_sync(kFull, active);
    if (!need) break;
    if (attempt >= kFusedRetryLimit) {  // never expected: chains end in bounded time
      if (lane == 0) atomicOr(&v.ctrl->err, kErrTimeout);
      break;
    }
    if (attempt) {
      retries += (lane == 0) ? __popc(need) : 0u;
      __nanosleep(64u << min(attempt, 6u));
    }
    const uint32_t v1 = active ? ld_acquire32(v.vers + b1) : 0u;
    // the stash words appended so far by this kernel (read with the probes: a
    // word appended later was in transit from one of the op's buckets, which
    // the second version read catches)
    const uint32_t tail = ld_relaxed32(&v.ctrl->stash_tail);
    PendCas pc{0, 0, 0, 0, 0};
    // the BitHash1 bucket of every open op
    uint32_t m = (active && op == OP_INSERT) ? ld_relaxed32(v.masks + b1) : 0u;
    cnt.probes += __popc(need);
    fused_stage<S>(v, sbuf, need, b1, lane);
    if (active)
      scan_staged_one<kModeMixed, S>(v, sbuf, lane, b1, key, val, op, m, done, st, outv, f1, s1,
                                     pc);
    // the BitHash2 bucket of the ops still open
    const unsigned need2 = __ballot_sync(kFull, active && !done);
    if (need2) {
      m = (active && !done && op == OP_INSERT) ? ld_relaxed32(v.masks + b2) : 0u;
      cnt.probes += __popc(need2);
      fused_stage<S>(v, sbuf, need2, b2, lane);
      if (active && !done)
        scan_staged_one<kModeMixed, S>(v, sbuf, lane, b2, key, val, op, m, done, st, outv, f2,
                                       s2, pc);
    }
    // an erase or replace is done once its CAS has succeeded
    bool retry = false;
    if (pc.kind) {
      if (pc.old == pc.cur) {
        if (pc.kind == 1) {
          atomicOr(v.masks + pc.b, 1u << pc.slot);
          cnt.size_delta -= 1;
        } else {
          cnt.replaced += 1;
        }
      } else {
        done = false;
        retry = true;
        st = ST_NOT_FOUND;
      }
    }
    // the stash: the sorted prefix, then what this kernel appended
    const bool miss = active && !done && !retry;
    uint32_t pos = 0;
    bool shit = false;
    if (miss && stash_n) {
      cnt.stash_lookups += 1;
      shit = stash_find(v, stash_n, key, pos);
    }
    const unsigned tneed = __ballot_sync(kFull, miss && !shit);
    if (tneed && tail > stash_n) {
      uint32_t tp = 0;
      if (stash_tail_find(v, stash_n, min(tail, v.stash_cap), tneed, key, lane, tp) && miss &&
          !shit) {
        shit = true;
        pos = tp;
      }
    }
    if (shit) {
      uint64_t* sp = v.stash_kv + pos;
      const uint64_t w = ld_relaxed64(sp);
      if (key_of(w) == key) {
        if (op == OP_FIND) {
          done = true;
          outv = val_of(w);
          st = ST_FOUND;
        } else if (op == OP_ERASE) {
          if (atomicCAS(ull(sp), w, kEmptyWord) == w) {
            done = true;
            st = ST_ERASED;
            cnt.size_delta -= 1;
            atomicExch(&v.ctrl->stash_dirty, 1u);
          } else {
            retry = true;
          }
        } else {
          if (atomicCAS(ull(sp), w, pack(key, val)) == w) {
            done = true;
            st = ST_REPLACED;
            cnt.replaced += 1;
          } else {
            retry = true;
          }
        }
      }
    }
    if (active && !done && !retry) {
      fence_acq_rel_gpu();
      const uint32_t w1 = ld_relaxed32(v.vers + b1);
      absent = (v1 & kTransitMask) == 0 && v1 == w1;
    }
  }

  // New keys: claim in the preferred bucket (two-choice), else the other;
  // keys that find both full join the eviction queue.
  bool to_evict = false;
  if (absent && op == OP_INSERT) {
    const uint64_t word = pack(key, val);
    const bool first1 = v.placement ? (f1 > 0) : (f1 >= f2);
    const uint32_t tb = first1 ? b1 : b2, ts = first1 ? s1 : s2;
    const uint32_t ob = first1 ? b2 : b1, os = first1 ? s2 : s1;
    bool placed = false;
    if (f1 + f2 > 0) {
      placed = claim_pub<S>(v, tb, word, ts < S ? (1u << ts) : 0u);
      if (!placed && ob != tb) placed = claim_pub<S>(v, ob, word, os < S ? (1u << os) : 0u);
    }
    if (placed) {
      st = ST_INSERTED;
      cnt.size_delta += 1;
      cnt.claimed += 1;
    } else {
      to_evict = true;
      cnt.overflowed += 1;
    }
  }
  if (has) {
    if (a.status && !to_evict) a.status[i] = st;
    if (a.vals_out) a.vals_out[i] = outv;
  }
  const unsigned em = __ballot_sync(kFull, to_evict);
  if (em) {
    // q.n < 32 here, so the queue holds the new entries
    if (to_evict) {
      const uint32_t r = q.n + __popc(em & ((1u << lane) - 1u));
      q.words[r] = pack(key, val);
      q.idx[r] = i;
    }
    q.n += __popc(em);
    if (q.n >= 32) fused_drain<S>(v, q, a.status, pend, resizable, oc, lane);
  }
}

// Ops [32c, 32c + 32) of a mixed batch in the single-kernel mode (one op per
// lane).  Finds and erases probe first without reading versions, since a hit
// needs no check (the word was seen in place): the BitHash1 bucket of each,
// then the BitHash2 bucket of those still open, staged in shared memory.
// Their misses, and erases whose CAS failed (the word moved), join the warp's
// queue for the checked probe; so do all inserts, which mostly miss (new
// keys) and would have to probe again.  The checked probe runs 32 queued ops
// at a time.
template <int S>
__device__ __forceinline__ void run_chunk_fused(const View& v, uint32_t stash_n, const OpPtrs a,
                                                uint32_t c, uint64_t n, const OpIn& in,
                                                const List pend, int resizable,
                                                LaneCounters& cnt, OvfCounters& oc,
                                                unsigned& retries, int lane, uint64_t* sbuf,
                                                OpQ& rq, EvictQ& q) {
  const uint32_t i = (c << 5) + lane;
  const bool valid = i < n;
  const uint32_t op = in.op, key = in.key, val = in.val;
  const bool reserved = valid && key >= kReservedKeyMin;
  const bool live = valid && !reserved;
  cnt.reserved |= reserved;
  const uint32_t b1 = lh_bucket(bithash1(key), v.M, v.p);
  const uint32_t b2 = lh_bucket(bithash2(key), v.M, v.p);
  const bool open = live && op != OP_INSERT;
  bool done = false;
  uint8_t st = reserved ? ST_RESERVED : ST_NOT_FOUND;
  uint32_t outv = 0;
  uint32_t fc = 0, fs = S;  // unused: finds and erases claim nothing
  PendCas pc{0, 0, 0, 0, 0};
  const unsigned need = __ballot_sync(kFull, open);
  if (need) {
    cnt.probes += __popc(need);
    fused_stage<S>(v, sbuf, need, b1, lane);
    if (open)
      scan_staged_one<kModeMixed, S>(v, sbuf, lane, b1, key, val, op, 0u, done, st, outv, fc, fs,
                                     pc);
    const unsigned need2 = __ballot_sync(kFull, open && !done);
    if (need2) {
      cnt.probes += __popc(need2);
      fused_stage<S>(v, sbuf, need2, b2, lane);
      if (open && !done)
        scan_staged_one<kModeMixed, S>(v, sbuf, lane, b2, key, val, op, 0u, done, st, outv, fc,
                                       fs, pc);
    }
  }
  if (pc.kind) {
    if (pc.old == pc.cur) {
      atomicOr(v.masks + pc.b, 1u << pc.slot);  // erases only here
      cnt.size_delta -= 1;
    } else {
      done = false;
      st = ST_NOT_FOUND;
    }
  }
  const bool to_check = live && !done;
  if (valid && !to_check) {
    if (a.status) a.status[i] = st;
    if (a.vals_out) __stcs(a.vals_out + i, outv);
  }
  const unsigned cm = __ballot_sync(kFull, to_check);
  if (cm) {
    // rq.n < 32 here, so the queue holds the new entries
    if (to_check) {
      const uint32_t r = rq.n + __popc(cm & ((1u << lane) - 1u));
      rq.kv[r] = pack(key, val);
      rq.oi[r] = (static_cast<uint64_t>(op) << 32) | i;
    }
    rq.n += __popc(cm);
    if (rq.n >= 32)
      fused_checked<S>(v, stash_n, a, rq, q, pend, resizable, cnt, oc, retries, lane, sbuf);
  }
}

// Shared-memory words per warp of the single-kernel batch: one staging round
// (32 buckets), the checked-probe queue (2 kFusedQ words), then the eviction
// queue (kFusedQ words and kFusedQ indices).
__host__ __device__ constexpr int fused_warp_words(int S) {
  return 32 * S + 3 * static_cast<int>(kFusedQ) + static_cast<int>(kFusedQ) / 2;
}
__host__ __device__ constexpr size_t fused_smem(int S) {
  return static_cast<size_t>(kOpsThreads / 32) * 8u * fused_warp_words(S);
}

template <int S>
__global__ void __launch_bounds__(kOpsThreads, 3)
    k_fused(View v, OpPtrs a, uint64_t n, List pend, int resizable) {
  extern __shared__ __align__(16) uint64_t fused_smem_words[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint64_t* mine = fused_smem_words + static_cast<size_t>(wib) * fused_warp_words(S);
  uint64_t* sbuf = mine;
  OpQ rq{mine + 32 * S, mine + 32 * S + kFusedQ, 0};
  EvictQ q{mine + 32 * S + 2 * kFusedQ, reinterpret_cast<uint32_t*>(mine + 32 * S + 3 * kFusedQ),
           0};
  const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t nchunks = static_cast<uint32_t>((n + 31) >> 5);
  const uint32_t stash_n = v.ctrl->stash_n;
  LaneCounters cnt;
  OvfCounters oc;
  unsigned retries = 0;
  // inputs are loaded one chunk ahead
  OpIn nxt{};
  if (warp0 < nchunks) nxt = load_in<kModeMixed>(a, warp0, n, lane);
  for (uint32_t c = warp0; c < nchunks; c += nwarps) {
    const OpIn cur = nxt;
    if (c + nwarps < nchunks) nxt = load_in<kModeMixed>(a, c + nwarps, n, lane);
    run_chunk_fused<S>(v, stash_n, a, c, n, cur, pend, resizable, cnt, oc, retries, lane, sbuf,
                       rq, q);
  }
  while (rq.n) fused_checked<S>(v, stash_n, a, rq, q, pend, resizable, cnt, oc, retries, lane, sbuf);
  while (q.n) fused_drain<S>(v, q, a.status, pend, resizable, oc, lane);
  // counters: one atomic per counter and block
  // (and the lanes' unused stash reservations go back in one atomic)
  __shared__ unsigned sum[9];
  if (threadIdx.x < 9) sum[threadIdx.x] = 0;
  __syncthreads();
  {
    const unsigned c9[9] = {oc.claim, oc.rounds, oc.locks, oc.to, oc.stash, oc.pend, oc.added,
                            retries, oc.reserved_in ? 1u : 0u};
    oc.reserved_in = nullptr;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const unsigned t = __reduce_add_sync(kFull, c9[k]);
      if (lane == 0 && t) atomicAdd(&sum[k], t);
    }
  }
  flush_counters_block(v, cnt, lane, sbuf, fused_smem_words, fused_warp_words(S));
  if (threadIdx.x == 0) {
    OvfCounters b;
    b.claim = sum[0];
    b.rounds = sum[1];
    b.locks = sum[2];
    b.to = sum[3];
    b.stash = sum[4];
    b.pend = sum[5];
    b.added = sum[6];
    flush_ovf_counters(v, b, true);
    if (sum[7]) atomicAdd(&v.ctrl->stats[kStFusedRetries], static_cast<unsigned long long>(sum[7]));
    if (sum[8]) atomicSub(&v.ctrl->stash_claims, sum[8]);
  }
}

// ----------------------------------------------------------------------------
// Stash maintenance (single CTA)
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint32_t sort_key(uint64_t w) { return key_of(w); }

// Bitonic sort of a[0, P) by key (P a power of two), one CTA.
__device__ void block_bitonic(uint64_t* a, unsigned P) {
  for (unsigned k = 2; k <= P; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      for (unsigned t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
        const unsigned low = t & (j - 1);
        const unsigned i = ((t - low) << 1) | low;
        const unsigned l = i | j;
        const uint64_t x = a[i], y = a[l];
        const bool up = (i & k) == 0;
        if ((sort_key(x) > sort_key(y)) == up) {
          a[i] = y;
          a[l] = x;
        }
      }
      __syncthreads();
    }
  }
}

// One CTA maintains the stash of the table of `v`; `smem` holds
// kMaintSmemWords words.
template <int S>
__device__ void maint_body(const View& v, uint64_t* smem) {
  __shared__ unsigned s_reins, s_live;
  Ctrl* c = v.ctrl;
  const unsigned tail = c->stash_tail;
  const unsigned sorted = c->stash_n;
  const unsigned dirty = c->stash_dirty;
  if (threadIdx.x == 0) {
    s_reins = 0;
    s_live = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the next call's op lists start empty
    c->ovf_n = 0;
    c->pend_n = 0;
  }
  if (tail == sorted && !dirty) return;

  // Move stash words back into a candidate bucket that has room.
  unsigned reins = 0;
  for (unsigned j = threadIdx.x; j < tail; j += blockDim.x) {
    const uint64_t w = v.stash_kv[j];
    if (w == kEmptyWord) continue;
    const uint32_t k = key_of(w);
    const uint32_t b1 = lh_bucket(bithash1(k), v.M, v.p);
    const uint32_t b2 = lh_bucket(bithash2(k), v.M, v.p);
    const uint32_t m1 = ld_relaxed32(v.masks + b1);
    bool ok = m1 && claim_store<S>(v, b1, __ffs(m1) - 1, w);
    if (!ok) {
      const uint32_t m2 = ld_relaxed32(v.masks + b2);
      ok = m2 && claim_store<S>(v, b2, __ffs(m2) - 1, w);
    }
    if (ok) {
      v.stash_kv[j] = kEmptyWord;
      ++reins;
    }
  }
  if (reins) atomicAdd(&s_reins, reins);
  __syncthreads();

  unsigned P = 1;
  while (P < tail) P <<= 1;
  if (P <= kMaintSmemWords) {
    for (unsigned j = threadIdx.x; j < P; j += blockDim.x) smem[j] = j < tail ? v.stash_kv[j] : kEmptyWord;
    __syncthreads();
    block_bitonic(smem, P);
    for (unsigned j = threadIdx.x; j < P; j += blockDim.x) v.stash_kv[j] = smem[j];
  } else {
    // [tail, P) is EMPTY by construction: the buffer is a power of two long
    // and every word past the live prefix is reset to EMPTY below.
    block_bitonic(v.stash_kv, P);
  }
  __syncthreads();

  // EMPTY words sort last: the live prefix ends at the first EMPTY word.
  unsigned live = 0;
  for (unsigned j = threadIdx.x; j < P; j += blockDim.x) {
    const uint64_t w = v.stash_kv[j];
    if (w != kEmptyWord) {
      v.stash_keys[j] = key_of(w);
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

template <int S>
__global__ void __launch_bounds__(kMaintThreads) k_maint(View v) {
  extern __shared__ uint64_t smem[];
  maint_body<S>(v, smem);
}

// ----------------------------------------------------------------------------
// Linear-hashing resize (Section IV-C)
// ----------------------------------------------------------------------------

// Expansion: warp w splits bucket src0 + w into its partner src0 + w + half.
// `v` carries the state after this launch.  A word leaves the source bucket
// when neither candidate address equals the source under the new state; it
// then belongs to the partner, where the movers are packed from slot 0 by a
// ballot-rank compaction.
template <int S>
__device__ __forceinline__ void split_pair(const View& v, uint32_t src, uint32_t half, int lane) {
  const uint32_t dst = src + half;
  uint64_t* sb = v.buckets + static_cast<uint64_t>(src) * S;
  uint64_t* db = v.buckets + static_cast<uint64_t>(dst) * S;
  const uint64_t word = lane < S ? sb[lane] : kEmptyWord;
  bool mv = false;
  if (word != kEmptyWord) {
    const uint32_t k = key_of(word);
    const uint32_t a1 = lh_bucket(bithash1(k), v.M, v.p);
    const uint32_t a2 = lh_bucket(bithash2(k), v.M, v.p);
    mv = (a1 != src) && (a2 != src);
  }
  const unsigned mm = __ballot_sync(kFull, mv);
  if (mv) {
    db[__popc(mm & ((1u << lane) - 1u))] = word;
    sb[lane] = kEmptyWord;
  }
  if (lane == 0) {
    constexpr uint32_t kValid = S >= 32 ? 0xFFFFFFFFu : ((1u << S) - 1u);
    v.masks[src] |= mm;
    const int nm = __popc(mm);
    v.masks[dst] = nm >= 32 ? 0u : ((0xFFFFFFFFu << nm) & kValid);
  }
}

template <int S>
__global__ void __launch_bounds__(256) k_split(View v, uint32_t src0, uint32_t count, uint32_t half) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= count) return;
  split_pair<S>(v, src0 + w, half, threadIdx.x & 31);
}

// Contraction pre-check: how many words of the batch's high buckets do not
// fit into the free slots of their low partner.
template <int S>
__global__ void __launch_bounds__(256) k_merge_excess(View v, uint32_t count) {
  const int lane = threadIdx.x & 31;
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= count) return;
  const uint32_t low = v.p + w;
  const uint32_t high = low + v.M + 1u;
  const uint64_t word =
      lane < S ? v.buckets[static_cast<uint64_t>(high) * S + lane] : kEmptyWord;
  const int live = __popc(__ballot_sync(kFull, word != kEmptyWord));
  const int fr = __popc(v.masks[low]);
  if (lane == 0 && live > fr) atomicAdd(&v.ctrl->merge_excess, static_cast<unsigned>(live - fr));
}

// Contraction: warp w merges high bucket (p + w + 2^m) into low bucket p + w,
// `v` carrying the state after this launch.  Live words take the free slots
// of the low bucket in rank order (select the r-th free bit); words that do
// not fit go to the overflow list and are placed by the eviction kernel.
template <int S>
__global__ void __launch_bounds__(256) k_merge(View v, uint32_t count, List ovf) {
  const int lane = threadIdx.x & 31;
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= count) return;
  const uint32_t low = v.p + w;
  const uint32_t high = low + v.M + 1u;
  uint64_t* lb = v.buckets + static_cast<uint64_t>(low) * S;
  uint64_t* hb = v.buckets + static_cast<uint64_t>(high) * S;
  const uint64_t word = lane < S ? hb[lane] : kEmptyWord;
  const bool live = word != kEmptyWord;
  const unsigned lm = __ballot_sync(kFull, live);
  const unsigned rank = __popc(lm & ((1u << lane) - 1u));
  const uint32_t fr = v.masks[low];
  const unsigned nfree = __popc(fr);
  const bool fits = live && rank < nfree;
  if (fits) {
    uint32_t m = fr;
    for (unsigned t = 0; t < rank; ++t) m &= m - 1u;
    lb[__ffs(m) - 1] = word;
  }
  const bool spill = live && !fits;
  const unsigned sm = __ballot_sync(kFull, spill);
  if (sm) {
    const int leader = __ffs(sm) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(ovf.count, static_cast<unsigned>(__popc(sm)));
    base = __shfl_sync(kFull, base, leader);
    if (spill) {
      const unsigned r = base + __popc(sm & ((1u << lane) - 1u));
      ovf.words[r] = word;
      ovf.idx[r] = kNoOp;
    }
  }
  if (lane < S) hb[lane] = kEmptyWord;
  if (lane == 0) {
    const unsigned used = __popc(lm) < nfree ? __popc(lm) : nfree;
    uint32_t m = fr;
    for (unsigned t = 0; t < used; ++t) m &= m - 1u;
    v.masks[low] = m;
    v.masks[high] = S >= 32 ? 0xFFFFFFFFu : ((1u << S) - 1u);
  }
}

__global__ void k_count_inserts(const uint8_t* __restrict__ ops, uint64_t n, unsigned* out) {
  unsigned c = 0;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    c += ops[i] == OP_INSERT;
  c = __reduce_add_sync(kFull, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ----------------------------------------------------------------------------
// Multi-table batches: many independent tables serviced by one launch per
// phase.  A batch is a list of segments (table, op range); segment s owns the
// 32-op chunks [chunk0_s, chunk0_{s+1}) of the batch.  Each table keeps its own
// control block, so counters, stash and sticky errors stay per table.
// ----------------------------------------------------------------------------

__device__ __forceinline__ OpPtrs seg_ptrs(const MultiSeg& S) {
  return OpPtrs{S.ops, S.keys, S.vals, S.vals_out, nullptr, S.status};
}

// Each warp takes a contiguous run of chunks, so it changes table only at
// segment boundaries and flushes its counters there.
template <int S>
__global__ void __launch_bounds__(kOpsThreads, HIVE_MULTI_MIN_BLOCKS)
    k_multi_ops(const MultiHdr* __restrict__ hdr, const MultiSeg* __restrict__ segs,
                const View* __restrict__ views, List ovf) {
  const int lane = threadIdx.x & 31;
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t total = hdr->total_chunks;
  const uint32_t ns = hdr->n_segs;
  const uint32_t c0 = static_cast<uint32_t>(static_cast<uint64_t>(total) * w / nw);
  const uint32_t c1 = static_cast<uint32_t>(static_cast<uint64_t>(total) * (w + 1) / nw);
  if (c0 >= c1) return;
  uint32_t lo = 0, hi = ns;  // last segment with chunk0 <= c0
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (segs[mid].chunk0 <= c0) lo = mid; else hi = mid;
  }
  uint32_t s = lo;
  View v = views[segs[s].table];
  uint32_t stash_n = v.ctrl->stash_n;
  OpPtrs a = seg_ptrs(segs[s]);
  LaneCounters cnt;
  for (uint32_t c = c0; c < c1; ++c) {
    if (s + 1 < ns && segs[s + 1].chunk0 <= c) {
      flush_counters(v, cnt, lane);
      do {
        ++s;
      } while (s + 1 < ns && segs[s + 1].chunk0 <= c);
      v = views[segs[s].table];
      stash_n = v.ctrl->stash_n;
      a = seg_ptrs(segs[s]);
    }
    run_chunk<kModeMixed, S>(v, stash_n, a, c - segs[s].chunk0, segs[s].n, ovf, s, cnt, lane);
  }
  flush_counters(v, cnt, lane);
}

// Steps 3-4 for the overflow list of a multi-table batch.  Inserts that find
// no room are reported FULL (a resizable table grows before its next batch).
template <int S>
__global__ void __launch_bounds__(kOvfThreads)
    k_multi_overflow(const MultiSeg* __restrict__ segs, const View* __restrict__ views, List in) {
  // one item per group of S lanes at a time
  const int lane = threadIdx.x & 31;
  const unsigned group0 = (blockIdx.x * blockDim.x + threadIdx.x) / S;
  const unsigned ngroups = (gridDim.x * blockDim.x) / S;
  const bool lead = (lane & (S - 1)) == 0;
  const unsigned total = *in.count;
  const List none{nullptr, nullptr, nullptr, nullptr};
  OvfCounters oc;
  for (unsigned it = group0; it < total; it += ngroups) {
    const uint32_t sg = in.seg[it];
    const View v = views[segs[sg].table];
    overflow_item<S>(v, in.words[it], in.idx[it], sg, segs[sg].status, 0, none, oc, lane);
    flush_ovf_counters(v, oc, lead);
  }
  release_reservation(oc, lead);
}

// One CTA per table of the batch: stash maintenance (exits at once when
// nothing changed).  The grid covers every table of the group, so a captured
// graph serves batches of any composition.
template <int S>
__global__ void __launch_bounds__(256)
    k_multi_maint(const MultiHdr* __restrict__ hdr, const View* __restrict__ views,
                  const uint32_t* __restrict__ touched) {
  extern __shared__ uint64_t smem[];
  if (blockIdx.x >= hdr->n_touched) return;
  maint_body<S>(views[touched[blockIdx.x]], smem);
}

// One wave of split launches over many tables: warp w runs pair
// w - pair0 of the job whose range holds w.  Jobs of one wave touch disjoint
// buckets (a table appears in a wave with splits of one round only).
template <int S>
__global__ void __launch_bounds__(256)
    k_multi_split(const MultiJob* __restrict__ jobs, uint32_t n_jobs, uint32_t total_pairs,
                  const View* __restrict__ views) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= total_pairs) return;
  uint32_t lo = 0, hi = n_jobs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jobs[mid].pair0 <= w) lo = mid; else hi = mid;
  }
  const MultiJob J = jobs[lo];
  View v = views[J.table];
  v.M = J.M;
  v.p = J.p;
  split_pair<S>(v, J.src0 + (w - J.pair0), J.half, threadIdx.x & 31);
}

// Size and stash fill of each table of the batch, for the host's resize
// policy (entries of tables outside the batch are left as they were).
__global__ void k_multi_gather(const MultiHdr* __restrict__ hdr, const View* __restrict__ views,
                               const uint32_t* __restrict__ touched,
                               unsigned long long* __restrict__ out) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= hdr->n_touched) return;
  const uint32_t t = touched[j];
  const Ctrl* c = views[t].ctrl;
  out[2 * t] = c->size;
  out[2 * t + 1] = (static_cast<unsigned long long>(c->err) << 32) | c->stash_claims;
}

// BitHash1 and BitHash2 of n keys (hive_hash).
__global__ void k_hash(const uint32_t* __restrict__ keys, uint64_t n, uint32_t* __restrict__ h1,
                       uint32_t* __restrict__ h2) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t k = __ldcs(keys + i);
    if (h1) __stcs(h1 + i, bithash1(k));
    if (h2) __stcs(h2 + i, bithash2(k));
  }
}

__global__ void k_fill_u32(uint32_t* __restrict__ p, uint64_t n, uint32_t value) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    p[i] = value;
}

// Launches a kernel on `s`, inside the table's persisting L2 window over the
// free masks when it has one (a per-launch attribute: the stream is left as
// it was).
template <typename... KArgs, typename... Args>
cudaError_t launch_in_window(const Launch& L, void (*kern)(KArgs...), unsigned grid,
                             unsigned block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  if (L.l2_bytes) {
    at[0].id = cudaLaunchAttributeAccessPolicyWindow;
    at[0].val.accessPolicyWindow.base_ptr = L.l2_base;
    at[0].val.accessPolicyWindow.num_bytes = L.l2_bytes;
    at[0].val.accessPolicyWindow.hitRatio = L.l2_hit;
    at[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    at[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <int MODE, int S, bool DEFER, int THREADS>
cudaError_t launch_ops_tt(const View& v, const OpPtrs& a, uint64_t n, List ovf, const Launch& L,
                          cudaStream_t s) {
  const uint64_t chunks = (n + 31) / 32;
  constexpr uint64_t warps_per_block = THREADS / 32;
  uint64_t blocks = (chunks + warps_per_block - 1) / warps_per_block;
  constexpr bool kStaged = staged_mode(MODE, S);
  const int per_sm = !kStaged ? L.ops_blocks_per_sm
                     : (MODE == kModeInsert ? L.staged_blocks_per_sm : L.staged1_blocks_per_sm);
  const uint64_t cap = static_cast<uint64_t>(L.num_sms) * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  const size_t smem = kStaged ? stage_smem(MODE, S, THREADS) : 0;
  if (MODE == kModeFind) {  // finds touch no free mask
    k_ops<MODE, S, false, THREADS><<<static_cast<unsigned>(blocks), THREADS, smem, s>>>(v, a, n,
                                                                                        ovf, 0);
    return cudaGetLastError();
  }
  // mask prefetch when the batch could touch about one mask sector per 16
  // buckets or more
  const int pf = n * 16 >= v.nb ? 1 : 0;
  return launch_in_window(L, k_ops<MODE, S, DEFER, THREADS>, static_cast<unsigned>(blocks), THREADS,
                          smem, s, v, a, n, ovf, pf);
}

template <int MODE, int S, bool DEFER = false>
cudaError_t launch_ops_t(const View& v, const uint8_t* ops, const uint32_t* keys,
                         const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* found,
                         uint8_t* status, List ovf, const Launch& L, cudaStream_t s) {
  const OpPtrs a{ops, keys, vals, vals_out, found, status};
  switch (L.ops_threads) {
    case 128:
      return launch_ops_tt<MODE, S, DEFER, 128>(v, a, n, ovf, L, s);
    case 512:
      return launch_ops_tt<MODE, S, DEFER, 512>(v, a, n, ovf, L, s);
    default:
      return launch_ops_tt<MODE, S, DEFER, 256>(v, a, n, ovf, L, s);
  }
}

template <int S>
cudaError_t launch_ops_s(int mode, const View& v, const uint8_t* ops, const uint32_t* keys,
                         const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* found,
                         uint8_t* status, List ovf, const Launch& L, cudaStream_t s, bool defer) {
  switch (mode) {
    case kModeFind:
      return launch_ops_t<kModeFind, S>(v, ops, keys, vals, n, vals_out, found, status, ovf, L, s);
    case kModeInsert:
      return launch_ops_t<kModeInsert, S>(v, ops, keys, vals, n, vals_out, found, status, ovf, L, s);
    case kModeErase:
      return launch_ops_t<kModeErase, S>(v, ops, keys, vals, n, vals_out, found, status, ovf, L, s);
    default:
      if (defer)
        return launch_ops_t<kModeMixed, S, true>(v, ops, keys, vals, n, vals_out, found, status, ovf,
                                                 L, s);
      return launch_ops_t<kModeMixed, S>(v, ops, keys, vals, n, vals_out, found, status, ovf, L, s);
  }
}

}  // namespace

cudaError_t launch_fused(const View& v, const uint8_t* ops, const uint32_t* keys,
                         const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* status,
                         List pend, int resizable, const Launch& L, cudaStream_t s) {
  const uint64_t chunks = (n + 31) / 32;
  const uint64_t warps_per_block = kOpsThreads / 32;
  uint64_t blocks = (chunks + warps_per_block - 1) / warps_per_block;
  const uint64_t cap = static_cast<uint64_t>(L.num_sms) * L.fused_blocks_per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  const OpPtrs a{ops, keys, vals, vals_out, nullptr, status};
  if (v.S == 16)
    k_fused<16><<<static_cast<unsigned>(blocks), kOpsThreads, fused_smem(16), s>>>(v, a, n, pend,
                                                                                   resizable);
  else
    k_fused<32><<<static_cast<unsigned>(blocks), kOpsThreads, fused_smem(32), s>>>(v, a, n, pend,
                                                                                   resizable);
  return cudaGetLastError();
}

cudaError_t launch_ops(int mode, const View& v, const uint8_t* ops, const uint32_t* keys,
                       const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* found,
                       uint8_t* status, List ovf, const Launch& L, cudaStream_t s, bool defer) {
  if (v.S == 16)
    return launch_ops_s<16>(mode, v, ops, keys, vals, n, vals_out, found, status, ovf, L, s, defer);
  return launch_ops_s<32>(mode, v, ops, keys, vals, n, vals_out, found, status, ovf, L, s, defer);
}

cudaError_t launch_claim(const View& v, List in, uint64_t n, List out, uint8_t* status,
                         const Launch& L, cudaStream_t s) {
  if (!n) return cudaSuccess;
  const uint32_t nchunks = static_cast<uint32_t>((n + 31) / 32);
  uint64_t blocks = ((nchunks + 31) / 32 + kClaimThreads / 32 - 1) / (kClaimThreads / 32);
  const uint64_t cap = static_cast<uint64_t>(L.num_sms) * L.claim_blocks_per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  // prefetch the masks when the batch could read about one sector per 16
  // buckets or more (a mixed batch of n ops holds at most n new keys)
  const int pf = n * 16 >= v.nb ? 1 : 0;
  if (v.S == 16)
    return launch_in_window(L, k_claim<16>, static_cast<unsigned>(blocks), kClaimThreads, 0, s, v,
                            in, nchunks, out, status, pf);
  return launch_in_window(L, k_claim<32>, static_cast<unsigned>(blocks), kClaimThreads, 0, s, v, in,
                          nchunks, out, status, pf);
}

cudaError_t launch_overflow(const View& v, List in, List pend, int resizable, uint8_t* status,
                            const Launch& L, cudaStream_t s) {
  const unsigned blocks = static_cast<unsigned>(L.num_sms * L.ovf_blocks_per_sm);
  if (v.S == 16)
    return launch_in_window(L, k_overflow<16>, blocks, kOvfThreads, 0, s, v, in, pend, resizable,
                            status);
  return launch_in_window(L, k_overflow<32>, blocks, kOvfThreads, 0, s, v, in, pend, resizable,
                          status);
}

cudaError_t launch_maintenance(const View& v, cudaStream_t s) {
  constexpr size_t smem = kMaintSmemWords * sizeof(uint64_t);
  if (v.S == 16)
    k_maint<16><<<1, kMaintThreads, smem, s>>>(v);
  else
    k_maint<32><<<1, kMaintThreads, smem, s>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_split(const View& v_new, uint32_t src0, uint32_t count, uint32_t half,
                         cudaStream_t s) {
  if (!count) return cudaSuccess;
  const unsigned blocks = (count * 32u + 255u) / 256u;
  if (v_new.S == 16)
    k_split<16><<<blocks, 256, 0, s>>>(v_new, src0, count, half);
  else
    k_split<32><<<blocks, 256, 0, s>>>(v_new, src0, count, half);
  return cudaGetLastError();
}

cudaError_t launch_merge_excess(const View& v_new, uint32_t count, cudaStream_t s) {
  if (!count) return cudaSuccess;
  const unsigned blocks = (count * 32u + 255u) / 256u;
  if (v_new.S == 16)
    k_merge_excess<16><<<blocks, 256, 0, s>>>(v_new, count);
  else
    k_merge_excess<32><<<blocks, 256, 0, s>>>(v_new, count);
  return cudaGetLastError();
}

cudaError_t launch_merge(const View& v_new, uint32_t count, List ovf, cudaStream_t s) {
  if (!count) return cudaSuccess;
  const unsigned blocks = (count * 32u + 255u) / 256u;
  if (v_new.S == 16)
    k_merge<16><<<blocks, 256, 0, s>>>(v_new, count, ovf);
  else
    k_merge<32><<<blocks, 256, 0, s>>>(v_new, count, ovf);
  return cudaGetLastError();
}

cudaError_t launch_count_inserts(const uint8_t* ops, uint64_t n, unsigned* out, cudaStream_t s) {
  if (!n) return cudaSuccess;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_count_inserts<<<static_cast<unsigned>(blocks), 256, 0, s>>>(ops, n, out);
  return cudaGetLastError();
}

cudaError_t launch_hash(const uint32_t* keys, uint64_t n, uint32_t* h1, uint32_t* h2,
                        cudaStream_t s) {
  if (!n) return cudaSuccess;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_hash<<<static_cast<unsigned>(blocks), 256, 0, s>>>(keys, n, h1, h2);
  return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, uint64_t n, uint32_t value, cudaStream_t s) {
  if (!n) return cudaSuccess;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  k_fill_u32<<<static_cast<unsigned>(blocks), 256, 0, s>>>(p, n, value);
  return cudaGetLastError();
}

cudaError_t launch_multi_ops(int S, const MultiHdr* hdr, const MultiSeg* segs, const View* views,
                             List ovf, const Launch& L, cudaStream_t s) {
  const unsigned blocks = static_cast<unsigned>(L.num_sms * L.multi_blocks_per_sm);
  if (S == 16)
    k_multi_ops<16><<<blocks, kOpsThreads, 0, s>>>(hdr, segs, views, ovf);
  else
    k_multi_ops<32><<<blocks, kOpsThreads, 0, s>>>(hdr, segs, views, ovf);
  return cudaGetLastError();
}

cudaError_t launch_multi_overflow(int S, const MultiSeg* segs, const View* views, List in,
                                  const Launch& L, cudaStream_t s) {
  const unsigned blocks = static_cast<unsigned>(L.num_sms * L.ovf_blocks_per_sm);
  if (S == 16)
    k_multi_overflow<16><<<blocks, kOvfThreads, 0, s>>>(segs, views, in);
  else
    k_multi_overflow<32><<<blocks, kOvfThreads, 0, s>>>(segs, views, in);
  return cudaGetLastError();
}

cudaError_t launch_multi_maint(int S, const MultiHdr* hdr, const View* views,
                               const uint32_t* touched, uint32_t max_tables, cudaStream_t s) {
  if (!max_tables) return cudaSuccess;
  constexpr size_t smem = kMaintSmemWords * sizeof(uint64_t);
  if (S == 16)
    k_multi_maint<16><<<max_tables, 256, smem, s>>>(hdr, views, touched);
  else
    k_multi_maint<32><<<max_tables, 256, smem, s>>>(hdr, views, touched);
  return cudaGetLastError();
}

cudaError_t launch_multi_split(int S, const MultiJob* jobs, uint32_t n_jobs, uint32_t total_pairs,
                               const View* views, cudaStream_t s) {
  if (!total_pairs) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((static_cast<uint64_t>(total_pairs) * 32 + 255) / 256);
  if (S == 16)
    k_multi_split<16><<<blocks, 256, 0, s>>>(jobs, n_jobs, total_pairs, views);
  else
    k_multi_split<32><<<blocks, 256, 0, s>>>(jobs, n_jobs, total_pairs, views);
  return cudaGetLastError();
}

cudaError_t launch_multi_gather(const MultiHdr* hdr, const View* views, const uint32_t* touched,
                                uint32_t max_tables, unsigned long long* out, cudaStream_t s) {
  if (!max_tables) return cudaSuccess;
  k_multi_gather<<<(max_tables + 255) / 256, 256, 0, s>>>(hdr, views, touched, out);
  return cudaGetLastError();
}

namespace {
// Shared-memory limits and resident blocks of the bulk kernels of one shape.
template <int S, int T>
cudaError_t occupancy_ops(Launch* L) {
  int b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ops<kModeFind, S, false, T>,
                                                                T, 0);
  if (e != cudaSuccess) return e;
  L->ops_blocks_per_sm = b > 0 ? b : 1;
  e = cudaFuncSetAttribute(k_ops<kModeFind, S, false, T>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(stage_smem(kModeFind, S, T)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ops<kModeInsert, S, false, T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(stage_smem(kModeInsert, S, T)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ops<kModeErase, S, false, T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(stage_smem(kModeErase, S, T)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ops<kModeMixed, S, false, T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(stage_smem(kModeMixed, S, T)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ops<kModeMixed, S, true, T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(stage_smem(kModeMixed, S, T)));
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ops<kModeInsert, S, false, T>, T,
                                                    stage_smem(kModeInsert, S, T));
  if (e != cudaSuccess) return e;
  L->staged_blocks_per_sm = b > 0 ? b : 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ops<kModeMixed, S, false, T>, T,
                                                    stage_smem(kModeMixed, S, T));
  if (e != cudaSuccess) return e;
  L->staged1_blocks_per_sm = b > 0 ? b : 1;
  return cudaSuccess;
}

template <int S>
cudaError_t occupancy_s(Launch* L) {
  int b = 0;
  cudaError_t e = L->ops_threads == 128   ? occupancy_ops<S, 128>(L)
                  : L->ops_threads == 512 ? occupancy_ops<S, 512>(L)
                                          : occupancy_ops<S, 256>(L);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fused<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(fused_smem(S)));
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused<S>, kOpsThreads, fused_smem(S));
  if (e != cudaSuccess) return e;
  L->fused_blocks_per_sm = b > 0 ? b : 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_multi_ops<S>, kOpsThreads, 0);
  if (e != cudaSuccess) return e;
  L->multi_blocks_per_sm = b > 0 ? b : 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_overflow<S>, kOvfThreads, 0);
  if (e != cudaSuccess) return e;
  L->ovf_blocks_per_sm = b > 0 ? b : 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_claim<S>, kClaimThreads, 0);
  if (e != cudaSuccess) return e;
  L->claim_blocks_per_sm = b > 0 ? b : 1;
  const int smem = static_cast<int>(kMaintSmemWords * sizeof(uint64_t));
  e = cudaFuncSetAttribute(k_multi_maint<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_maint<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
}  // namespace

cudaError_t query_occupancy(Launch* L, int S) {
  if (L->ops_threads != 128 && L->ops_threads != 512) L->ops_threads = 256;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&L->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  return S == 16 ? occupancy_s<16>(L) : occupancy_s<32>(L);
}

}  // namespace hive
