// Internal interface between the host library (hive_host.cpp) and the kernels
// (hive_kernels.cu).  Not installed; the public ABI is include/hive.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hive.h"

namespace hive {

constexpr uint32_t kSlots = 32;                    // default S, slots per bucket (Section III-A)
constexpr uint64_t kEmptyWord = ~0ull;             // empty slot: key 0xFFFFFFFF
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;
constexpr uint32_t kReservedKeyMin = 0xFFFFFFFEu;  // keys >= this are reserved
constexpr uint32_t kNoOp = 0xFFFFFFFFu;            // list entry without a caller op

// Sticky error bits in Ctrl::err.
enum : uint32_t {
  kErrReserved = 1u << 0,
  kErrFull = 1u << 1,
  kErrTimeout = 1u << 2,
  kErrContract = 1u << 3,
};

// Counter slots in Ctrl::stats (same order as hive_stats_t).
enum : int {
  kStReplaced = 0,
  kStClaimedFast,
  kStOverflowed,
  kStClaimedSlow,
  kStEvictRounds,
  kStLockAcquired,
  kStLockTimeouts,
  kStStashed,
  kStPending,
  kStStashReinserted,
  kStSplits,
  kStMerges,
  kStProbes,
  kStStashLookups,
  kStFusedRetries,
  kNumStats = 16
};

// Device-resident control block of one table.
struct alignas(128) Ctrl {
  unsigned long long size;   // live entries (buckets + stash)
  unsigned int stash_n;      // sorted, searchable prefix of the stash
  unsigned int stash_tail;   // append cursor; [stash_n, stash_tail) unsorted
  unsigned int stash_claims; // appended + reserved by running eviction chains
  unsigned int stash_dirty;  // a stash word was erased since the last maintenance
  unsigned int ovf_n;        // entries in the overflow list (P1 -> P2)
  unsigned int pend_n;       // entries in the pending list (no room found)
  unsigned int err;          // sticky error bits
  unsigned int merge_excess; // words a merge batch cannot keep in the low bucket
  unsigned int n_insert;     // insert ops counted in a mixed batch
  unsigned int pad0[5];
  unsigned long long stats[kNumStats];
};

// Everything a kernel needs to reach one table; passed by value.
struct View {
  uint64_t* buckets;     // [nb_max * S] packed words (value << 32 | key)
  uint32_t* masks;       // [nb_max] free masks, bit i set = slot i free
  uint32_t* locks;       // [nb_max] bucket locks (eviction only)
  uint32_t* vers;        // [nb_max] bucket versions (single-kernel batches)
  uint64_t* stash_kv;    // [stash_alloc] stash words, EMPTY padded
  uint32_t* stash_keys;  // [stash_cap] keys of the sorted prefix
  Ctrl* ctrl;
  uint32_t M;            // linear-hashing index mask 2^m - 1
  uint32_t p;            // split pointer
  uint32_t nb;           // buckets in use
  uint32_t stash_cap;    // appends never pass this
  uint32_t max_evictions;
  uint32_t lock_spin_limit;
  uint32_t placement;    // 0 balanced, 1 BitHash1 first
  uint32_t S;            // slots per bucket: 16 or 32
  uint32_t stage_spin_limit;  // tries of a staged-copy wait before it gives up
};

// An op list handed from the bulk kernel to the eviction kernel.
struct List {
  uint64_t* words;
  uint32_t* idx;   // caller op index or kNoOp
  unsigned int* count;
  uint32_t* seg;   // multi-table batches: segment of each entry (else NULL)
  uint8_t* chunk_cnt;  // mixed batches: new keys of each 32-op chunk (see k_claim)
};

// One (table, op range) of a multi-table batch; 64 bytes.
struct MultiSeg {
  uint32_t table;        // index into the batch's view array
  uint32_t n;            // ops
  uint32_t chunk0;       // first 32-op chunk of this segment within the batch
  uint32_t pad;
  const uint8_t* ops;    // HIVE_OP_* per op
  const uint32_t* keys;
  const uint32_t* vals;  // insert values (nullable)
  uint32_t* vals_out;    // find results (nullable)
  uint8_t* status;       // per-op status (nullable)
  uint64_t pad2;
};

// One split launch of one table inside a wave of a multi-table batch.
struct MultiJob {
  uint32_t table, src0, count, half;
  uint32_t pair0;  // first warp of this job within the wave
  uint32_t M, p;   // the table's linear-hashing state after this job
  uint32_t pad;
};

struct MultiHdr {
  uint32_t n_segs, total_chunks, n_tables;
  uint32_t n_touched;  // distinct tables of the batch, listed after the views
};

enum OpMode : int { kModeFind = 0, kModeInsert = 1, kModeErase = 2, kModeMixed = 3 };

struct Launch {
  int num_sms;
  int ops_threads;           // block shape of the bulk kernels: 128, 256 or 512 threads
  int ops_blocks_per_sm;     // bulk kernel, fragments loaded from global memory
  int staged_blocks_per_sm;  // bulk kernel, paired insert rounds staged in shared memory
  int staged1_blocks_per_sm; // bulk kernel, single-bucket rounds staged in shared memory
  int fused_blocks_per_sm;   // single-kernel mixed batch
  int ovf_blocks_per_sm;
  int multi_blocks_per_sm;
  int claim_blocks_per_sm;   // claims of a mixed batch's new keys
  // persisting L2 window over the free masks for the kernels that claim
  // slots (l2_bytes = 0: none)
  void* l2_base;
  size_t l2_bytes;
  float l2_hit;
};

// Kernel launchers (hive_kernels.cu).  Each returns the launch error.
// defer (mixed batches): new keys go to list A chunk by chunk for
// launch_claim instead of claiming in the bulk kernel.
cudaError_t launch_ops(int mode, const View& v, const uint8_t* ops, const uint32_t* keys,
                       const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* found,
                       uint8_t* status, List ovf, const Launch& L, cudaStream_t s,
                       bool defer = false);
cudaError_t launch_overflow(const View& v, List in, List pend, int resizable, uint8_t* status,
                            const Launch& L, cudaStream_t s);
// Claims for the new keys of a mixed batch of n ops, left in `in` chunk by
// chunk by the bulk kernel; items with both buckets full go to `out`.
cudaError_t launch_claim(const View& v, List in, uint64_t n, List out, uint8_t* status,
                         const Launch& L, cudaStream_t s);
cudaError_t launch_maintenance(const View& v, cudaStream_t s);
cudaError_t launch_split(const View& v_new, uint32_t src0, uint32_t count, uint32_t half,
                         cudaStream_t s);
cudaError_t launch_merge_excess(const View& v_new, uint32_t count, cudaStream_t s);
cudaError_t launch_merge(const View& v_new, uint32_t count, List ovf, cudaStream_t s);
cudaError_t launch_fused(const View& v, const uint8_t* ops, const uint32_t* keys,
                         const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* status,
                         List pend, int resizable, const Launch& L, cudaStream_t s);
cudaError_t launch_count_inserts(const uint8_t* ops, uint64_t n, unsigned int* out,
                                 cudaStream_t s);
cudaError_t launch_multi_ops(int S, const MultiHdr* hdr, const MultiSeg* segs, const View* views,
                             List ovf, const Launch& L, cudaStream_t s);
cudaError_t launch_multi_overflow(int S, const MultiSeg* segs, const View* views, List in,
                                  const Launch& L, cudaStream_t s);
cudaError_t launch_multi_maint(int S, const MultiHdr* hdr, const View* views,
                               const uint32_t* touched, uint32_t max_tables, cudaStream_t s);
cudaError_t launch_multi_split(int S, const MultiJob* jobs, uint32_t n_jobs, uint32_t total_pairs,
                               const View* views, cudaStream_t s);
cudaError_t launch_fill_u32(uint32_t* p, uint64_t n, uint32_t value, cudaStream_t s);
cudaError_t launch_hash(const uint32_t* keys, uint64_t n, uint32_t* h1, uint32_t* h2,
                        cudaStream_t s);
cudaError_t launch_multi_gather(const MultiHdr* hdr, const View* views, const uint32_t* touched,
                                uint32_t max_tables, unsigned long long* out, cudaStream_t s);
cudaError_t query_occupancy(Launch* L, int S);

// ---- tables with 32-bit entries (hive32_*) ----
struct View32 {
  uint32_t* buckets;     // [nb * 32] entries
  uint32_t* masks;       // [nb] free masks
  uint32_t* locks;       // [nb] bucket locks (eviction only)
  uint32_t* stash_kv;    // [stash_alloc] stash entries, EMPTY padded
  uint32_t* stash_keys;  // [stash_cap] keys of the sorted prefix
  Ctrl* ctrl;
  uint32_t M, p, nb, stash_cap, max_evictions, lock_spin_limit;
  int layout;            // HIVE32_KEY16_VAL16 or HIVE32_KEY_ONLY
};
struct Ops32 {
  const uint8_t* ops;
  const uint32_t* keys;
  const uint32_t* vals;
  uint32_t* vals_out;
  uint8_t* found;
  uint8_t* status;
};
struct List32 {
  uint32_t* words;
  uint32_t* idx;
  unsigned int* count;
};
cudaError_t launch32_ops(int mode, const View32& v, const Ops32& a, uint64_t n, const List32& ovf,
                         int num_sms, cudaStream_t s);
cudaError_t launch32_overflow(const View32& v, const List32& in, uint8_t* status, int blocks,
                              cudaStream_t s);
cudaError_t launch32_maint(const View32& v, cudaStream_t s);
cudaError_t setup32(int layout, int* blocks_per_sm);

}  // namespace hive

namespace hive {
// A device array on CUDA virtual memory: `reserved` bytes of address space,
// the first `committed` of them backed by physical chunks of `gran` bytes.
struct GrowArray {
  uint64_t base = 0;
  size_t reserved = 0, committed = 0, gran = 0;
  int device = 0;
  std::vector<uint64_t> handles;  // physical allocations, mapped back to back from base
  std::vector<size_t> sizes;      // bytes of each
};
cudaError_t grow_reserve(GrowArray* a, size_t max_bytes, int device);
cudaError_t grow_commit(GrowArray* a, size_t bytes, cudaStream_t s);  // new chunks filled 0xFF
void grow_decommit(GrowArray* a, size_t bytes);  // caller ensures no kernel uses the tail
void grow_free(GrowArray* a);
}  // namespace hive

// Device staging of the host-buffer calls (hive_*_host), two slots.
struct HostIO {
  bool ready = false;
  uint8_t* ops[2] = {nullptr, nullptr};
  uint32_t* keys[2] = {nullptr, nullptr};
  uint32_t* vals[2] = {nullptr, nullptr};
  uint32_t* out[2] = {nullptr, nullptr};
  uint8_t* st[2] = {nullptr, nullptr};
  cudaEvent_t in_ready[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  cudaEvent_t free[2] = {nullptr, nullptr};
  cudaStream_t up = nullptr, down = nullptr;
};

// The table object behind the opaque handle of include/hive.h.
struct hive_table {
  hive_config cfg;
  uint32_t S = 32;  // slots per bucket
  int device = 0;
  hive::Launch L{};
  uint64_t nb_init = 0, nb_max = 0, nb = 0;
  uint32_t M = 0, p = 0;
  uint32_t stash_cap = 0;
  uint64_t stash_alloc = 0;
  uint64_t* buckets = nullptr;
  uint32_t* masks = nullptr;
  uint32_t* locks = nullptr;  // [2 nb_max]: bucket locks, then bucket versions
  uint64_t* stash_kv = nullptr;
  uint32_t* stash_keys = nullptr;
  hive::Ctrl* ctrl = nullptr;
  hive::Ctrl* host_ctrl = nullptr;  // pinned readback buffer
  uint64_t list_cap = 0;         // entries of list A
  uint64_t lb_cap = 0;           // entries of list B (0: not allocated)
  uint64_t* la_words = nullptr;  // list A: bulk kernel -> eviction kernel
  uint32_t* la_idx = nullptr;
  uint8_t* la_cnt = nullptr;     // list A per-chunk counts (mixed batches)
  uint64_t* lb_words = nullptr;  // list B: items that found no room
  uint32_t* lb_idx = nullptr;
  uint64_t size_host = 0;       // exact after each resizable call
  uint64_t splits = 0, merges = 0;
  bool merge_deferred = false;
  // profiling hook: events bracketing each launch while enabled
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> ev_pool;
  HostIO io;  // host-buffer call staging (allocated on first use)
  hive::GrowArray bucket_vm;  // resizable tables: buckets on virtual memory
  bool vmm = false;
  bool check_contract = false;  // HIVE_DEBUG at creation: update calls check the batch contract
};

// Helpers shared by the translation units of the library (hive_host.cpp
// defines these).
namespace hive {
View make_view(const hive_table* t);
// The next expansion launch of a table (Section IV-C1): bucket pairs
// (src0 + i, src0 + i + half) for i < count, leaving the table at (M, p).
struct SplitPlan {
  uint32_t src0, count, half, M, p;
};
// Advances the host-side state of t by one split launch and returns its plan;
// false when the table is at nb_max.
bool plan_split(hive_table* t, SplitPlan* out);
bool over_grow(const hive_table* t, uint64_t live, uint64_t nb);
bool under_shrink(const hive_table* t, uint64_t live, uint64_t nb);
// Contraction loop after a batch (Section IV-C2); reads counters back.
hive_status contract_table(hive_table* t, cudaStream_t s);
hive_status mark_stash_dirty(hive_table* t, cudaStream_t s);
void free_staging(hive_table* t);  // releases the host-buffer call staging
// Resizable tables on virtual memory: back buckets [0, nb) with physical memory.
hive_status ensure_committed(hive_table* t, cudaStream_t s);
bool table_view(const hive_table* t, View* v, Launch* L, bool* resizable);
// Every device allocation of the library goes through here, so that a test
// can make one of them fail on the host (hive_debug_fail_alloc).
cudaError_t dev_alloc_raw(void** p, size_t bytes);
void set_fail_alloc(uint32_t n);  // hive_debug_fail_alloc
template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc_raw(reinterpret_cast<void**>(p), bytes);
}
void set_last_error(const std::string& msg);  // text returned by hive_last_error()
// Batch-contract debugging (hive_contract.cpp): whether HIVE_DEBUG asks for
// the check, and the check of a batch whose arrays the GPU addresses (copied
// to the host on `s` first).
bool contract_check_env();
hive_status check_contract_device(const uint8_t* ops, uint32_t op, const uint32_t* keys,
                                  uint64_t n, uint32_t key_limit, cudaStream_t s);
}  // namespace hive
