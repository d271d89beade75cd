// Host side of the Hive hash table library: the C ABI of include/hive.h, the
// table object, and the sequencing of kernels per call.
//
// Per mutating call the kernels run in phases on the caller's stream:
//   P1  k_ops: finds, erases and replaces (step 1) and claims of new keys
//       (step 2) -- none of these moves an existing key, so they run together;
//   P2  k_overflow: bounded cuckoo eviction and the stash (steps 3-4) for
//       inserts whose candidate buckets were full; no op searches for a key
//       while entries move;
//   M   k_maint: stash maintenance, so the next call sees a compact sorted
//       stash.
// Section III says the paper runs all operations in one monolithic kernel but
// does not show that a lookup cannot miss a key while an eviction carries it
// between buckets; running evictions in their own phase removes that race.
//
// Resizable tables follow the load-factor policy of Section IV-C: before a
// batch, split bucket pairs in launches of at most K pairs (never crossing a
// round) until the worst-case load (size + inserts) is at or under the upper
// threshold; after the batch, merge pairs while the load is under the lower
// threshold and the table is above its initial size.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hive.h"
#include "hive_internal.h"

using namespace hive;

namespace {

thread_local std::string g_err;

hive_status fail(hive_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

hive_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? HIVE_ERR_OOM : HIVE_ERR_CUDA;
}

#define HIVE_CK(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr uint64_t kMaxBuckets = 1ull << 31;

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace


namespace {

cudaEvent_t ev_get(hive_table* t) {
  if (!t->ev_pool.empty()) {
    cudaEvent_t e = t->ev_pool.back();
    t->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch `call` on stream s; with profiling on, bracket it with events.
#define HIVE_LAUNCH(t, kind, s, call)                                       \
  do {                                                                      \
    cudaEvent_t a_ = nullptr;                                               \
    if ((t)->prof) {                                                        \
      a_ = ev_get(t);                                                       \
      cudaEventRecord(a_, (s));                                             \
    }                                                                       \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);                     \
    if ((t)->prof) {                                                        \
      cudaEvent_t b_ = ev_get(t);                                           \
      cudaEventRecord(b_, (s));                                             \
      (t)->recs.push_back(hive_table::Rec{(kind), a_, b_});                 \
    }                                                                       \
  } while (0)

}  // namespace

View hive::make_view(const hive_table* t) {
  View v{};
  v.buckets = t->buckets;
  v.masks = t->masks;
  v.locks = t->locks;
  v.vers = t->locks + t->nb_max;
  v.stash_kv = t->stash_kv;
  v.stash_keys = t->stash_keys;
  v.ctrl = t->ctrl;
  v.M = t->M;
  v.p = t->p;
  v.nb = static_cast<uint32_t>(t->nb);
  v.stash_cap = t->stash_cap;
  v.max_evictions = t->cfg.max_evictions;
  v.lock_spin_limit = t->cfg.lock_spin_limit;
  v.placement = t->cfg.placement;
  v.S = t->S;
  v.stage_spin_limit = t->cfg.stage_wait_limit ? t->cfg.stage_wait_limit : (1u << 22);
  return v;
}

namespace {

List list_a(const hive_table* t) {
  return List{t->la_words, t->la_idx, &t->ctrl->ovf_n, nullptr, t->la_cnt};
}
List list_b(const hive_table* t) { return List{t->lb_words, t->lb_idx, &t->ctrl->pend_n}; }

void free_lists(hive_table* t) {
  cudaFree(t->la_words);
  cudaFree(t->la_idx);
  cudaFree(t->lb_words);
  cudaFree(t->lb_idx);
  cudaFree(t->la_cnt);
  t->la_cnt = nullptr;
  t->la_words = t->lb_words = nullptr;
  t->la_idx = t->lb_idx = nullptr;
  t->list_cap = t->lb_cap = 0;
}

// The op lists hold at most one entry per op of a call (or per word of a
// merge batch), so they grow to the largest call seen.
// List B exists for resizable tables (pending items) and once a mixed batch
// has run (its claim kernel hands full-bucket items from A to B).
hive_status ensure_lists(hive_table* t, uint64_t n, bool need_b = false) {
  const bool two = t->cfg.resizable != 0 || need_b || t->lb_cap != 0;
  if (n <= t->list_cap && (!two || n <= t->lb_cap)) return HIVE_OK;
  const uint64_t cap = std::max<uint64_t>(next_pow2(std::max(n, t->list_cap)), 1u << 16);
  HIVE_CK(cudaDeviceSynchronize());
  free_lists(t);
  cudaError_t e = dev_alloc(&t->la_words, cap * sizeof(uint64_t));
  if (e == cudaSuccess) e = dev_alloc(&t->la_idx, cap * sizeof(uint32_t));
  if (e == cudaSuccess && two) e = dev_alloc(&t->lb_words, cap * sizeof(uint64_t));
  if (e == cudaSuccess && two) e = dev_alloc(&t->lb_idx, cap * sizeof(uint32_t));
  if (e == cudaSuccess && two) e = dev_alloc(&t->la_cnt, cap / 32);
  if (e != cudaSuccess) {
    free_lists(t);
    return cuda_fail(e, "allocating op lists");
  }
  t->list_cap = cap;
  t->lb_cap = two ? cap : 0;
  return HIVE_OK;
}

hive_status readback(hive_table* t, cudaStream_t s) {
  HIVE_CK(cudaMemcpyAsync(t->host_ctrl, t->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  HIVE_CK(cudaStreamSynchronize(s));
  return HIVE_OK;
}

// One expansion launch (Section IV-C1).
hive_status split_step(hive_table* t, cudaStream_t s, bool* did) {
  SplitPlan pl{};
  *did = plan_split(t, &pl);
  if (!*did) return HIVE_OK;
  hive_status st = ensure_committed(t, s);
  if (st != HIVE_OK) return st;
  View v = make_view(t);
  v.M = pl.M;
  v.p = pl.p;
  HIVE_LAUNCH(t, HIVE_K_SPLIT, s, launch_split(v, pl.src0, pl.count, pl.half, s));
  return HIVE_OK;
}

// Buckets in use after the splits that a batch with `live` keys needs.
uint64_t grown_nb(const hive_table* t, uint64_t live) {
  uint64_t M = t->M, p = t->p, nb = t->nb;
  while (over_grow(t, live, nb) && nb < t->nb_max) {
    const uint64_t step = std::min<uint64_t>({t->cfg.resize_batch, M + 1 - p, t->nb_max - nb});
    if (step == 0) break;
    p += step;
    nb += step;
    if (p == M + 1) {
      M = 2 * M + 1;
      p = 0;
    }
  }
  return nb;
}

// Before a batch with up to n_ins new keys.
hive_status grow_for(hive_table* t, uint64_t n_ins, cudaStream_t s) {
  // back every bucket the batch's splits create with one mapping call
  if (t->vmm) {
    const uint64_t nb = grown_nb(t, t->size_host + n_ins);
    HIVE_CK(grow_commit(&t->bucket_vm, nb * t->S * sizeof(uint64_t), s));
  }
  // K-pair steps of one round touch disjoint buckets and are fused into one
  // launch; the policy still advances K pairs at a time.
  bool any = false, have = false;
  SplitPlan acc{};
  while (over_grow(t, t->size_host + n_ins, t->nb) && t->nb < t->nb_max) {
    SplitPlan pl{};
    if (!plan_split(t, &pl)) break;
    any = true;
    if (have && pl.half == acc.half && pl.src0 == acc.src0 + acc.count) {
      acc.count += pl.count;
      acc.M = pl.M;
      acc.p = pl.p;
      continue;
    }
    if (have) {
      hive_status st = ensure_committed(t, s);
      if (st != HIVE_OK) return st;
      View v = make_view(t);
      v.M = acc.M;
      v.p = acc.p;
      HIVE_LAUNCH(t, HIVE_K_SPLIT, s, launch_split(v, acc.src0, acc.count, acc.half, s));
    }
    acc = pl;
    have = true;
  }
  if (have) {
    hive_status st = ensure_committed(t, s);
    if (st != HIVE_OK) return st;
    View v = make_view(t);
    v.M = acc.M;
    v.p = acc.p;
    HIVE_LAUNCH(t, HIVE_K_SPLIT, s, launch_split(v, acc.src0, acc.count, acc.half, s));
  }
  if (any && t->host_ctrl->stash_n) return mark_stash_dirty(t, s);
  return HIVE_OK;
}

// After P1+P2 on a resizable table: place items that found no room by growing,
// then run maintenance, read the size back, and contract while under the lower
// threshold.  `status` receives FULL for ops that still find no room at
// nb_max.  The pending items are in list B, or in list A with !pending_in_b.
hive_status finish_resizable(hive_table* t, uint8_t* status, cudaStream_t s,
                             bool pending_in_b = true) {
  hive_status st = readback(t, s);
  if (st != HIVE_OK) return st;
  bool in_b = pending_in_b;
  while ((in_b ? t->host_ctrl->pend_n : t->host_ctrl->ovf_n) != 0) {
    bool did = false;
    st = split_step(t, s, &did);
    if (st != HIVE_OK) return st;
    View v = make_view(t);
    List in = in_b ? list_b(t) : list_a(t);
    List out = in_b ? list_a(t) : list_b(t);
    HIVE_CK(cudaMemsetAsync(out.count, 0, sizeof(unsigned), s));
    // at nb_max the eviction kernel runs in fixed mode: what still finds no
    // room is reported FULL
    HIVE_LAUNCH(t, HIVE_K_EVICT, s, launch_overflow(v, in, out, did ? 1 : 0, status, t->L, s));
    HIVE_CK(cudaMemsetAsync(in.count, 0, sizeof(unsigned), s));
    st = readback(t, s);
    if (st != HIVE_OK) return st;
    in_b = !in_b;
    if (!did) break;
  }
  if (t->host_ctrl->stash_n) {
    st = mark_stash_dirty(t, s);
    if (st != HIVE_OK) return st;
  }
  HIVE_LAUNCH(t, HIVE_K_MAINT, s, launch_maintenance(make_view(t), s));
  st = readback(t, s);
  if (st != HIVE_OK) return st;
  t->size_host = t->host_ctrl->size;

  return contract_table(t, s);
}

}  // namespace

bool hive::over_grow(const hive_table* t, uint64_t live, uint64_t nb) {
  return static_cast<unsigned __int128>(live) * t->cfg.grow_den >
         static_cast<unsigned __int128>(t->S) * nb * t->cfg.grow_num;
}
bool hive::under_shrink(const hive_table* t, uint64_t live, uint64_t nb) {
  return static_cast<unsigned __int128>(live) * t->cfg.shrink_den <
         static_cast<unsigned __int128>(t->S) * nb * t->cfg.shrink_num;
}


// After a resize the stash may have words that now fit a bucket; make the
// next maintenance pass look at it.
hive_status hive::mark_stash_dirty(hive_table* t, cudaStream_t s) {
  HIVE_CK(cudaMemsetAsync(&t->ctrl->stash_dirty, 1, 1, s));
  return HIVE_OK;
}

hive_status hive::ensure_committed(hive_table* t, cudaStream_t s) {
  if (!t->vmm) return HIVE_OK;
  HIVE_CK(grow_commit(&t->bucket_vm, t->nb * t->S * sizeof(uint64_t), s));
  return HIVE_OK;
}

hive_status hive::contract_table(hive_table* t, cudaStream_t s) {
  // Contraction (Section IV-C2), planned on the host from the size alone.
  // The K-pair steps of one round form a wave: one pre-check of the words that
  // cannot stay in their low bucket, one merge launch, one eviction launch for
  // those words.  Merging moves words and loses none, so the size -- and with
  // it the policy -- needs no read-back between waves.
  hive_status st = HIVE_OK;
  t->merge_deferred = false;
  bool merged = false;
  uint64_t max_wave = ~0ull;
  while (t->nb > t->nb_init && under_shrink(t, t->size_host, t->nb)) {
    uint32_t M = t->M, p = t->p;
    if (p == 0) {
      if (M == 0) break;
      M >>= 1;
      p = M + 1u;
    }
    const uint32_t p_start = p;
    uint64_t nb = t->nb;
    while (nb > t->nb_init && under_shrink(t, t->size_host, nb) && p_start - p < max_wave) {
      const uint64_t step = std::min<uint64_t>({t->cfg.resize_batch, p, nb - t->nb_init});
      if (step == 0 || over_grow(t, t->size_host, nb - step)) break;
      p -= static_cast<uint32_t>(step);
      nb -= step;
      if (p == 0) break;  // the next step regresses the round: next wave
    }
    const uint32_t count = p_start - p;
    if (count == 0) break;
    hive_table trial = *t;
    trial.M = M;
    trial.p = p;
    trial.nb = nb;
    const View vn = make_view(&trial);
    HIVE_CK(cudaMemsetAsync(&t->ctrl->merge_excess, 0, sizeof(unsigned), s));
    HIVE_LAUNCH(t, HIVE_K_MERGE, s, launch_merge_excess(vn, count, s));
    st = readback(t, s);
    if (st != HIVE_OK) return st;
    const uint64_t free_stash = t->stash_cap - t->host_ctrl->stash_claims;
    if (t->host_ctrl->merge_excess > free_stash) {
      if (count > t->cfg.resize_batch) {
        max_wave = t->cfg.resize_batch;  // retry this round one K-step at a time
        continue;
      }
      t->merge_deferred = true;
      break;
    }
    st = ensure_lists(t, static_cast<uint64_t>(count) * t->S);
    if (st != HIVE_OK) return st;
    HIVE_CK(cudaMemsetAsync(&t->ctrl->ovf_n, 0, sizeof(unsigned), s));
    HIVE_LAUNCH(t, HIVE_K_MERGE, s, launch_merge(vn, count, list_a(t), s));
    t->M = trial.M;
    t->p = trial.p;
    t->nb = trial.nb;
    t->merges += count;
    HIVE_LAUNCH(t, HIVE_K_EVICT, s,
                launch_overflow(make_view(t), list_a(t), list_b(t), 0, nullptr, t->L, s));
    merged = true;
  }
  if (merged) {
    HIVE_LAUNCH(t, HIVE_K_MAINT, s, launch_maintenance(make_view(t), s));
    st = readback(t, s);
    if (st != HIVE_OK) return st;
    t->size_host = t->host_ctrl->size;
    if (t->vmm) {
      // the work above has completed; buckets past nb are empty and unused,
      // so whole allocations above them go back
      const size_t need = t->nb * t->S * sizeof(uint64_t);
      if (t->bucket_vm.committed > need + 2 * t->bucket_vm.gran) grow_decommit(&t->bucket_vm, need);
    }
  }
  return HIVE_OK;
}

bool hive::plan_split(hive_table* t, SplitPlan* out) {
  const uint64_t room = static_cast<uint64_t>(t->M) + 1 - t->p;
  const uint64_t step = std::min<uint64_t>({t->cfg.resize_batch, room, t->nb_max - t->nb});
  if (step == 0) return false;
  out->src0 = t->p;
  out->half = t->M + 1u;
  out->count = static_cast<uint32_t>(step);
  t->p += static_cast<uint32_t>(step);
  t->nb += step;
  if (t->p == t->M + 1u) {
    t->M = 2u * t->M + 1u;
    t->p = 0;
  }
  out->M = t->M;
  out->p = t->p;
  t->splits += step;
  return true;
}

namespace {

hive_status check_table(hive_table* t) {
  if (!t) return fail(HIVE_ERR_INVALID_ARG, "table is NULL");
  return HIVE_OK;
}

hive_status check_n(uint64_t n) {
  if (n >= (1ull << 32)) return fail(HIVE_ERR_INVALID_ARG, "n must be below 2^32 per call");
  return HIVE_OK;
}

}  // namespace

namespace hive {
namespace {
std::atomic<uint32_t> g_fail_alloc{0};  // 0: off; n: the n-th allocation from now fails
}  // namespace
cudaError_t dev_alloc_raw(void** p, size_t bytes) {
  uint32_t c = g_fail_alloc.load();
  while (c != 0 && !g_fail_alloc.compare_exchange_weak(c, c - 1)) {
  }
  if (c == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}
void set_fail_alloc(uint32_t n) { g_fail_alloc.store(n); }
bool table_view(const hive_table* t, View* v, Launch* L, bool* resizable) {
  if (!t) return false;
  *v = make_view(t);
  *L = t->L;
  *resizable = t->cfg.resizable != 0;
  return true;
}
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace hive

extern "C" {

void hive_config_default(hive_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->initial_slots = 1ull << 20;
  cfg->max_slots = 1ull << 20;
  cfg->bucket_slots = kSlots;
  cfg->max_evictions = 16;
  cfg->resize_batch = 1024;
  cfg->stash_permille = 10;
  cfg->grow_num = 9;
  cfg->grow_den = 10;
  cfg->shrink_num = 2;
  cfg->shrink_den = 5;
  cfg->resizable = 0;
  cfg->placement = HIVE_PLACE_BALANCED;
  cfg->lock_spin_limit = 1u << 14;
}

// The persisting L2 window of a table's free masks (hive_config.l2_persist):
// as many mask bytes as one window may cover, and a persisting set-aside of
// the context at least that large (never lowered, capped at the device's
// maximum).  With a set-aside smaller than the window, the hit ratio scales
// down so that the persisting lines fit.
static cudaError_t setup_l2_window(hive_table* t) {
  int max_win = 0, max_persist = 0;
  cudaError_t e = cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, t->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, t->device);
  if (e != cudaSuccess) return e;
  if (max_win <= 0 || max_persist <= 0) return cudaSuccess;  // no persisting L2 here
  const size_t bytes = std::min<size_t>(t->nb_max * sizeof(uint32_t), static_cast<size_t>(max_win));
  size_t cur = 0;
  if ((e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize)) != cudaSuccess) return e;
  if (cur < bytes) {
    const size_t want = std::min<size_t>(bytes, static_cast<size_t>(max_persist));
    if ((e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize)) != cudaSuccess) return e;
  }
  if (cur == 0) return cudaSuccess;
  t->L.l2_base = t->masks;
  t->L.l2_bytes = bytes;
  t->L.l2_hit = cur >= bytes ? 1.0f : static_cast<float>(cur) / static_cast<float>(bytes);
  return cudaSuccess;
}

hive_status hive_create(const hive_config* cfg, void* stream, hive_table** out) {
  if (!cfg || !out) return fail(HIVE_ERR_INVALID_ARG, "cfg and out must not be NULL");
  *out = nullptr;
  if (cfg->bucket_slots != 16 && cfg->bucket_slots != 32)
    return fail(HIVE_ERR_INVALID_ARG, "bucket_slots must be 16 or 32");
  if (cfg->initial_slots == 0) return fail(HIVE_ERR_INVALID_ARG, "initial_slots must be > 0");
  if (cfg->max_evictions == 0 || cfg->resize_batch == 0 || cfg->lock_spin_limit == 0)
    return fail(HIVE_ERR_INVALID_ARG, "max_evictions, resize_batch, lock_spin_limit must be > 0");
  if (cfg->grow_den == 0 || cfg->shrink_den == 0 || cfg->grow_num > cfg->grow_den ||
      static_cast<uint64_t>(cfg->shrink_num) * cfg->grow_den >=
          static_cast<uint64_t>(cfg->grow_num) * cfg->shrink_den)
    return fail(HIVE_ERR_INVALID_ARG, "need 0 <= shrink < grow <= 1");
  if (cfg->stash_permille > 1000 || cfg->placement > HIVE_PLACE_FIRST || cfg->blocks_per_sm > 64 ||
      cfg->map_on_demand > 1 || cfg->l2_persist > 1 ||
      (cfg->block_threads != 0 && cfg->block_threads != 128 && cfg->block_threads != 256 &&
       cfg->block_threads != 512) ||
      cfg->resizable > 1)
    return fail(HIVE_ERR_INVALID_ARG,
                "bad stash_permille, placement, resizable, blocks_per_sm, map_on_demand, "
                "l2_persist or block_threads");

  hive_table* t = new (std::nothrow) hive_table();
  if (!t) return fail(HIVE_ERR_OOM, "host allocation failed");
  t->cfg = *cfg;
  t->check_contract = contract_check_env();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t S = cfg->bucket_slots;
  t->S = S;
  t->nb_init = (cfg->initial_slots + S - 1) / S;
  t->nb_max = cfg->resizable ? std::max(t->nb_init, (cfg->max_slots + S - 1) / S) : t->nb_init;
  if (t->nb_max > kMaxBuckets) {
    delete t;
    return fail(HIVE_ERR_INVALID_ARG, "capacity above 2^36 slots");
  }
  t->nb = t->nb_init;
  uint64_t pow2 = 1;
  while (pow2 * 2 <= t->nb_init) pow2 *= 2;
  t->M = static_cast<uint32_t>(pow2 - 1);
  t->p = static_cast<uint32_t>(t->nb_init - pow2);
  const uint64_t cap_slots = t->nb_max * S;
  uint64_t sc = (cap_slots * cfg->stash_permille + 999) / 1000;
  sc = std::max<uint64_t>(sc, 1024);
  sc = (sc + 31) / 32 * 32;
  if (sc > (1ull << 31)) sc = 1ull << 31;
  t->stash_cap = static_cast<uint32_t>(sc);
  t->stash_alloc = next_pow2(sc);

  cudaError_t e = cudaGetDevice(&t->device);
  t->L.ops_threads = cfg->block_threads ? static_cast<int>(cfg->block_threads) : 256;
  if (e == cudaSuccess) e = query_occupancy(&t->L, static_cast<int>(S));
  if (e == cudaSuccess && cfg->blocks_per_sm) {
    const int cap = static_cast<int>(cfg->blocks_per_sm);
    t->L.ops_blocks_per_sm = std::min(t->L.ops_blocks_per_sm, cap);
    t->L.staged_blocks_per_sm = std::min(t->L.staged_blocks_per_sm, cap);
    t->L.staged1_blocks_per_sm = std::min(t->L.staged1_blocks_per_sm, cap);
  }
  if (e == cudaSuccess && cfg->resizable && cfg->map_on_demand) {
    // reserve the address range of nb_max buckets, back only nb_init of them
    if (grow_reserve(&t->bucket_vm, t->nb_max * S * sizeof(uint64_t), t->device) == cudaSuccess) {
      t->vmm = true;
      t->buckets = reinterpret_cast<uint64_t*>(t->bucket_vm.base);
      e = grow_commit(&t->bucket_vm, t->nb_init * S * sizeof(uint64_t), s);
    } else {
      cudaGetLastError();
    }
  }
  if (e == cudaSuccess && !t->vmm)
    e = dev_alloc(&t->buckets, t->nb_max * S * sizeof(uint64_t));
  if (e == cudaSuccess) e = dev_alloc(&t->masks, t->nb_max * sizeof(uint32_t));
  if (e == cudaSuccess) e = dev_alloc(&t->locks, 2 * t->nb_max * sizeof(uint32_t));
  if (e == cudaSuccess) e = dev_alloc(&t->stash_kv, t->stash_alloc * sizeof(uint64_t));
  if (e == cudaSuccess) e = dev_alloc(&t->stash_keys, t->stash_cap * sizeof(uint32_t));
  if (e == cudaSuccess) e = dev_alloc(&t->ctrl, sizeof(Ctrl));
  if (e == cudaSuccess) e = cudaMallocHost(&t->host_ctrl, sizeof(Ctrl));
  if (e == cudaSuccess) {
    std::memset(t->host_ctrl, 0, sizeof(Ctrl));
    if (!t->vmm) e = cudaMemsetAsync(t->buckets, 0xFF, t->nb_max * S * sizeof(uint64_t), s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(t->masks, 0xFF, t->nb_max * sizeof(uint32_t), s);
  if (e == cudaSuccess && S < 32) e = launch_fill_u32(t->masks, t->nb_max, (1u << S) - 1u, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->locks, 0, 2 * t->nb_max * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->stash_kv, 0xFF, t->stash_alloc * sizeof(uint64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->ctrl, 0, sizeof(Ctrl), s);
  if (e == cudaSuccess && cfg->l2_persist) e = setup_l2_window(t);
  if (e != cudaSuccess) {
    hive_status st = cuda_fail(e, "hive_create");
    hive_destroy(t);
    return st;
  }
  *out = t;
  return HIVE_OK;
}

hive_status hive_destroy(hive_table* t) {
  if (!t) return HIVE_OK;
  cudaDeviceSynchronize();
  if (t->vmm)
    grow_free(&t->bucket_vm);
  else
    cudaFree(t->buckets);
  cudaFree(t->masks);
  cudaFree(t->locks);
  cudaFree(t->stash_kv);
  cudaFree(t->stash_keys);
  cudaFree(t->ctrl);
  if (t->host_ctrl) cudaFreeHost(t->host_ctrl);
  free_lists(t);
  free_staging(t);
  for (const auto& r : t->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : t->ev_pool) cudaEventDestroy(e);
  delete t;
  return HIVE_OK;
}

hive_status hive_insert(hive_table* t, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                        uint8_t* status, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if ((st = check_n(n)) != HIVE_OK) return st;
  if (n == 0) return HIVE_OK;
  if (!keys || !vals) return fail(HIVE_ERR_INVALID_ARG, "keys and vals must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (t->check_contract &&
      (st = check_contract_device(nullptr, HIVE_OP_INSERT, keys, n, kReservedKeyMin, s)) != HIVE_OK)
    return st;
  if ((st = ensure_lists(t, n)) != HIVE_OK) return st;
  if (t->cfg.resizable && (st = grow_for(t, n, s)) != HIVE_OK) return st;
  const View v = make_view(t);
  HIVE_LAUNCH(t, HIVE_K_INSERT, s,
              launch_ops(kModeInsert, v, nullptr, keys, vals, n, nullptr, nullptr, status,
                         list_a(t), t->L, s));
  HIVE_LAUNCH(t, HIVE_K_EVICT, s,
              launch_overflow(v, list_a(t), list_b(t), t->cfg.resizable, status, t->L, s));
  if (t->cfg.resizable) return finish_resizable(t, status, s);
  HIVE_LAUNCH(t, HIVE_K_MAINT, s, launch_maintenance(v, s));
  return HIVE_OK;
}

hive_status hive_find(hive_table* t, const uint32_t* keys, uint64_t n, uint32_t* vals_out,
                      uint8_t* found, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if ((st = check_n(n)) != HIVE_OK) return st;
  if (n == 0) return HIVE_OK;
  if (!keys || !vals_out) return fail(HIVE_ERR_INVALID_ARG, "keys and vals_out must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HIVE_LAUNCH(t, HIVE_K_FIND, s,
              launch_ops(kModeFind, make_view(t), nullptr, keys, nullptr, n, vals_out, found,
                         nullptr, list_a(t), t->L, s));
  return HIVE_OK;
}

hive_status hive_erase(hive_table* t, const uint32_t* keys, uint64_t n, uint8_t* status,
                       void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if ((st = check_n(n)) != HIVE_OK) return st;
  if (n == 0) return HIVE_OK;
  if (!keys) return fail(HIVE_ERR_INVALID_ARG, "keys must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (t->check_contract &&
      (st = check_contract_device(nullptr, HIVE_OP_ERASE, keys, n, kReservedKeyMin, s)) != HIVE_OK)
    return st;
  const View v = make_view(t);
  HIVE_LAUNCH(t, HIVE_K_ERASE, s,
              launch_ops(kModeErase, v, nullptr, keys, nullptr, n, nullptr, nullptr, status,
                         list_a(t), t->L, s));
  if (t->cfg.resizable) {
    if ((st = ensure_lists(t, 1)) != HIVE_OK) return st;
    return finish_resizable(t, status, s);
  }
  HIVE_LAUNCH(t, HIVE_K_MAINT, s, launch_maintenance(v, s));
  return HIVE_OK;
}

// Mixed batches of at least this many ops claim their new keys in a second
// kernel (launch_claim) after every find, erase and replace: at high load the
// slots the batch's erases free then take most of the keys whose buckets
// were full when probed.  Smaller batches claim in the bulk kernel and save
// the launch.
constexpr uint64_t kDeferMin = 1u << 18;

hive_status hive_execute(hive_table* t, const uint8_t* ops, const uint32_t* keys,
                         const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* status,
                         void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if ((st = check_n(n)) != HIVE_OK) return st;
  if (n == 0) return HIVE_OK;
  if (!ops || !keys) return fail(HIVE_ERR_INVALID_ARG, "ops and keys must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (t->check_contract &&
      (st = check_contract_device(ops, HIVE_OP_FIND, keys, n, kReservedKeyMin, s)) != HIVE_OK)
    return st;
  if ((st = ensure_lists(t, n, true)) != HIVE_OK) return st;
  if (t->cfg.resizable) {
    HIVE_CK(cudaMemsetAsync(&t->ctrl->n_insert, 0, sizeof(unsigned), s));
    HIVE_LAUNCH(t, HIVE_K_COUNT, s, launch_count_inserts(ops, n, &t->ctrl->n_insert, s));
    if ((st = readback(t, s)) != HIVE_OK) return st;
    if ((st = grow_for(t, t->host_ctrl->n_insert, s)) != HIVE_OK) return st;
  }
  const View v = make_view(t);
  // Both op lists are empty here: every mutating call ends with the
  // maintenance kernel, which resets their counts.
  if (n < kDeferMin) {
    // P1 with the claims of new keys, then eviction and stash for the keys
    // whose buckets were both full
    HIVE_LAUNCH(t, HIVE_K_MIXED, s,
                launch_ops(kModeMixed, v, ops, keys, vals, n, vals_out, nullptr, status,
                           list_a(t), t->L, s));
    HIVE_LAUNCH(t, HIVE_K_EVICT, s,
                launch_overflow(v, list_a(t), list_b(t), t->cfg.resizable, status, t->L, s));
    if (t->cfg.resizable) return finish_resizable(t, status, s);
    HIVE_LAUNCH(t, HIVE_K_MAINT, s, launch_maintenance(v, s));
    return HIVE_OK;
  }
  // P1: finds, erases and replaces; the new keys wait in A chunk by chunk
  // (reading 14: no op of P1 moves a word, and the claims of P2 then see
  // every slot that P1's erases freed)
  HIVE_LAUNCH(t, HIVE_K_MIXED, s,
              launch_ops(kModeMixed, v, ops, keys, vals, n, vals_out, nullptr, status,
                         list_a(t), t->L, s, true));
  // P2: claims (A -> B for keys whose buckets are both full), then eviction
  // and stash (B, with pending items appended to A, whose count is still 0)
  HIVE_LAUNCH(t, HIVE_K_CLAIM, s, launch_claim(v, list_a(t), n, list_b(t), status, t->L, s));
  HIVE_LAUNCH(t, HIVE_K_EVICT, s,
              launch_overflow(v, list_b(t), list_a(t), t->cfg.resizable, status, t->L, s));
  if (t->cfg.resizable) return finish_resizable(t, status, s, false);
  HIVE_LAUNCH(t, HIVE_K_MAINT, s, launch_maintenance(v, s));
  return HIVE_OK;
}

hive_status hive_execute_fused(hive_table* t, const uint8_t* ops, const uint32_t* keys,
                               const uint32_t* vals, uint64_t n, uint32_t* vals_out,
                               uint8_t* status, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if ((st = check_n(n)) != HIVE_OK) return st;
  if (n == 0) return HIVE_OK;
  if (!ops || !keys) return fail(HIVE_ERR_INVALID_ARG, "ops and keys must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (t->check_contract &&
      (st = check_contract_device(ops, HIVE_OP_FIND, keys, n, kReservedKeyMin, s)) != HIVE_OK)
    return st;
  if ((st = ensure_lists(t, n)) != HIVE_OK) return st;
  if (t->cfg.resizable) {
    HIVE_CK(cudaMemsetAsync(&t->ctrl->n_insert, 0, sizeof(unsigned), s));
    HIVE_LAUNCH(t, HIVE_K_COUNT, s, launch_count_inserts(ops, n, &t->ctrl->n_insert, s));
    if ((st = readback(t, s)) != HIVE_OK) return st;
    if ((st = grow_for(t, t->host_ctrl->n_insert, s)) != HIVE_OK) return st;
  }
  // inserts that find no room at all go to list B, the pending list that
  // finish_resizable drains
  HIVE_LAUNCH(t, HIVE_K_FUSED, s,
              launch_fused(make_view(t), ops, keys, vals, n, vals_out, status, list_b(t),
                           t->cfg.resizable, t->L, s));
  if (t->cfg.resizable) return finish_resizable(t, status, s);
  HIVE_LAUNCH(t, HIVE_K_MAINT, s, launch_maintenance(make_view(t), s));
  return HIVE_OK;
}

hive_status hive_size(hive_table* t, uint64_t* out, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (!out) return fail(HIVE_ERR_INVALID_ARG, "out must not be NULL");
  if ((st = readback(t, static_cast<cudaStream_t>(stream))) != HIVE_OK) return st;
  *out = t->host_ctrl->size;
  return HIVE_OK;
}

hive_status hive_reserve(hive_table* t, uint64_t slots, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (!t->cfg.resizable) {
    if (slots <= t->nb * t->S) return HIVE_OK;
    return fail(HIVE_ERR_INVALID_ARG, "a fixed-capacity table cannot grow");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool any = false;
  while (t->nb * t->S < slots && t->nb < t->nb_max) {
    bool did = false;
    if ((st = split_step(t, s, &did)) != HIVE_OK) return st;
    if (!did) break;
    any = true;
  }
  if (any) {
    // stash words may now fit a bucket
    if ((st = mark_stash_dirty(t, s)) != HIVE_OK) return st;
    HIVE_LAUNCH(t, HIVE_K_MAINT, s, launch_maintenance(make_view(t), s));
  }
  return HIVE_OK;
}

hive_status hive_memory(hive_table* t, uint64_t* committed, uint64_t* reserved) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (!committed || !reserved) return fail(HIVE_ERR_INVALID_ARG, "outputs must not be NULL");
  const uint64_t bucket_max = t->nb_max * t->S * sizeof(uint64_t);
  const uint64_t bucket_now = t->vmm ? t->bucket_vm.committed : bucket_max;
  const uint64_t other = t->nb_max * 3 * sizeof(uint32_t) + t->stash_alloc * sizeof(uint64_t) +
                         t->stash_cap * sizeof(uint32_t) + sizeof(Ctrl) +
                         (t->list_cap + t->lb_cap) * 12 + t->lb_cap / 32;
  *committed = bucket_now + other;
  *reserved = bucket_max + other;
  return HIVE_OK;
}

hive_status hive_capacity(hive_table* t, uint64_t* slots_out) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (!slots_out) return fail(HIVE_ERR_INVALID_ARG, "slots_out must not be NULL");
  *slots_out = t->nb * t->S;
  return HIVE_OK;
}

hive_status hive_clear(hive_table* t, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Buckets at or past nb are kept empty by construction; only [0, nb) and
  // the stash need resetting.
  HIVE_CK(cudaMemsetAsync(t->buckets, 0xFF, t->nb * t->S * sizeof(uint64_t), s));
  HIVE_CK(cudaMemsetAsync(t->masks, 0xFF, t->nb * sizeof(uint32_t), s));
  if (t->S < 32) HIVE_CK(launch_fill_u32(t->masks, t->nb, (1u << t->S) - 1u, s));
  HIVE_CK(cudaMemsetAsync(t->locks, 0, t->nb * sizeof(uint32_t), s));
  HIVE_CK(cudaMemsetAsync(t->stash_kv, 0xFF, t->stash_alloc * sizeof(uint64_t), s));
  HIVE_CK(cudaMemsetAsync(t->ctrl, 0, sizeof(Ctrl), s));
  t->nb = t->nb_init;
  uint64_t pow2 = 1;
  while (pow2 * 2 <= t->nb_init) pow2 *= 2;
  t->M = static_cast<uint32_t>(pow2 - 1);
  t->p = static_cast<uint32_t>(t->nb_init - pow2);
  t->size_host = 0;
  t->splits = t->merges = 0;
  std::memset(t->host_ctrl, 0, sizeof(Ctrl));
  return HIVE_OK;
}

hive_status hive_check(hive_table* t, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = readback(t, s)) != HIVE_OK) return st;
  const unsigned err = t->host_ctrl->err;
  HIVE_CK(cudaMemsetAsync(&t->ctrl->err, 0, sizeof(unsigned), s));
  HIVE_CK(cudaStreamSynchronize(s));
  if (err & kErrReserved) return fail(HIVE_ERR_RESERVED_KEY, "an op used a reserved key");
  if (err & kErrFull) return fail(HIVE_ERR_FULL, "an insert found no room (FULL)");
  if (err & kErrTimeout)
    return fail(HIVE_ERR_TIMEOUT, "a bounded wait gave up (bucket lock or staged copies)");
  if (err & kErrContract) return fail(HIVE_ERR_CONTRACT, "one key was updated twice in a call");
  return HIVE_OK;
}

hive_status hive_hash(const uint32_t* keys, uint64_t n, uint32_t* h1_out, uint32_t* h2_out,
                      void* stream) {
  if (n == 0) return HIVE_OK;
  if (!keys || (!h1_out && !h2_out))
    return fail(HIVE_ERR_INVALID_ARG, "keys and at least one output must not be NULL");
  HIVE_CK(launch_hash(keys, n, h1_out, h2_out, static_cast<cudaStream_t>(stream)));
  return HIVE_OK;
}

hive_status hive_debug_fail_alloc(uint32_t n) {
  set_fail_alloc(n);
  return HIVE_OK;
}

hive_status hive_debug_hold_lock(hive_table* t, uint64_t bucket, int held, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (bucket != UINT64_MAX && bucket >= t->nb)
    return fail(HIVE_ERR_INVALID_ARG, "bucket is not in use");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a held lock word is any non-zero value; bytes of 1 make 0x01010101
  const int byte = held ? 1 : 0;
  if (bucket == UINT64_MAX)
    HIVE_CK(cudaMemsetAsync(t->locks, byte, t->nb * sizeof(uint32_t), s));
  else
    HIVE_CK(cudaMemsetAsync(t->locks + bucket, byte, sizeof(uint32_t), s));
  return HIVE_OK;
}

hive_status hive_debug_set_versions(hive_table* t, uint32_t value, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (value & 0xFFFFu)
    return fail(HIVE_ERR_INVALID_ARG, "the low 16 bits (words in transit) must be 0");
  HIVE_CK(launch_fill_u32(t->locks + t->nb_max, t->nb_max, value,
                          static_cast<cudaStream_t>(stream)));
  return HIVE_OK;
}

hive_status hive_stats(hive_table* t, hive_stats_t* out, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (!out) return fail(HIVE_ERR_INVALID_ARG, "out must not be NULL");
  if ((st = readback(t, static_cast<cudaStream_t>(stream))) != HIVE_OK) return st;
  const unsigned long long* c = t->host_ctrl->stats;
  out->replaced = c[kStReplaced];
  out->claimed_fast = c[kStClaimedFast];
  out->overflowed = c[kStOverflowed];
  out->claimed_slow = c[kStClaimedSlow];
  out->evict_rounds = c[kStEvictRounds];
  out->lock_acquired = c[kStLockAcquired];
  out->lock_timeouts = c[kStLockTimeouts];
  out->stashed = c[kStStashed];
  out->pending = c[kStPending];
  out->stash_reinserted = c[kStStashReinserted];
  out->splits = t->splits;
  out->merges = t->merges;
  out->probes = c[kStProbes];
  out->stash_lookups = c[kStStashLookups];
  out->fused_retries = c[kStFusedRetries];
  return HIVE_OK;
}

hive_status hive_profile_enable(hive_table* t, int enable) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  t->prof = enable != 0;
  return HIVE_OK;
}

hive_status hive_profile_read(hive_table* t, hive_profile_t* out) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (!out) return fail(HIVE_ERR_INVALID_ARG, "out must not be NULL");
  for (const auto& r : t->recs) {
    HIVE_CK(cudaEventSynchronize(r.b));
    float ms = 0.f;
    HIVE_CK(cudaEventElapsedTime(&ms, r.a, r.b));
    if (r.kind >= 0 && r.kind < HIVE_K_KINDS) {
      out->ms[r.kind] += ms;
      out->launches[r.kind] += 1;
    }
    t->ev_pool.push_back(r.a);
    t->ev_pool.push_back(r.b);
  }
  t->recs.clear();
  return HIVE_OK;
}

hive_status hive_dump(hive_table* t, hive_image* img, void* stream) {
  hive_status st = check_table(t);
  if (st != HIVE_OK) return st;
  if (!img) return fail(HIVE_ERR_INVALID_ARG, "img must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = readback(t, s)) != HIVE_OK) return st;
  img->nb = t->nb;
  img->S = t->S;
  img->M = t->M;
  img->p = t->p;
  img->reserved0 = 0;
  img->stash_n = t->host_ctrl->stash_tail;
  img->stash_cap = t->stash_cap;
  img->size = t->host_ctrl->size;
  img->pending = t->host_ctrl->pend_n;
  if (!img->buckets) return HIVE_OK;
  if (!img->masks || !img->locks || (!img->stash && img->stash_n))
    return fail(HIVE_ERR_INVALID_ARG, "image arrays must not be NULL");
  HIVE_CK(cudaMemcpyAsync(img->buckets, t->buckets, t->nb * t->S * sizeof(uint64_t),
                          cudaMemcpyDeviceToHost, s));
  HIVE_CK(cudaMemcpyAsync(img->masks, t->masks, t->nb * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  HIVE_CK(cudaMemcpyAsync(img->locks, t->locks, t->nb * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (img->stash_n)
    HIVE_CK(cudaMemcpyAsync(img->stash, t->stash_kv, img->stash_n * sizeof(uint64_t),
                            cudaMemcpyDeviceToHost, s));
  HIVE_CK(cudaStreamSynchronize(s));
  return HIVE_OK;
}

const char* hive_last_error(void) { return g_err.c_str(); }

}  // extern "C"
