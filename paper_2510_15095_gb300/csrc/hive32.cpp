// C ABI of the tables with 32-bit entries (hive32_* in include/hive.h).
//
// Fixed capacity; per call the kernels run in the same phases as the 64-bit
// table: k32_ops (finds, erases, replaces, claims), k32_overflow (eviction and
// stash for inserts whose two buckets were full), k32_maint (stash
// maintenance).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "hive.h"
#include "hive_internal.h"

using namespace hive;

struct hive32_table {
  hive32_config cfg{};
  int device = 0;
  uint64_t nb = 0;
  uint32_t M = 0, p = 0;
  uint32_t stash_cap = 0;
  uint64_t stash_alloc = 0;
  uint32_t* buckets = nullptr;
  uint32_t* masks = nullptr;
  uint32_t* locks = nullptr;
  uint32_t* stash_kv = nullptr;
  uint32_t* stash_keys = nullptr;
  Ctrl* ctrl = nullptr;
  Ctrl* host_ctrl = nullptr;
  uint32_t* list_words = nullptr;
  uint32_t* list_idx = nullptr;
  uint64_t list_cap = 0;
  int num_sms = 0, blocks_per_sm = 1;
  bool check_contract = false;  // HIVE_DEBUG at creation: update calls check the batch contract
};

namespace {

hive_status fail32(hive_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

hive_status cuda_fail32(cudaError_t e, const char* what) {
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? HIVE_ERR_OOM : HIVE_ERR_CUDA;
}

#define H32_CK(call)                                      \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail32(e_, #call); \
  } while (0)

constexpr uint32_t kS = 32;
constexpr uint64_t kMaxBuckets32 = 1ull << 31;

View32 view32(const hive32_table* t) {
  View32 v{};
  v.buckets = t->buckets;
  v.masks = t->masks;
  v.locks = t->locks;
  v.stash_kv = t->stash_kv;
  v.stash_keys = t->stash_keys;
  v.ctrl = t->ctrl;
  v.M = t->M;
  v.p = t->p;
  v.nb = static_cast<uint32_t>(t->nb);
  v.stash_cap = t->stash_cap;
  v.max_evictions = t->cfg.max_evictions;
  v.lock_spin_limit = t->cfg.lock_spin_limit;
  v.layout = static_cast<int>(t->cfg.layout);
  return v;
}

List32 list32(const hive32_table* t) {
  return List32{t->list_words, t->list_idx, &t->ctrl->ovf_n};
}

hive_status check32(const hive32_table* t) {
  if (!t) return fail32(HIVE_ERR_INVALID_ARG, "table is NULL");
  return HIVE_OK;
}

hive_status ensure_list32(hive32_table* t, uint64_t n) {
  if (n <= t->list_cap) return HIVE_OK;
  uint64_t cap = 1u << 16;
  while (cap < n) cap <<= 1;
  H32_CK(cudaDeviceSynchronize());
  cudaFree(t->list_words);
  cudaFree(t->list_idx);
  t->list_words = nullptr;
  t->list_idx = nullptr;
  t->list_cap = 0;
  cudaError_t e = cudaMalloc(&t->list_words, cap * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&t->list_idx, cap * sizeof(uint32_t));
  if (e != cudaSuccess) return cuda_fail32(e, "allocating the overflow list");
  t->list_cap = cap;
  return HIVE_OK;
}

hive_status readback32(hive32_table* t, cudaStream_t s) {
  H32_CK(cudaMemcpyAsync(t->host_ctrl, t->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  H32_CK(cudaStreamSynchronize(s));
  return HIVE_OK;
}

// One batch: bulk kernel, then (for batches with inserts) eviction and
// stash, then stash maintenance.
hive_status run32(hive32_table* t, int mode, const uint8_t* ops, const uint32_t* keys,
                  const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* found,
                  uint8_t* status, cudaStream_t s) {
  hive_status st = check32(t);
  if (st != HIVE_OK) return st;
  if (n >= (1ull << 32)) return fail32(HIVE_ERR_INVALID_ARG, "n must be below 2^32 per call");
  if (n == 0) return HIVE_OK;
  if (!keys) return fail32(HIVE_ERR_INVALID_ARG, "keys must not be NULL");
  if (mode == kModeMixed && !ops) return fail32(HIVE_ERR_INVALID_ARG, "ops must not be NULL");
  if (mode == kModeInsert && !vals && t->cfg.layout != HIVE32_KEY_ONLY)
    return fail32(HIVE_ERR_INVALID_ARG, "vals must not be NULL");
  const bool ins = mode == kModeInsert || mode == kModeMixed;
  if (t->check_contract && mode != kModeFind) {
    const uint32_t op = mode == kModeInsert ? HIVE_OP_INSERT : mode == kModeErase ? HIVE_OP_ERASE
                                                                                  : HIVE_OP_FIND;
    const uint32_t key_limit = t->cfg.layout == HIVE32_KEY16_VAL16 ? 0xFFFEu : 0xFFFFFFFEu;
    if ((st = check_contract_device(mode == kModeMixed ? ops : nullptr, op, keys, n, key_limit, s)) !=
        HIVE_OK)
      return st;
  }
  if (ins && (st = ensure_list32(t, n)) != HIVE_OK) return st;
  const View32 v = view32(t);
  const Ops32 a{ops, keys, vals, vals_out, found, status};
  H32_CK(launch32_ops(mode, v, a, n, list32(t), t->num_sms, s));
  if (ins) H32_CK(launch32_overflow(v, list32(t), status, t->num_sms * 8, s));
  if (mode != kModeFind) H32_CK(launch32_maint(v, s));
  return HIVE_OK;
}

void free32(hive32_table* t) {
  cudaFree(t->buckets);
  cudaFree(t->masks);
  cudaFree(t->locks);
  cudaFree(t->stash_kv);
  cudaFree(t->stash_keys);
  cudaFree(t->ctrl);
  cudaFree(t->list_words);
  cudaFree(t->list_idx);
  if (t->host_ctrl) cudaFreeHost(t->host_ctrl);
}

}  // namespace

extern "C" {

void hive32_config_default(hive32_config* cfg) {
  if (!cfg) return;
  cfg->slots = 1u << 20;
  cfg->layout = HIVE32_KEY16_VAL16;
  cfg->max_evictions = 16;
  cfg->stash_permille = 10;
  cfg->lock_spin_limit = 1u << 16;
}

hive_status hive32_create(const hive32_config* cfg, void* stream, hive32_table** out) {
  if (!cfg || !out) return fail32(HIVE_ERR_INVALID_ARG, "cfg and out must not be NULL");
  *out = nullptr;
  if (cfg->layout != HIVE32_KEY16_VAL16 && cfg->layout != HIVE32_KEY_ONLY)
    return fail32(HIVE_ERR_INVALID_ARG, "layout must be HIVE32_KEY16_VAL16 or HIVE32_KEY_ONLY");
  if (cfg->slots < kS) return fail32(HIVE_ERR_INVALID_ARG, "slots must be at least 32");
  if (cfg->max_evictions < 1 || cfg->max_evictions > 64)
    return fail32(HIVE_ERR_INVALID_ARG, "max_evictions must be in 1..64");
  if (cfg->lock_spin_limit == 0) return fail32(HIVE_ERR_INVALID_ARG, "lock_spin_limit must be > 0");
  if (cfg->stash_permille > 1000) return fail32(HIVE_ERR_INVALID_ARG, "stash_permille must be <= 1000");
  const uint64_t nb = (cfg->slots + kS - 1) / kS;
  if (nb > kMaxBuckets32) return fail32(HIVE_ERR_INVALID_ARG, "too many slots");
  hive32_table* t = new (std::nothrow) hive32_table();
  if (!t) return fail32(HIVE_ERR_OOM, "host allocation failed");
  t->cfg = *cfg;
  t->check_contract = contract_check_env();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->nb = nb;
  uint64_t pow2 = 1;
  while (pow2 * 2 <= nb) pow2 *= 2;
  t->M = static_cast<uint32_t>(pow2 - 1);
  t->p = static_cast<uint32_t>(nb - pow2);
  const uint64_t want = std::max<uint64_t>(1024, (nb * kS * cfg->stash_permille + 999) / 1000);
  t->stash_cap = static_cast<uint32_t>(std::min<uint64_t>((want + 31) / 32 * 32, 1ull << 31));
  uint64_t alloc = 1;
  while (alloc < t->stash_cap) alloc <<= 1;
  t->stash_alloc = alloc;
  cudaError_t e = cudaGetDevice(&t->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device);
  if (e == cudaSuccess) e = setup32(static_cast<int>(cfg->layout), &t->blocks_per_sm);
  if (e == cudaSuccess) e = cudaMalloc(&t->buckets, nb * kS * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&t->masks, nb * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&t->locks, nb * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&t->stash_kv, t->stash_alloc * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&t->stash_keys, t->stash_cap * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&t->ctrl, sizeof(Ctrl));
  if (e == cudaSuccess) e = cudaMallocHost(&t->host_ctrl, sizeof(Ctrl));
  if (e == cudaSuccess) e = cudaMemsetAsync(t->buckets, 0xFF, nb * kS * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->masks, 0xFF, nb * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->locks, 0, nb * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->stash_kv, 0xFF, t->stash_alloc * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->ctrl, 0, sizeof(Ctrl), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    hive_status st = cuda_fail32(e, "hive32_create");
    free32(t);
    delete t;
    return st;
  }
  std::memset(t->host_ctrl, 0, sizeof(Ctrl));
  *out = t;
  return HIVE_OK;
}

hive_status hive32_destroy(hive32_table* t) {
  if (!t) return HIVE_OK;
  cudaDeviceSynchronize();
  free32(t);
  delete t;
  return HIVE_OK;
}

hive_status hive32_insert(hive32_table* t, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                          uint8_t* status, void* stream) {
  return run32(t, kModeInsert, nullptr, keys, vals, n, nullptr, nullptr, status,
               static_cast<cudaStream_t>(stream));
}

hive_status hive32_find(hive32_table* t, const uint32_t* keys, uint64_t n, uint32_t* vals_out,
                        uint8_t* found, void* stream) {
  return run32(t, kModeFind, nullptr, keys, nullptr, n, vals_out, found, nullptr,
               static_cast<cudaStream_t>(stream));
}

hive_status hive32_erase(hive32_table* t, const uint32_t* keys, uint64_t n, uint8_t* status,
                         void* stream) {
  return run32(t, kModeErase, nullptr, keys, nullptr, n, nullptr, nullptr, status,
               static_cast<cudaStream_t>(stream));
}

hive_status hive32_execute(hive32_table* t, const uint8_t* ops, const uint32_t* keys,
                           const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* status,
                           void* stream) {
  return run32(t, kModeMixed, ops, keys, vals, n, vals_out, nullptr, status,
               static_cast<cudaStream_t>(stream));
}

hive_status hive32_size(hive32_table* t, uint64_t* out, void* stream) {
  hive_status st = check32(t);
  if (st != HIVE_OK) return st;
  if (!out) return fail32(HIVE_ERR_INVALID_ARG, "out must not be NULL");
  if ((st = readback32(t, static_cast<cudaStream_t>(stream))) != HIVE_OK) return st;
  *out = t->host_ctrl->size;
  return HIVE_OK;
}

hive_status hive32_clear(hive32_table* t, void* stream) {
  hive_status st = check32(t);
  if (st != HIVE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  H32_CK(cudaMemsetAsync(t->buckets, 0xFF, t->nb * kS * sizeof(uint32_t), s));
  H32_CK(cudaMemsetAsync(t->masks, 0xFF, t->nb * sizeof(uint32_t), s));
  H32_CK(cudaMemsetAsync(t->locks, 0, t->nb * sizeof(uint32_t), s));
  H32_CK(cudaMemsetAsync(t->stash_kv, 0xFF, t->stash_alloc * sizeof(uint32_t), s));
  H32_CK(cudaMemsetAsync(t->ctrl, 0, sizeof(Ctrl), s));
  return HIVE_OK;
}

hive_status hive32_check(hive32_table* t, void* stream) {
  hive_status st = check32(t);
  if (st != HIVE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = readback32(t, s)) != HIVE_OK) return st;
  const unsigned err = t->host_ctrl->err;
  H32_CK(cudaMemsetAsync(&t->ctrl->err, 0, sizeof(unsigned), s));
  H32_CK(cudaStreamSynchronize(s));
  if (err & kErrReserved) return fail32(HIVE_ERR_RESERVED_KEY, "an op used a reserved or out-of-range key");
  if (err & kErrFull) return fail32(HIVE_ERR_FULL, "an insert found no room (FULL)");
  if (err & kErrTimeout) return fail32(HIVE_ERR_TIMEOUT, "a bounded wait gave up");
  if (err & kErrContract) return fail32(HIVE_ERR_CONTRACT, "one key was updated twice in a call");
  return HIVE_OK;
}

hive_status hive32_stats(hive32_table* t, hive_stats_t* out, void* stream) {
  hive_status st = check32(t);
  if (st != HIVE_OK) return st;
  if (!out) return fail32(HIVE_ERR_INVALID_ARG, "out must not be NULL");
  if ((st = readback32(t, static_cast<cudaStream_t>(stream))) != HIVE_OK) return st;
  const unsigned long long* c = t->host_ctrl->stats;
  std::memset(out, 0, sizeof(*out));
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
  out->probes = c[kStProbes];
  return HIVE_OK;
}

hive_status hive32_dump(hive32_table* t, hive32_image* img, void* stream) {
  hive_status st = check32(t);
  if (st != HIVE_OK) return st;
  if (!img) return fail32(HIVE_ERR_INVALID_ARG, "img must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = readback32(t, s)) != HIVE_OK) return st;
  img->nb = t->nb;
  img->M = t->M;
  img->p = t->p;
  img->layout = t->cfg.layout;
  img->stash_n = t->host_ctrl->stash_n;
  img->stash_cap = t->stash_cap;
  img->size = t->host_ctrl->size;
  img->pending = t->host_ctrl->pend_n;
  if (!img->buckets) return HIVE_OK;
  if (!img->masks || !img->locks || !img->stash)
    return fail32(HIVE_ERR_INVALID_ARG, "image arrays must all be given");
  H32_CK(cudaMemcpyAsync(img->buckets, t->buckets, t->nb * kS * sizeof(uint32_t),
                         cudaMemcpyDeviceToHost, s));
  H32_CK(cudaMemcpyAsync(img->masks, t->masks, t->nb * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  H32_CK(cudaMemcpyAsync(img->locks, t->locks, t->nb * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (img->stash_n)
    H32_CK(cudaMemcpyAsync(img->stash, t->stash_kv, img->stash_n * sizeof(uint32_t),
                           cudaMemcpyDeviceToHost, s));
  H32_CK(cudaStreamSynchronize(s));
  return HIVE_OK;
}

}  // extern "C"
