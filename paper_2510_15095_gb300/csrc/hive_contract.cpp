// Host-side check of the batch contract (hive_check_batch in include/hive.h).
//
// Section III-D runs all operations of a batch concurrently, so a batch has
// one result only when no key is updated twice in it and, in a mixed batch,
// no key is both updated and searched.  The library does not enforce this on
// the fast path; this check is the debugging aid.  It groups the ops by key
// with a stable two-pass LSD radix sort on the 32-bit key (16 bits a pass), so
// that the ops of one key stay in array order, then walks each group.
//
// With HIVE_DEBUG set in the environment when a table is created, every
// update call on it (multi-table batches included) first copies its key and
// op arrays to the host and runs this check; a batch that fails returns
// HIVE_ERR_INVALID_ARG and queues nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include "hive.h"
#include "hive_internal.h"

namespace hive {
namespace {

bool is_update(uint32_t op) { return op == HIVE_OP_INSERT || op == HIVE_OP_ERASE; }

hive_status host_oom() {
  set_last_error("batch contract check: host allocation failed");
  return HIVE_ERR_OOM;
}

// Indices of the ops whose key is below key_limit, stably sorted by key
// (the ops of one key keep their array order).
std::vector<uint32_t> sorted_by_key(const uint32_t* keys, uint64_t n, uint32_t key_limit) {
  std::vector<uint32_t> idx, tmp;
  idx.reserve(n);
  for (uint64_t i = 0; i < n; ++i)
    if (keys[i] < key_limit) idx.push_back(static_cast<uint32_t>(i));
  tmp.resize(idx.size());
  std::vector<uint64_t> cnt(1u << 16);
  for (int pass = 0; pass < 2; ++pass) {
    const int sh = 16 * pass;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (uint32_t i : idx) ++cnt[(keys[i] >> sh) & 0xFFFF];
    uint64_t run = 0;
    for (auto& c : cnt) {
      const uint64_t x = c;
      c = run;
      run += x;
    }
    for (uint32_t i : idx) tmp[cnt[(keys[i] >> sh) & 0xFFFF]++] = i;
    idx.swap(tmp);
  }
  return idx;
}

}  // namespace

bool contract_check_env() {
  const char* e = std::getenv("HIVE_DEBUG");
  return e && *e && std::string(e) != "0";
}

hive_status check_contract_device(const uint8_t* ops, uint32_t op, const uint32_t* keys,
                                  uint64_t n, uint32_t key_limit, cudaStream_t s) {
  if (n == 0) return HIVE_OK;
  std::vector<uint32_t> hk;
  std::vector<uint8_t> ho;
  try {
    hk.resize(n);
    ho.resize(ops ? n : 0);
  } catch (const std::bad_alloc&) {
    return host_oom();
  }
  cudaError_t e = cudaMemcpyAsync(hk.data(), keys, n * sizeof(uint32_t), cudaMemcpyDefault, s);
  if (e == cudaSuccess && ops) e = cudaMemcpyAsync(ho.data(), ops, n, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(std::string("batch contract check: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return HIVE_ERR_CUDA;
  }
  uint64_t bad = 0;
  return hive_check_batch(ops ? ho.data() : nullptr, op, hk.data(), n, key_limit, &bad);
}

}  // namespace hive

extern "C" hive_status hive_check_batch(const uint8_t* h_ops, uint32_t op, const uint32_t* h_keys,
                                        uint64_t n, uint32_t key_limit, uint64_t* first_bad) {
  using hive::set_last_error;
  if (first_bad) *first_bad = n;
  if (n >= (1ull << 32)) {
    set_last_error("n must be below 2^32 per call");
    return HIVE_ERR_INVALID_ARG;
  }
  if (n == 0) return HIVE_OK;
  if (!h_keys) {
    set_last_error("keys must not be NULL");
    return HIVE_ERR_INVALID_ARG;
  }
  if (!h_ops && !hive::is_update(op)) return HIVE_OK;  // a find batch always passes
  std::vector<uint32_t> idx;
  try {
    idx = hive::sorted_by_key(h_keys, n, key_limit);
  } catch (const std::bad_alloc&) {
    return hive::host_oom();
  }
  // a group is the ops of one key in array order; the first op that makes
  // the prefix [0, i] break the contract is the second update of a key, or
  // an update after a find of it, or a find after an update of it
  uint64_t bad = n;
  for (size_t g = 0; g < idx.size();) {
    size_t end = g + 1;
    while (end < idx.size() && h_keys[idx[end]] == h_keys[idx[g]]) ++end;
    bool upd = false, fnd = false;
    for (size_t j = g; j < end; ++j) {
      const uint32_t i = idx[j];
      const bool u = hive::is_update(h_ops ? h_ops[i] : op);
      if ((u && (upd || fnd)) || (!u && upd)) {
        if (i < bad) bad = i;
        break;
      }
      upd |= u;
      fnd |= !u;
    }
    g = end;
  }
  if (bad == n) return HIVE_OK;
  if (first_bad) *first_bad = bad;
  char msg[160];
  std::snprintf(msg, sizeof msg,
                "batch contract: op %llu repeats key %u of an earlier op (an update twice, "
                "or an update and a find)",
                static_cast<unsigned long long>(bad), h_keys[bad]);
  set_last_error(msg);
  return HIVE_ERR_INVALID_ARG;
}
