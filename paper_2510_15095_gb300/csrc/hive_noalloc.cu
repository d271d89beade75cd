// hive_insert_noalloc: the fixed-table insert that allocates nothing.
//
// hive_insert keeps its overflow list (the inserts whose two candidate buckets
// were full, handed from the bulk kernel to the eviction kernel) in memory the
// table grows on demand with cudaMalloc, after a device synchronisation.  Some
// callers cannot let that happen: a serving process whose device memory is
// all pre-reserved by another allocator (a raw cudaMalloc there can fail or
// fragment the pool), or a latency-bound loop that must never stall every
// stream behind a device-wide synchronisation.  This entry point runs the
// same three kernels (bulk insert, eviction + stash, stash maintenance) but
// keeps the overflow list in the file-scope array below, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array is a fixed kNoAllocMaxOps entries (12 bytes each, 3 MiB plus a
// counter); every GPU that loads the library holds it until the process
// exits.  All calls share it and it keeps the last call's contents, so each
// call clears the list counter first, and calls whose work overlaps on the
// GPU (for example on two streams) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hive.h"
#include "hive_internal.h"

namespace {

constexpr uint64_t kNoAllocMaxOps = 1ull << 18;

struct NoAllocScratch {
  uint64_t words[kNoAllocMaxOps];  // packed words of overflowing inserts
  uint32_t idx[kNoAllocMaxOps];    // their op indices
  unsigned int count;              // list length
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device.  In host code the symbol is
// only a host-side stand-in, so its address is asked of the runtime, with the
// device current, on the first call there.  The answer belongs to the CUDA
// context that loaded the module: after cudaDeviceReset the next call runs in
// a new context, where the array may sit elsewhere.  So the cached address is
// kept with the id of the context it came from (cuCtxGetId) and asked again
// when the current context's id differs; where the driver offers no context
// ids, the address is asked on every call.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoAllocScratch* g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

struct CtxIds {
  bool ok = false;
  CUresult (*current)(CUcontext*) = nullptr;
  CUresult (*id)(CUcontext, unsigned long long*) = nullptr;
};

template <class F>
bool fetch_entry(const char* name, F* out) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  *out = reinterpret_cast<F>(p);
  return true;
}

const CtxIds& ctx_ids() {
  static CtxIds c = [] {
    CtxIds r;
    r.ok = fetch_entry("cuCtxGetCurrent", &r.current) && fetch_entry("cuCtxGetId", &r.id);
    return r;
  }();
  return c;
}

// Id of the calling thread's current context (0: unknown).
unsigned long long current_ctx_id() {
  const CtxIds& c = ctx_ids();
  if (!c.ok) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (c.current(&ctx) != CUDA_SUCCESS || !ctx || c.id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

cudaError_t scratch_address(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // cudaGetDevice leaves the device's primary context current for the
  // runtime, so the id read next is the one kernels of this call run in
  const unsigned long long ctx = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev] || ctx == 0 || ctx != g_ctx_id[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<NoAllocScratch*>(p);
    g_ctx_id[dev] = ctx;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

hive_status noalloc_fail(hive_status s, const std::string& msg) {
  hive::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" hive_status hive_insert_noalloc(hive_table* t, const uint32_t* keys,
                                           const uint32_t* vals, uint64_t n, uint8_t* status,
                                           void* stream) {
  hive::View v{};
  hive::Launch L{};
  bool resizable = false;
  if (!hive::table_view(t, &v, &L, &resizable))
    return noalloc_fail(HIVE_ERR_INVALID_ARG, "hive_insert_noalloc: table is NULL");
  if (resizable)
    return noalloc_fail(HIVE_ERR_INVALID_ARG,
                        "hive_insert_noalloc: only fixed-capacity tables (resizing may allocate)");
  if (n > kNoAllocMaxOps)
    return noalloc_fail(HIVE_ERR_INVALID_ARG,
                        "hive_insert_noalloc: n = " + std::to_string(n) +
                            " exceeds the fixed scratch of " + std::to_string(kNoAllocMaxOps) +
                            " ops; split the batch or use hive_insert");
  if (n == 0) return HIVE_OK;
  if (!keys || !vals)
    return noalloc_fail(HIVE_ERR_INVALID_ARG, "hive_insert_noalloc: keys and vals must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (t->check_contract) {  // HIVE_DEBUG (host memory only)
    const hive_status st =
        hive::check_contract_device(nullptr, HIVE_OP_INSERT, keys, n, hive::kReservedKeyMin, s);
    if (st != HIVE_OK) return st;
  }
  NoAllocScratch* sc = nullptr;
  cudaError_t e = scratch_address(&sc);
  if (e != cudaSuccess)
    return noalloc_fail(HIVE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  const hive::List ovf{sc->words, sc->idx, &sc->count};
  if ((e = cudaMemsetAsync(&sc->count, 0, sizeof(unsigned int), s)) != cudaSuccess ||
      (e = hive::launch_ops(hive::kModeInsert, v, nullptr, keys, vals, n, nullptr, nullptr, status,
                            ovf, L, s)) != cudaSuccess ||
      (e = hive::launch_overflow(v, ovf, hive::List{nullptr, nullptr, nullptr}, 0, status, L, s)) !=
          cudaSuccess ||
      (e = hive::launch_maintenance(v, s)) != cudaSuccess)
    return noalloc_fail(HIVE_ERR_CUDA, std::string("hive_insert_noalloc: ") + cudaGetErrorString(e));
  return HIVE_OK;
}
