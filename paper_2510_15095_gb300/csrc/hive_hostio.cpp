// Host-buffer calls: the op arrays live in host memory.  The batch is cut into
// chunks that stream through two device staging slots: chunk i's inputs go up
// on the copy-in stream while chunk i-1 runs on the caller's stream and chunk
// i-2's results come down on the copy-out stream.  With pinned host buffers
// the three overlap (the C2C link and the kernels work at once); pageable
// buffers still work, the copies then block.  Chunking a batch does not change
// its results under the batch contract.  Each call returns once every output
// is in host memory.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include <algorithm>
#include <atomic>
#include <string>

#include "hive.h"
#include "hive_internal.h"

using namespace hive;

namespace {

#ifndef HIVE_IO_CHUNK_LOG2
#define HIVE_IO_CHUNK_LOG2 22
#endif
constexpr uint64_t kChunkOps = 1ull << HIVE_IO_CHUNK_LOG2;  // ops per chunk and staging slot

hive_status hfail(hive_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

hive_status hcuda(cudaError_t e, const char* what) {
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? HIVE_ERR_OOM : HIVE_ERR_CUDA;
}

#define HCK(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return hcuda(e_, #call); \
  } while (0)

// Staging of one table, allocated on first use and kept until destroy.
hive_status ensure_staging(hive_table* t) {
  HostIO& io = t->io;
  if (io.ready) return HIVE_OK;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = hive::dev_alloc(&io.ops[k], kChunkOps);
    if (e == cudaSuccess) e = hive::dev_alloc(&io.keys[k], kChunkOps * 4);
    if (e == cudaSuccess) e = hive::dev_alloc(&io.vals[k], kChunkOps * 4);
    if (e == cudaSuccess) e = hive::dev_alloc(&io.out[k], kChunkOps * 4);
    if (e == cudaSuccess) e = hive::dev_alloc(&io.st[k], kChunkOps);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io.in_ready[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io.done[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io.free[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io.up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io.down, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_staging(t);
    return hcuda(e, "allocating host-io staging");
  }
  io.ready = true;
  return HIVE_OK;
}

enum Kind { kIns, kFind, kExec };

hive_status run_chunks(hive_table* t, Kind kind, const uint8_t* h_ops, const uint32_t* h_keys,
                       const uint32_t* h_vals, uint64_t n, uint32_t* h_out, uint8_t* h_st,
                       cudaStream_t s) {
  hive_status st = HIVE_OK;
  HostIO& io = t->io;
  const uint64_t chunks = (n + kChunkOps - 1) / kChunkOps;
  for (uint64_t c = 0; c < chunks; ++c) {
    const int k = static_cast<int>(c & 1);
    const uint64_t off = c * kChunkOps;
    const uint64_t m = std::min(kChunkOps, n - off);
    // inputs: after the slot's previous results have been copied out
    HCK(cudaStreamWaitEvent(io.up, io.free[k], 0));
    if (kind == kExec) HCK(cudaMemcpyAsync(io.ops[k], h_ops + off, m, cudaMemcpyHostToDevice, io.up));
    HCK(cudaMemcpyAsync(io.keys[k], h_keys + off, m * 4, cudaMemcpyHostToDevice, io.up));
    if (h_vals && kind != kFind)
      HCK(cudaMemcpyAsync(io.vals[k], h_vals + off, m * 4, cudaMemcpyHostToDevice, io.up));
    HCK(cudaEventRecord(io.in_ready[k], io.up));
    // the op itself, on the caller's stream
    HCK(cudaStreamWaitEvent(s, io.in_ready[k], 0));
    if (kind == kIns)
      st = hive_insert(t, io.keys[k], io.vals[k], m, h_st ? io.st[k] : nullptr, s);
    else if (kind == kFind)
      st = hive_find(t, io.keys[k], m, io.out[k], h_st ? io.st[k] : nullptr, s);
    else
      st = hive_execute(t, io.ops[k], io.keys[k], h_vals ? io.vals[k] : nullptr, m,
                        h_out ? io.out[k] : nullptr, h_st ? io.st[k] : nullptr, s);
    if (st != HIVE_OK) return st;
    HCK(cudaEventRecord(io.done[k], s));
    // results
    HCK(cudaStreamWaitEvent(io.down, io.done[k], 0));
    if (h_out && kind != kIns)
      HCK(cudaMemcpyAsync(h_out + off, io.out[k], m * 4, cudaMemcpyDeviceToHost, io.down));
    if (h_st) HCK(cudaMemcpyAsync(h_st + off, io.st[k], m, cudaMemcpyDeviceToHost, io.down));
    HCK(cudaEventRecord(io.free[k], io.down));
  }
  HCK(cudaStreamSynchronize(io.down));
  return HIVE_OK;
}

// Direct access.  On a GPU whose kernels reach host memory coherently
// through the CPU-GPU link (the device attribute
// PageableMemoryAccessUsesHostPageTables; GB300's NVLink-C2C), pinned or
// registered host arrays go to the device-pointer calls as they are: the
// kernels read the inputs and write the results across the link, with no
// staging copies.  Measured on the 2^26-slot bench step: finds 2.20 ms
// direct against 3.06 staged (2.17 from device memory), mixed 1.22 against
// 1.83, insert 4.08 against 4.60.  Pageable arrays, and every array on other
// GPUs, take the staged path; HIVE_HOSTIO_STAGED=1 in the environment
// forces it.
//
// query_coherent: *yes = whether the current device has that access (cached
// per device); returns the CUDA error of the query, if any.
cudaError_t query_coherent(int* yes) {
  static std::atomic<int> cached[64];  // 0 unknown, 1 yes, 2 no (zero-initialised)
  *yes = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int c = cached[dev].load(std::memory_order_relaxed);
  if (!c) {
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    c = v ? 1 : 2;
    cached[dev].store(c, std::memory_order_relaxed);
  }
  *yes = c == 1;
  return cudaSuccess;
}

bool coherent_host_access() {
  int yes = 0;
  return query_coherent(&yes) == cudaSuccess && yes;
}

// The address a kernel uses for p, when p is device-reachable without a
// copy: pinned or registered host memory, device or managed memory.
bool device_view(const void* p, const void** out) {
  *out = nullptr;
  if (!p) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *out = a.devicePointer;
    return true;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    *out = p;
    return true;
  }
  return false;
}

bool staged_forced() {
  const char* e = std::getenv("HIVE_HOSTIO_STAGED");
  return e && e[0] && std::strcmp(e, "0") != 0;
}

hive_status run_host(hive_table* t, Kind kind, const uint8_t* h_ops, const uint32_t* h_keys,
                     const uint32_t* h_vals, uint64_t n, uint32_t* h_out, uint8_t* h_st,
                     cudaStream_t s) {
  if (!t) return hfail(HIVE_ERR_INVALID_ARG, "table is NULL");
  if (n >= (1ull << 32)) return hfail(HIVE_ERR_INVALID_ARG, "n must be below 2^32 per call");
  if (n == 0) return HIVE_OK;
  if (!h_keys || (kind == kIns && !h_vals) || (kind == kFind && !h_out) || (kind == kExec && !h_ops))
    return hfail(HIVE_ERR_INVALID_ARG, "a required host array is NULL");
  hive_status st = HIVE_OK;
  if (t->check_contract && kind != kFind) {
    // the chunks are checked one by one as well; this catches a key repeated
    // across chunks
    uint64_t bad = 0;
    st = hive_check_batch(kind == kExec ? h_ops : nullptr, HIVE_OP_INSERT, h_keys, n,
                          kReservedKeyMin, &bad);
    if (st != HIVE_OK) return st;
  }
  if (!staged_forced() && coherent_host_access()) {
    const void *ops = nullptr, *keys = nullptr, *vals = nullptr, *out = nullptr, *sts = nullptr;
    if (device_view(h_ops, &ops) && device_view(h_keys, &keys) && device_view(h_vals, &vals) &&
        device_view(h_out, &out) && device_view(h_st, &sts)) {
      const uint32_t* k = static_cast<const uint32_t*>(keys);
      const uint32_t* v = static_cast<const uint32_t*>(vals);
      uint32_t* o = static_cast<uint32_t*>(const_cast<void*>(out));
      uint8_t* r = static_cast<uint8_t*>(const_cast<void*>(sts));
      if (kind == kIns)
        st = hive_insert(t, k, v, n, r, s);
      else if (kind == kFind)
        st = hive_find(t, k, n, o, r, s);
      else
        st = hive_execute(t, static_cast<const uint8_t*>(ops), k, v, n, o, r, s);
      // the call returns with every result in host memory, as the staged path does
      cudaError_t e = cudaStreamSynchronize(s);
      if (st == HIVE_OK && e != cudaSuccess) return hcuda(e, "cudaStreamSynchronize");
      return st;
    }
  }
  if ((st = ensure_staging(t)) != HIVE_OK) return st;
  st = run_chunks(t, kind, h_ops, h_keys, h_vals, n, h_out, h_st, s);
  if (st != HIVE_OK) {
    // an error part-way leaves copies of earlier chunks queued: finish them
    // before returning, so that no copy touches the caller's host arrays
    // after the call (the error text already set is kept)
    cudaStreamSynchronize(t->io.up);
    cudaStreamSynchronize(t->io.down);
    cudaGetLastError();
  }
  return st;
}

}  // namespace

void hive::free_staging(hive_table* t) {
  HostIO& io = t->io;
  for (int k = 0; k < 2; ++k) {
    cudaFree(io.ops[k]);
    cudaFree(io.keys[k]);
    cudaFree(io.vals[k]);
    cudaFree(io.out[k]);
    cudaFree(io.st[k]);
    if (io.in_ready[k]) cudaEventDestroy(io.in_ready[k]);
    if (io.done[k]) cudaEventDestroy(io.done[k]);
    if (io.free[k]) cudaEventDestroy(io.free[k]);
  }
  if (io.up) cudaStreamDestroy(io.up);
  if (io.down) cudaStreamDestroy(io.down);
  io = HostIO{};
}

extern "C" {

hive_status hive_insert_host(hive_table* t, const uint32_t* h_keys, const uint32_t* h_vals,
                             uint64_t n, uint8_t* h_status, void* stream) {
  return run_host(t, kIns, nullptr, h_keys, h_vals, n, nullptr, h_status,
                  static_cast<cudaStream_t>(stream));
}

hive_status hive_find_host(hive_table* t, const uint32_t* h_keys, uint64_t n,
                           uint32_t* h_vals_out, uint8_t* h_found, void* stream) {
  return run_host(t, kFind, nullptr, h_keys, nullptr, n, h_vals_out, h_found,
                  static_cast<cudaStream_t>(stream));
}

hive_status hive_execute_host(hive_table* t, const uint8_t* h_ops, const uint32_t* h_keys,
                              const uint32_t* h_vals, uint64_t n, uint32_t* h_vals_out,
                              uint8_t* h_status, void* stream) {
  return run_host(t, kExec, h_ops, h_keys, h_vals, n, h_vals_out, h_status,
                  static_cast<cudaStream_t>(stream));
}

hive_status hive_host_direct_access(int* out) {
  if (!out) return hfail(HIVE_ERR_INVALID_ARG, "hive_host_direct_access: out is NULL");
  int yes = 0;
  cudaError_t e = query_coherent(&yes);
  if (e != cudaSuccess) return hcuda(e, "querying host access of the device");
  *out = yes;
  return HIVE_OK;
}

}  // extern "C"
