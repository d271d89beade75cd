// Growable device arrays on CUDA virtual memory management.
//
// A resizable table reserves the virtual address range of its largest bucket
// array once and maps physical memory into it in granularity-sized chunks as
// linear hashing splits buckets, and unmaps chunks after merges have emptied
// them.  The committed HBM then follows the table's capacity instead of its
// maximum.  The driver calls are fetched through the runtime
// (cudaGetDriverEntryPointByVersion), so the library does not link libcuda.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "hive_internal.h"

namespace hive {
namespace {

struct DriverVmm {
  bool ok = false;
  CUresult (*reserve)(CUdeviceptr*, size_t, size_t, CUdeviceptr, unsigned long long) = nullptr;
  CUresult (*free_va)(CUdeviceptr, size_t) = nullptr;
  CUresult (*create)(CUmemGenericAllocationHandle*, size_t, const CUmemAllocationProp*,
                     unsigned long long) = nullptr;
  CUresult (*release)(CUmemGenericAllocationHandle) = nullptr;
  CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle,
                  unsigned long long) = nullptr;
  CUresult (*unmap)(CUdeviceptr, size_t) = nullptr;
  CUresult (*set_access)(CUdeviceptr, size_t, const CUmemAccessDesc*, size_t) = nullptr;
  CUresult (*granularity)(size_t*, const CUmemAllocationProp*,
                          CUmemAllocationGranularity_flags) = nullptr;
};

std::once_flag g_once;
DriverVmm g_vmm;

template <class F>
bool fetch(const char* name, F* out) {
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

const DriverVmm& vmm() {
  std::call_once(g_once, [] {
    DriverVmm d;
    d.ok = fetch("cuMemAddressReserve", &d.reserve) && fetch("cuMemAddressFree", &d.free_va) &&
           fetch("cuMemCreate", &d.create) && fetch("cuMemRelease", &d.release) &&
           fetch("cuMemMap", &d.map) && fetch("cuMemUnmap", &d.unmap) &&
           fetch("cuMemSetAccess", &d.set_access) &&
           fetch("cuMemGetAllocationGranularity", &d.granularity);
    g_vmm = d;
  });
  return g_vmm;
}

CUmemAllocationProp prop_for(int device) {
  CUmemAllocationProp p{};
  p.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  p.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  p.location.id = device;
  return p;
}

}  // namespace

cudaError_t grow_reserve(GrowArray* a, size_t max_bytes, int device) {
  const DriverVmm& d = vmm();
  if (!d.ok) return cudaErrorNotSupported;
  a->device = device;
  const CUmemAllocationProp p = prop_for(device);
  size_t g = 0;
  if (d.granularity(&g, &p, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || !g)
    return cudaErrorNotSupported;
  a->gran = g;
  a->reserved = (max_bytes + g - 1) / g * g;
  CUdeviceptr base = 0;
  if (d.reserve(&base, a->reserved, g, 0, 0) != CUDA_SUCCESS) return cudaErrorMemoryAllocation;
  a->base = base;
  a->committed = 0;
  return cudaSuccess;
}

// Maps at least `bytes` (rounded up to the granularity). Growth maps one
// physical allocation per call, at least as large as what is already mapped
// (the mapped size at least doubles), so that a table growing batch by batch
// makes a logarithmic number of driver calls.
cudaError_t grow_commit(GrowArray* a, size_t bytes, cudaStream_t s) {
  const DriverVmm& d = vmm();
  const size_t g = a->gran;
  const size_t want = std::min(a->reserved, (bytes + g - 1) / g * g);
  if (a->committed >= want) return cudaSuccess;
  size_t delta = want - a->committed;
  const size_t step = (a->committed + g - 1) / g * g;
  delta = std::min(a->reserved - a->committed, std::max(delta, step));
  const CUmemAllocationProp p = prop_for(a->device);
  CUmemAccessDesc acc{};
  acc.location = p.location;
  acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  CUmemGenericAllocationHandle h = 0;
  if (d.create(&h, delta, &p, 0) != CUDA_SUCCESS) return cudaErrorMemoryAllocation;
  const CUdeviceptr at = a->base + a->committed;
  if (d.map(at, delta, 0, h, 0) != CUDA_SUCCESS) {
    d.release(h);
    return cudaErrorMemoryAllocation;
  }
  if (d.set_access(at, delta, &acc, 1) != CUDA_SUCCESS) {
    d.unmap(at, delta);
    d.release(h);
    return cudaErrorMemoryAllocation;
  }
  a->handles.push_back(h);
  a->sizes.push_back(delta);
  a->committed += delta;
  // new buckets start empty (all-ones words)
  return cudaMemsetAsync(reinterpret_cast<void*>(at), 0xFF, delta, s);
}

// Unmaps whole allocations from the top while what stays mapped still
// covers `bytes`.
void grow_decommit(GrowArray* a, size_t bytes) {
  const DriverVmm& d = vmm();
  while (!a->handles.empty() && a->committed - a->sizes.back() >= bytes) {
    const size_t sz = a->sizes.back();
    a->committed -= sz;
    d.unmap(a->base + a->committed, sz);
    d.release(a->handles.back());
    a->handles.pop_back();
    a->sizes.pop_back();
  }
}

void grow_free(GrowArray* a) {
  if (!a->base) return;
  grow_decommit(a, 0);
  vmm().free_va(a->base, a->reserved);
  *a = GrowArray{};
}

}  // namespace hive
