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

cudaError_t grow_commit(GrowArray* a, size_t bytes, cudaStream_t s) {
  const DriverVmm& d = vmm();
  const size_t want = std::min(a->reserved, (bytes + a->gran - 1) / a->gran * a->gran);
  const CUmemAllocationProp p = prop_for(a->device);
  CUmemAccessDesc acc{};
  acc.location = p.location;
  acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  while (a->committed < want) {
    CUmemGenericAllocationHandle h = 0;
    if (d.create(&h, a->gran, &p, 0) != CUDA_SUCCESS) return cudaErrorMemoryAllocation;
    const CUdeviceptr at = a->base + a->committed;
    if (d.map(at, a->gran, 0, h, 0) != CUDA_SUCCESS) {
      d.release(h);
      return cudaErrorMemoryAllocation;
    }
    if (d.set_access(at, a->gran, &acc, 1) != CUDA_SUCCESS) {
      d.unmap(at, a->gran);
      d.release(h);
      return cudaErrorMemoryAllocation;
    }
    a->handles.push_back(h);
    // new buckets start empty (all-ones words)
    cudaError_t e = cudaMemsetAsync(reinterpret_cast<void*>(at), 0xFF, a->gran, s);
    if (e != cudaSuccess) return e;
    a->committed += a->gran;
  }
  return cudaSuccess;
}

void grow_decommit(GrowArray* a, size_t bytes) {
  const DriverVmm& d = vmm();
  const size_t keep = (bytes + a->gran - 1) / a->gran * a->gran;
  while (a->committed > keep && !a->handles.empty()) {
    a->committed -= a->gran;
    d.unmap(a->base + a->committed, a->gran);
    d.release(a->handles.back());
    a->handles.pop_back();
  }
}

void grow_free(GrowArray* a) {
  if (!a->base) return;
  grow_decommit(a, 0);
  vmm().free_va(a->base, a->reserved);
  *a = GrowArray{};
}

}  // namespace hive
