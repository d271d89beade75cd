// Device helpers shared by the kernel files: per-op codes, the BitHash
// mixes and the linear-hashing address, relaxed/acquire memory access, and
// the bulk-copy (TMA) + mbarrier primitives used to stage bucket reads in
// shared memory.  Everything is inline and internal to each file.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hive {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Per-op status codes (same numbers as include/hive.h).
enum : uint8_t {
  ST_INSERTED = 0,
  ST_REPLACED = 1,
  ST_ERASED = 2,
  ST_NOT_FOUND = 3,
  ST_FOUND = 4,
  ST_FULL = 5,
  ST_RESERVED = 6
};
enum : uint32_t { OP_INSERT = 0, OP_FIND = 1, OP_ERASE = 2 };

// ----------------------------------------------------------------------------
// Hashing and addressing
// ----------------------------------------------------------------------------

// BitHash1 of Section III-C without the final reduction: Thomas Wang's
// 32-bit integer hash (the variant of his shift/xor/multiply avalanche that
// starts with (k << 15) - k - 1 and multiplies by 2057 = 1 + 2^3 + 2^11 near
// the end), a bijection of 32-bit words.
__device__ __forceinline__ uint32_t bithash1(uint32_t k) {
  uint32_t x = (k << 15) - k - 1u;
  x = x ^ (x >> 12);
  x = x + (x << 2);
  x = x ^ (x >> 4);
  x = x * 2057u;
  return x ^ (x >> 16);
}

// BitHash2 of Section III-C without the final reduction: Bob Jenkins'
// six-step 32-bit integer hash, alternating an add of a constant with a
// shift, then an xor with a constant with a shift; each add of a shifted
// copy is the multiplication by 1 + 2^s it equals.
__device__ __forceinline__ uint32_t bithash2(uint32_t k) {
  uint32_t x = k * 4097u + 0x7ED55D16u;
  x = x ^ (x >> 19) ^ 0xC761C23Cu;
  x = x * 33u + 0x165667B1u;
  x = (x + 0xD3A2646Cu) ^ (x << 9);
  x = x * 9u + 0xFD7046C5u;
  return x ^ (x >> 16) ^ 0xB55A4F09u;
}

// Linear-hashing address (Section IV-C): buckets below the split pointer have
// been split this round and use one more hash bit.
__device__ __forceinline__ uint32_t lh_bucket(uint32_t h, uint32_t M, uint32_t p) {
  const uint32_t b = h & M;
  return b < p ? (h & (2u * M + 1u)) : b;
}

// ----------------------------------------------------------------------------
// Memory access helpers
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t* p) {
  uint64_t r;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(r) : "l"(p) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t ld_relaxed32(const uint32_t* p) {
  uint32_t r;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
  return r;
}
__device__ __forceinline__ void st_relaxed64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long* ull(uint64_t* p) {
  return reinterpret_cast<unsigned long long*>(p);
}

// ---- TMA bulk copies (cp.async.bulk) into shared memory, mbarrier-tracked ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The same test without suspending the thread (a single poll).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// One bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void lds_frag(const uint64_t* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(smem_u32(p)));
}
// Ampere-style asynchronous 16-byte copy global -> shared through the
// load/store path, and its group commit / wait.  HIVE_CP_ASYNC_L1 selects
// the L1-caching form (.ca) over the L2-only form (.cg): with Zipf-skewed
// lookups the hot buckets are then served from L1 (measured: Zipf(0.99) finds
// 38.8 against 21.3 Gops/s, uniform finds 31.3 against 29.3).
#ifndef HIVE_CP_ASYNC_L1
#define HIVE_CP_ASYNC_L1 1
#endif
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  if (HIVE_CP_ASYNC_L1)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
// The L2-only form, for reads that must not be served from a stale L1 line
// (the single-kernel batch, where chains and erases change buckets
// concurrently).
__device__ __forceinline__ void cp_async16_cg(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
// Orders this thread's memory accesses before the fence ahead of those after
// it (acquire and release at GPU scope; no store-to-load ordering needed).
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}
// Asks L2 to fetch [p, p + bytes) from memory (bytes a multiple of 16, p
// 16-byte aligned); nothing waits for it.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Spreads a bulk L2 prefetch of [base, base + bytes) over the blocks of a
// grid, 64 KB per instruction, issued by one thread of each block.
__device__ __forceinline__ void prefetch_l2_grid(const void* base, uint64_t bytes) {
  if (threadIdx.x != 0) return;
  constexpr uint64_t kPiece = 64 * 1024;
  const char* b = static_cast<const char*>(base);
  bytes &= ~static_cast<uint64_t>(15);
  for (uint64_t off = static_cast<uint64_t>(blockIdx.x) * kPiece; off < bytes;
       off += static_cast<uint64_t>(gridDim.x) * kPiece) {
    const uint64_t len = bytes - off < kPiece ? bytes - off : kPiece;
    prefetch_l2_bulk(b + off, static_cast<uint32_t>(len));
  }
}
__device__ __forceinline__ uint32_t ld_acquire32(const uint32_t* p) {
  uint32_t r;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
  return r;
}

}  // namespace
}  // namespace hive
