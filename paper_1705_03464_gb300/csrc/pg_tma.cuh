// TMA (cp.async.bulk.tensor) and mbarrier helpers for sm_103a, written as
// inline PTX, plus host-side tensor-map encoding through the driver entry
// point. Every wait is bounded by %globaltimer; a kernel that gives up sets
// an error word the host turns into PG_ERR_TIMEOUT.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pg {
namespace tma {

// error codes written to the device error word
enum : int { kErrNone = 0, kErrTmaTimeout = 1 };

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised barriers and generic-proxy writes to shared memory
// visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Named barrier `id` (1..15) over the n threads (a multiple of 32) of the
// warps that reach it; bar_or also returns whether any of them passed pred != 0.
__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ int bar_or(int id, int n, int pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred), "r"(id), "r"(n)
      : "memory");
  return (int)r;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase `parity` of `bar` to complete, for at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// 4D tiled load global -> shared, completion counted on `bar`. The shared
// destination must be 128-byte aligned; a misaligned one is not issued, so
// the waiting side runs into its bounded wait and reports an error.
__device__ __forceinline__ void load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                        int c1, int c2, int c3) {
  if (smem_addr(dst) & 127u) return;
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_addr(bar))
      : "memory");
}

// 5D tiled load (same rules as load_4d), with an L2 cache policy.
__device__ __forceinline__ void load_5d_hint(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                             int c1, int c2, int c3, int c4, uint64_t policy) {
  if (smem_addr(dst) & 127u) return;
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// 5D tiled store shared -> global, completion tracked by the issuing
// thread's bulk async groups, with an L2 cache policy. The shared source must
// be 128-byte aligned (else nothing is stored) and written before the store
// by threads that then ran fence_async_shared; every coordinate is >= 0.
__device__ __forceinline__ void store_5d_hint(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                              int c3, int c4, uint64_t policy) {
  if (smem_addr(src) & 127u) return;
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group.L2::cache_hint"
      " [%0, {%1, %2, %3, %4, %5}], [%6], %7;" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(src)), "l"(policy)
      : "memory");
}
// Closes the bulk async group of the stores issued so far by this thread.
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until every committed bulk store of this thread has read its shared
// source (the buffer may then be overwritten).
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Waits until every committed bulk store of this thread is complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 5D tiled prefetch of a box from global memory into L2 (no shared memory,
// no completion to wait for): a later load of the same box finds it in L2.
__device__ __forceinline__ void prefetch_5d(const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4) {
  asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
               : "memory");
}

// L2 eviction policies for cache-hinted accesses (createpolicy): streamed
// data that is read or written once is marked evict-first, data that the
// same CTA re-reads soon is marked evict-last.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// load_4d with an L2 cache policy.
__device__ __forceinline__ void load_4d_hint(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                             int c1, int c2, int c3, uint64_t policy) {
  if (smem_addr(dst) & 127u) return;
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// Global loads and stores of one complex value with an L2 cache policy.
__device__ __forceinline__ float2 ld_hint(const float2* p, uint64_t policy) {
  float2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(p), "l"(policy));
  return v;
}
__device__ __forceinline__ double2 ld_hint(const double2* p, uint64_t policy) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(p), "l"(policy));
  return v;
}
__device__ __forceinline__ void st_hint(float2* p, float2 v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y),
               "l"(policy)
               : "memory");
}
__device__ __forceinline__ void st_hint(double2* p, double2 v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y),
               "l"(policy)
               : "memory");
}

// Asynchronous 8- or 16-byte copies global -> shared (cp.async), for row
// gathers that TMA boxes cannot express. Completion is per thread:
// cp_async_wait_all() waits for the calling thread's own copies, which are
// loads from valid addresses and always complete.
__device__ __forceinline__ void cp_async(float2* dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async(double2* dst, const double2* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace tma

// Host: a 4D tensor map over 8-byte elements, dims/strides innermost first
// (strides in bytes for dims 1..3), box {b0, b1, b2, b3}. Returns false if the
// driver rejects it.
bool encode_map_4d(CUtensorMap* map, const void* base, const uint64_t dims[4],
                   const uint64_t strides_bytes[3], const uint32_t box[4]);

// As encode_map_4d with five dimensions (strides for dims 1..4).
bool encode_map_5d(CUtensorMap* map, const void* base, const uint64_t dims[5],
                   const uint64_t strides_bytes[4], const uint32_t box[5]);

// Test of the bounded waits: one CTA waits on an mbarrier nothing completes
// for limit_ns and sets *err (device) to kErrTmaTimeout when it gives up.
cudaError_t launch_wait_selftest(uint64_t limit_ns, int* err, cudaStream_t s);

}  // namespace pg
