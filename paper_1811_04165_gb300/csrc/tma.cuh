// Bulk asynchronous copies (TMA, untiled) and mbarrier helpers for sm_103a,
// written as inline PTX.  Every wait is bounded: a wait that runs out records
// an error code in the caller's status word instead of spinning forever.
#pragma once

#include <cstdint>

namespace sps {

// Status bits written by kernels into the plan's device status word.
enum : uint32_t { kStatusWaitTimeout = 1u, kStatusBounds = 2u };

// Bounds-checked build (compiled with -DSPS_BOUNDS_CHECK=1): the de-dispersion
// passes test every staged shared-memory read against the extent of its stage;
// a read that would leave the stage is not made (zeros are added instead) and
// sets kStatusBounds in the status word.  Off in the normal build.
#ifndef SPS_BOUNDS_CHECK
#define SPS_BOUNDS_CHECK 0
#endif
constexpr bool kBoundsCheck = SPS_BOUNDS_CHECK != 0;

// In the bounds-checked build: true when a read of a staged row at byte offset
// `off` stays within `limit` (the largest offset whose whole row fits the
// stage); otherwise records the violation and returns false.
__device__ __forceinline__ bool stage_read_ok(uint32_t off, int64_t limit, uint32_t* status) {
  if (!kBoundsCheck || (int64_t)off <= limit) return true;
  if (status) atomicOr(status, kStatusBounds);
  return false;
}

// About 2^22 polls of try_wait (each may suspend briefly): seconds, far longer
// than any copy this library issues takes.
constexpr uint32_t kMaxPolls = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy completing on `bar`.  dst, src 16-byte aligned;
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar` for at most `polls` polls; false (and the
// status bit set) when it runs out.
__device__ __forceinline__ bool mbar_wait_polls(uint64_t* bar, uint32_t parity, uint32_t* status, uint32_t polls) {
  for (uint32_t i = 0; i < polls; i++)
    if (mbar_try_wait(bar, parity)) return true;
  if (status) atomicOr(status, kStatusWaitTimeout);
  return false;
}

// Bounded wait for phase `parity` of `bar`; false (and the status bit set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* status) {
  return mbar_wait_polls(bar, parity, status, kMaxPolls);
}

}  // namespace sps
