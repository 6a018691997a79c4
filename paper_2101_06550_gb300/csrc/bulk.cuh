// Bulk asynchronous global->shared copies completed on an mbarrier (the TMA
// copy engine's non-tensor form, sm_90 and later), with a bounded wait.
//
// A tile of `rows` rows, each `row_bytes` contiguous bytes at `src + r * src_pitch`,
// lands at `dst + r * row_bytes`.  One thread issues every copy; all threads of
// the CTA then wait on the barrier.  Addresses and sizes must be multiples of
// 16 bytes (checked by the host before choosing the staged kernels).
#pragma once

#include <stdint.h>

#include "chx_internal.cuh"

namespace chx {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
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

// Waits for phase `parity` of the barrier.  Gives up after `limit` polls
// (each try_wait itself suspends for a hardware-defined time), records
// CHX_ETIMEOUT in *status and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status, int limit = 1 << 22) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  set_status(status, CHX_ETIMEOUT);
  return false;
}

// Issues the tile copy (call from one thread after mbar_init + __syncthreads).
__device__ __forceinline__ void bulk_tile_load(void* dst, const char* src, size_t src_pitch, uint32_t row_bytes,
                                               int rows, uint64_t* bar) {
  mbar_expect_tx(bar, row_bytes * (uint32_t)rows);
  for (int r = 0; r < rows; ++r) bulk_g2s((char*)dst + (size_t)r * row_bytes, src + (size_t)r * src_pitch, row_bytes, bar);
}

}  // namespace chx
