// Shared-memory barriers (mbarrier) and bulk asynchronous copies (cp.async.bulk), in inline
// PTX, for the kernels that stage data through the asynchronous proxy.
#pragma once

#include <cstdint>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// SM clocks a bounded device wait gives an awaited arrival before it gives up (~1 s)
#define TTS_WAIT_LIMIT 2000000000LL
// Bounded wait for the phase with the given parity: gives up after `limit` SM clocks.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, long long limit = TTS_WAIT_LIMIT) {
  const long long t0 = clock64();
  while (!mbar_try(a, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// bytes (a multiple of 16, both addresses 16-byte aligned) from global to this CTA's shared
// memory, completing on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
// orders this thread's generic-proxy shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
