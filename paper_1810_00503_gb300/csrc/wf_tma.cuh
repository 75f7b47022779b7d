// Tensor-memory-accelerator (TMA) copies and mbarriers for the persistent
// FFT-stage kernels.  One thread issues a tile's 2-D copies; the block waits
// on the mbarrier's transaction count.  Every wait is bounded by a limit in SM
// clock cycles (wf_opts.spin_limit, by default WF_WAIT_CYCLES_DEFAULT, about
// 2 s at the maximum clock): a wait that gives up reports it to the caller.
#pragma once
#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched at run time)
#include <stdint.h>

__device__ __forceinline__ uint32_t wf_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void wf_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(wf_smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void wf_mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void wf_mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(wf_smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool wf_mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(wf_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity`; false if it did not complete within
// `limit` SM clock cycles.
__device__ __forceinline__ bool wf_mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  if (wf_mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!wf_mbar_try(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// 2-D tiled copy global -> shared of one box at element coordinates (x, y);
// x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void wf_tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          wf_smem_u32(dst)),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(wf_smem_u32(bar))
      : "memory");
}

