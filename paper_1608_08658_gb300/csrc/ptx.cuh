// Inline-PTX helpers for sm_103a: shared-memory mbarriers, TMA tile loads,
// the global timer used to bound every wait.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace wave {
namespace dev {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Ends an mbarrier object so that its word can be initialised again (a CTA
// that runs the step body over several column segments).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
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

// Wait for the phase of `bar` with the given parity to complete.  Gives up
// (returns false) when `abort_flag` becomes non-zero or after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                  unsigned long long limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (mbar_test(bar, parity)) return true;
    if (abort_flag != nullptr && *abort_flag) return false;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Sponge term of one axis: eta_max/nbl^2 * delta^2, delta = points into the layer.
// The damping arithmetic (this product, the sum over axes and k = eta cm/(2dt))
// uses explicitly rounded operations, so no kernel fuses it into an FMA
// differently from another: every kernel that takes a step (single step,
// batched step, two-level pass) produces the same bits.
__device__ __forceinline__ float sponge_term(int i, int n, int nbl, float em_over_nbl2) {
  const int d = max(max(nbl - i, i - (n - 1 - nbl)), 0);
  return __fmul_rn(em_over_nbl2, static_cast<float>(d * d));
}

// Sum of the sponge terms of two or three axes, in a fixed order.
__device__ __forceinline__ float sponge_sum(float a, float b) { return __fadd_rn(a, b); }

// Power-of-two slab scale s with amax/s in [2^14, 2^15), built from the
// exponent field of amax (no rounding involved); 1 for an all-zero slab.
__device__ __forceinline__ float slab_scale(float amax) {
  if (!(amax > 0.f)) return 1.f;
  int e = static_cast<int>((__float_as_uint(amax) >> 23) & 0xffu);
  int se = e - 14;
  se = se < 1 ? 1 : (se > 253 ? 253 : se);
  return __uint_as_float(static_cast<unsigned>(se) << 23);
}

__device__ __forceinline__ float slab_inv_scale(float s) {
  const int se = static_cast<int>((__float_as_uint(s) >> 23) & 0xffu);
  return __uint_as_float(static_cast<unsigned>(254 - se) << 23);
}

}  // namespace dev
}  // namespace wave
