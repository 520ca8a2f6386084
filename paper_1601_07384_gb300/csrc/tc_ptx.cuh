// Inline-PTX wrappers for the 5th-generation tensor cores of sm_103a (tcgen05): tensor-memory
// allocation, the single-thread MMA with shared-memory operand descriptors, completion through an
// mbarrier, and the warp loads of the accumulator from tensor memory.
#pragma once
#include <cstdint>

#include "lp_ptx.cuh"

namespace stdg {

// Shared-memory matrix descriptor, K-major operand without swizzling: the tile is a grid of core
// matrices of 8 rows x 16 bytes (128 contiguous bytes each); lbo = byte distance between core matrices
// adjacent along K, sbo = byte distance between core matrices adjacent along M (or N).
//   bits  0-13: start address >> 4      bits 16-29: lbo >> 4      bits 32-45: sbo >> 4
//   bits 46-47: descriptor version (1)   bits 49-51: base offset (0)   bits 61-63: swizzle (0: none)
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16 with bfloat16 A and B, binary32 accumulator, both operands
// K-major, M x N tile:  bits 4-5: D format (1 = f32), 7-9: A format (1 = bf16), 10-12: B format,
// 15/16: A/B major (0 = K), 17-22: N >> 3, 24-28: M >> 4.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// allocate ncols (a power of two >= 32) tensor-memory columns; the base address is written to *slot
// (whole warp, converged)
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D (tensor memory) = A B^T (accumulate == 0) or D += A B^T, one thread
__device__ __forceinline__ void tc_mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// the mbarrier gets one arrival once every earlier MMA of this thread has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 8 consecutive binary32 columns of the calling thread's tensor-memory lane (warp w reads lanes
// 32w .. 32w + 31; taddr carries the lane in bits 16-31 and the column in bits 0-15)
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace stdg
