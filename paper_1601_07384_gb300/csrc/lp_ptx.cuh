// PTX helpers shared by the low-precision operator kernels: shared-memory addresses, mbarriers,
// 1-D TMA bulk copies, cp.async, and the split of a binary64 into a pair of binary32.
#pragma once
#include <cstdint>

namespace stdg {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// try_wait with a suspend-time hint: the waiting thread is descheduled until the phase completes
// or the hint (ns) expires, so waiting warps do not take issue slots from working ones
__device__ __forceinline__ bool mbar_wait_hint(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// start moving `bytes` (a multiple of 16, 16-byte aligned source) from global memory into L2
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// split a binary64 into hi (truncated to 24 significant bits) + lo (next bits, rounded to 24),
// with integer operations only (no binary64 instruction per element)
__device__ __forceinline__ float2 df_split(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(u >> 63) << 31;
  const int e = (int)((u >> 52) & 0x7FF);
  const int E = e - 1023;
  if (e == 0 || E < -126) return make_float2(0.0f, 0.0f);                 // below binary32's normal range
  if (E > 127) return make_float2(__int_as_float(sign | 0x7F800000u), 0.0f);  // beyond binary32
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  const float hi = __int_as_float((int)(sign | ((unsigned int)(E + 127) << 23) | (unsigned int)(m >> 29)));
  const unsigned int rem = (unsigned int)(m & 0x1FFFFFFFull);                // 29 low fraction bits
  float lo = 0.0f;
  if (rem) {
    const unsigned int fb = __float_as_uint((float)rem);                      // rem * 2^(E-52):
    const int be = (int)((fb >> 23) & 0xFF) - (52 - E);                       // rescale the exponent
    if (be > 0) lo = __uint_as_float(sign | ((unsigned int)be << 23) | (fb & 0x7FFFFFu));
  }
  return make_float2(hi, lo);
}

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// packed binary32 subtraction (sub.rn.f32x2, sm_100 and later)
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// error-free difference on both halves of two float2 values: s + e = a - b exactly
// (the sum above with b negated, the negation folded into the operations)
__device__ __forceinline__ void df_two_diff2(float2 a, float2 b, float2& s, float2& e) {
  s = f2_sub(a, b);
  const float2 bb = f2_sub(s, a);                 // -b as far as s carries it
  e = f2_sub(f2_sub(a, f2_sub(s, bb)), __fadd2_rn(b, bb));
}

}  // namespace stdg
