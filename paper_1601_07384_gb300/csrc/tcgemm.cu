// Dense products of the learned preconditioner's layers on the tensor cores (tcgen05, kind::f16):
//   D(m, n) = Sum_k A(m, k) B(n, k)   with A, B rounded to bfloat16, accumulated in binary32
// followed by the layer epilogue (bias, accumulate into D, ReLU with the pre-activation kept).  One CTA
// (4 warps) owns a tile of 128 rows of D and all N <= 256 columns; its accumulator lives in tensor
// memory (128 lanes x N columns).  The operands are read with arbitrary element strides, converted to
// bfloat16 and written into shared memory in the K-major core-matrix layout (8 rows x 16 bytes per
// core matrix); one thread issues the MMAs (M = 128, K = 16 each) for every 64-wide slice of K and
// commits them to an mbarrier; after the last slice every warp reads its 32 lanes of the accumulator.
// A second grid dimension splits K into ranges written to separate output slices (weight gradients:
// partial sums over chunks of tets, reduced afterwards in a fixed order).
#include <cuda_bf16.h>

#include "solver.h"
#include "tc_ptx.cuh"

namespace stdg {


constexpr int kTcRows = 128;                 // M of one MMA and of the CTA tile
constexpr int kTcKC = 64;                    // K slice staged at a time (4 MMAs of K = 16)
constexpr long kTcSpin = 4000;               // bounded waits (each try suspends up to 1 ms)

// byte offset of element (r, k) of a K-major tile with kTcKC columns: core matrix (r / 8, k / 8) at
// ((r / 8) (kTcKC / 8) + k / 8) 128, row r % 8 at 16 (r % 8), element k % 8 at 2 (k % 8)
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)((((r >> 3) * (kTcKC / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__global__ void __launch_bounds__(128, 1) k_tc_gemm(TcGemmArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const int Np = (a.N + 15) & ~15;           // the MMA's N: a multiple of 16 for M = 128
  unsigned char* As = tsm;                   // 128 x 64 bfloat16 = 16 KB
  unsigned char* Bs = tsm + kTcRows * kTcKC * 2;   // Np x 64 bfloat16
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)Np * kTcKC * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcRows;
  const int kbeg = blockIdx.y * a.ksplit, kend = min(a.K, kbeg + a.ksplit);
  uint32_t ncols = 32;
  while ((int)ncols < Np) ncols <<= 1;
  if (warp == 0) tc_alloc(tslot, ncols);
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc_idesc_bf16(kTcRows, Np);
  const __nv_bfloat16* Bh = static_cast<const __nv_bfloat16*>(a.B);
  const float* Bf = static_cast<const float*>(a.B);
  bool bad = false;
  uint32_t phase = 0;
  for (int k0 = kbeg; k0 < kend && !bad; k0 += kTcKC) {
    // stage the slices of A and B (zero outside the matrices and past kend)
    for (int e = tid; e < kTcRows * kTcKC; e += blockDim.x) {
      const int r = e / kTcKC, kk = e % kTcKC;
      const int m = m0 + r, k = k0 + kk;
      const float v = (m < a.M && k < kend) ? a.A[m * a.sAm + k * a.sAk] : 0.0f;
      *reinterpret_cast<__nv_bfloat16*>(As + tc_off(r, kk)) = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < Np * kTcKC; e += blockDim.x) {
      const int r = e / kTcKC, kk = e % kTcKC, k = k0 + kk;
      float v = 0.0f;
      if (r < a.N && k < kend) {
        if (a.b_ones_last && r == a.N - 1) v = 1.0f;
        else v = a.b_bf16 ? __bfloat162float(Bh[r * a.sBn + k * a.sBk]) : Bf[r * a.sBn + k * a.sBk];
      }
      *reinterpret_cast<__nv_bfloat16*>(Bs + tc_off(r, kk)) = __float2bfloat16_rn(v);
    }
    fence_async_smem();                      // generic stores -> the tensor cores' (async) reads
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < kTcKC / 16; ++ks) {
        // K = 16 per MMA: two core matrices along K (lbo 128 bytes), 8-row groups 1024 bytes apart
        const uint64_t ad = tc_smem_desc(smem_u32(As) + ks * 256, 128, (kTcKC / 8) * 128);
        const uint64_t bd = tc_smem_desc(smem_u32(Bs) + ks * 256, 128, (kTcKC / 8) * 128);
        tc_mma_bf16(tmem, ad, bd, idesc, (k0 > kbeg || ks > 0) ? 1u : 0u);
      }
      tc_commit(bar);
    }
    long spins = 0;                          // the MMAs have read the slices before they are rewritten
    while (!mbar_wait_hint(bar, phase))
      if (++spins > kTcSpin) { bad = true; break; }
    phase ^= 1u;
    bad = __syncthreads_or(bad) != 0;
  }
  tc_fence_after();
  if (bad) {
    if (tid == 0) atomicExch(a.err, 1);
  } else {
    const bool any = kbeg < kend;            // no K range: the product is 0
    const int row = m0 + warp * 32 + lane;
    float* Dz = a.D + (int64_t)blockIdx.y * a.dsplit;
    for (int c0 = 0; c0 < Np; c0 += 8) {
      float v[8];
      tc_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row >= a.M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = c0 + j;
        if (n >= a.N) break;
        float o = (any ? v[j] : 0.0f) + (a.bias ? a.bias[n] : 0.0f);
        const int64_t idx = (int64_t)row * a.ldd + n;
        if (a.accumulate) o += Dz[idx];
        if (a.relu) {
          if (a.pre) a.pre[idx] = o;
          o = fmaxf(o, 0.0f);
        }
        Dz[idx] = o;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, ncols);
}

// Launch: D (+)= A B^T over all of K (ksplit <= 0) or in K ranges of ksplit (grid.y ranges, outputs
// dsplit apart).  At most two CTAs per SM (shared memory), so that their tensor-memory allocations
// (<= 256 columns each) always fit in the SM's 512 columns.
cudaError_t launch_tc_gemm(TcGemmArgs a, cudaStream_t st) {
  if (a.N < 1 || a.N > 256 || a.M < 1) return cudaErrorInvalidValue;
  if (a.ksplit <= 0) a.ksplit = a.K > 0 ? a.K : 1;
  const int Np = (a.N + 15) & ~15;
  const size_t need = (size_t)kTcRows * kTcKC * 2 + (size_t)Np * kTcKC * 2 + 64;
  const size_t smem = need > 100 * 1024 ? need : 100 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nsplit = a.K > 0 ? (a.K + a.ksplit - 1) / a.ksplit : 1;
  dim3 grid((a.M + kTcRows - 1) / kTcRows, nsplit);
  k_tc_gemm<<<grid, 128, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace stdg

using namespace stdg;

// Test entry of the tensor-core product (binary32 A, B rounded to bfloat16, binary32 result):
// D[m * ldd + n] = Sum_k A[m * lda + k] B[n * ldb + k], 1 <= N <= 256.
extern "C" stdg_status stdg_tc_gemm_bf16(const float* A_dev, int64_t lda, const float* B_dev, int64_t ldb,
                                         float* D_dev, int64_t ldd, int M, int N, int K, void* stream) {
  if (!A_dev || !B_dev || !D_dev || M < 1 || N < 1 || N > 256 || K < 1) {
    set_error("stdg_tc_gemm_bf16: invalid argument (1 <= N <= 256)");
    return STDG_EINVAL;
  }
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { set_error("stdg_tc_gemm_bf16: cudaMalloc failed"); return STDG_ENOMEM; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(err, 0, sizeof(int), st);
  TcGemmArgs a{};
  a.M = M; a.N = N; a.K = K; a.ksplit = 0;
  a.A = A_dev; a.sAm = lda; a.sAk = 1;
  a.B = B_dev; a.sBn = ldb; a.sBk = 1; a.b_bf16 = 0;
  a.D = D_dev; a.ldd = ldd; a.dsplit = 0;
  a.err = err;
  cudaError_t e = launch_tc_gemm(a, st);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(err);
  if (e != cudaSuccess) { set_error("stdg_tc_gemm_bf16: %s", cudaGetErrorString(e)); return STDG_ECUDA; }
  if (herr) { set_error("stdg_tc_gemm_bf16: a bounded wait for the tensor cores gave up"); return STDG_ETIMEOUT; }
  return STDG_OK;
}
