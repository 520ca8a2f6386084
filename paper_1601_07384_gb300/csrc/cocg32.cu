// Binary32 vector kernels of the inner COCG solves of the mixed-precision viscous refinement.
//
// The decoupled viscous systems (block-diagonal time matrix R, blocks of size 1 or 2) couple time
// columns a and a + 1 only inside a 2 x 2 block, so the COCG multipliers M (alpha, beta in the real
// Ng x Ng form) and the cross products their scalars need are tridiagonal in the time index: three
// binary32 multiply-adds per entry instead of Ng binary64 ones.  The inner solve is asked for a
// residual reduction of 1e-5, well inside binary32 rounding; the binary64 outer refinement forms its
// residual with the binary64-accurate operator, so the rounding here changes the number of outer steps,
// not the accuracy of the result.  Partial sums are binary32 over a thread's few dozen rows and across
// the lanes of a warp, then binary64 across warps and blocks, in a fixed order (results repeat bit for
// bit).
#include "solver.h"

namespace stdg {
namespace {

constexpr int kC32Blocks = 1216;    // 8 x 152 SMs
constexpr int kC32Threads = 256;

// warp sum in binary32 (binary64 shuffle-adds would cost FP64-pipe time per thread on sm_103a)
__device__ __forceinline__ float c32_warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// out = float((I (x) M) in): converted to binary32 first, mixed in binary32
template <int NG>
__global__ void __launch_bounds__(kC32Threads) k_c32_mix_to32(int ne, int N, Mix32 M, const double* __restrict__ in,
                                                            float* __restrict__ out) {
  const int64_t total = (int64_t)ne * N;
  const int Nst = N * NG;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int64_t o = i * Nst + (e - i * N);
    float v[NG];
#pragma unroll
    for (int b = 0; b < NG; ++b) v[b] = (float)in[o + b * N];
#pragma unroll
    for (int a = 0; a < NG; ++a) {
      float t = 0.0f;
#pragma unroll
      for (int b = 0; b < NG; ++b) t = fmaf(M.v[a * NG + b], v[b], t);
      out[o + a * N] = t;
    }
  }
}

// x += (I (x) M) y: mixed in binary32, added in binary64
template <int NG>
__global__ void __launch_bounds__(kC32Threads) k_c32_mix_acc64(int ne, int N, Mix32 M, const float* __restrict__ y,
                                                             double* __restrict__ x) {
  const int64_t total = (int64_t)ne * N;
  const int Nst = N * NG;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int64_t o = i * Nst + (e - i * N);
    float v[NG];
#pragma unroll
    for (int b = 0; b < NG; ++b) v[b] = y[o + b * N];
#pragma unroll
    for (int a = 0; a < NG; ++a) {
      float t = 0.0f;
#pragma unroll
      for (int b = 0; b < NG; ++b) t = fmaf(M.v[a * NG + b], v[b], t);
      x[o + a * N] += (double)t;
    }
  }
}

// Cross products C[a][b] = Sum u[a][k] v[b][k] for |a - b| <= 1 (the others are written as 0):
// partials part[block * Ng^2 + a Ng + b]
template <int NG>
__global__ void __launch_bounds__(kC32Threads) k_c32_cross(int ne, int N, const float* __restrict__ u,
                                                         const float* __restrict__ v, double* __restrict__ part) {
  float cd[NG], cu[NG], cl[NG];                   // C[a][a], C[a][a+1], C[a+1][a]
#pragma unroll
  for (int a = 0; a < NG; ++a) cd[a] = cu[a] = cl[a] = 0.0f;
  const int64_t total = (int64_t)ne * N;
  const int Nst = N * NG;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int64_t o = i * Nst + (e - i * N);
    float uu[NG], vv[NG];
#pragma unroll
    for (int a = 0; a < NG; ++a) { uu[a] = u[o + a * N]; vv[a] = v[o + a * N]; }
#pragma unroll
    for (int a = 0; a < NG; ++a) {
      cd[a] = fmaf(uu[a], vv[a], cd[a]);
      if (a + 1 < NG) {
        cu[a] = fmaf(uu[a], vv[a + 1], cu[a]);
        cl[a] = fmaf(uu[a + 1], vv[a], cl[a]);
      }
    }
  }
  __shared__ double red[3 * NG][kC32Threads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NG; ++a) {                  // binary32 within the warp, binary64 across warps
    const float sd = c32_warp_sum_f(cd[a]);
    const float su = c32_warp_sum_f(cu[a]);
    const float sl = c32_warp_sum_f(cl[a]);
    if (lane == 0) { red[3 * a][w] = sd; red[3 * a + 1][w] = su; red[3 * a + 2][w] = sl; }
  }
  __syncthreads();
  if (threadIdx.x < NG * NG) {
    const int a = threadIdx.x / NG, b = threadIdx.x - a * NG;
    int src = -1;
    if (b == a) src = 3 * a;
    else if (b == a + 1) src = 3 * a + 1;
    else if (b == a - 1) src = 3 * b + 2;
    double t = 0.0;
    if (src >= 0)
      for (int k = 0; k < kC32Threads / 32; ++k) t += red[src][k];
    part[(size_t)blockIdx.x * NG * NG + threadIdx.x] = t;
  }
}

// the tridiagonal entries of M (binary64 on the device) as binary32: row a is
// md[a] v[a] + mu[a] v[a+1] + ml[a] v[a-1]
template <int NG>
__device__ __forceinline__ void c32_load_mix(const double* __restrict__ M, float* md, float* mu, float* ml) {
  if (threadIdx.x < NG) {
    const int a = threadIdx.x;
    md[a] = (float)M[a * NG + a];
    mu[a] = a + 1 < NG ? (float)M[a * NG + a + 1] : 0.0f;
    ml[a] = a > 0 ? (float)M[a * NG + a - 1] : 0.0f;
  }
  __syncthreads();
}

template <int NG>
__device__ __forceinline__ float c32_row(const float* md, const float* mu, const float* ml, const float (&v)[NG],
                                         int a) {
  float t = md[a] * v[a];
  if (a + 1 < NG) t = fmaf(mu[a], v[a + 1], t);
  if (a > 0) t = fmaf(ml[a], v[a - 1], t);
  return t;
}

// y += M p, r -= M q; with want, partials of ||(I (x) W) r||^2
template <int NG>
__global__ void __launch_bounds__(kC32Threads) k_c32_update(int ne, int N, const double* __restrict__ Mdev,
                                                          float* __restrict__ y, float* __restrict__ r,
                                                          const float* __restrict__ p, const float* __restrict__ q,
                                                          Mix32 W, double* __restrict__ part, int want) {
  __shared__ float md[NG], mu[NG], ml[NG];
  c32_load_mix<NG>(Mdev, md, mu, ml);
  const int64_t total = (int64_t)ne * N;
  const int Nst = N * NG;
  float acc = 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int64_t o = i * Nst + (e - i * N);
    float pp[NG], qq[NG], rn[NG];
#pragma unroll
    for (int a = 0; a < NG; ++a) { pp[a] = p[o + a * N]; qq[a] = q[o + a * N]; }
#pragma unroll
    for (int a = 0; a < NG; ++a) {
      y[o + a * N] += c32_row<NG>(md, mu, ml, pp, a);
      rn[a] = r[o + a * N] - c32_row<NG>(md, mu, ml, qq, a);
      r[o + a * N] = rn[a];
    }
    if (want) {
#pragma unroll
      for (int c = 0; c < NG; ++c) {
        float t = 0.0f;
#pragma unroll
        for (int a = 0; a < NG; ++a) t = fmaf(W.v[c * NG + a], rn[a], t);
        acc = fmaf(t, t, acc);
      }
    }
  }
  if (!want) return;                              // uniform over the grid
  __shared__ double red[kC32Threads / 32];
  const double s = (double)c32_warp_sum_f(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kC32Threads / 32; ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}

// p = z + M p
template <int NG>
__global__ void __launch_bounds__(kC32Threads) k_c32_dir(int ne, int N, const double* __restrict__ Mdev,
                                                       const float* __restrict__ z, float* __restrict__ p) {
  __shared__ float md[NG], mu[NG], ml[NG];
  c32_load_mix<NG>(Mdev, md, mu, ml);
  const int64_t total = (int64_t)ne * N;
  const int Nst = N * NG;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int64_t o = i * Nst + (e - i * N);
    float pp[NG];
#pragma unroll
    for (int a = 0; a < NG; ++a) pp[a] = p[o + a * N];
#pragma unroll
    for (int a = 0; a < NG; ++a) p[o + a * N] = z[o + a * N] + c32_row<NG>(md, mu, ml, pp, a);
  }
}

}  // namespace

#define STDG_C32_NG_SWITCH(NGV, CALL) \
  switch (NGV) {                      \
    case 1: { constexpr int G = 1; CALL; } break; \
    case 2: { constexpr int G = 2; CALL; } break; \
    case 3: { constexpr int G = 3; CALL; } break; \
    case 4: { constexpr int G = 4; CALL; } break; \
    default: { constexpr int G = 5; CALL; } break; \
  }

void c32_mix_to32(cudaStream_t st, int ne, int N, int Ng, const Mix32& M, const double* in, float* out) {
  STDG_C32_NG_SWITCH(Ng, (k_c32_mix_to32<G><<<kC32Blocks, kC32Threads, 0, st>>>(ne, N, M, in, out)));
}
void c32_mix_acc64(cudaStream_t st, int ne, int N, int Ng, const Mix32& M, const float* y, double* x) {
  STDG_C32_NG_SWITCH(Ng, (k_c32_mix_acc64<G><<<kC32Blocks, kC32Threads, 0, st>>>(ne, N, M, y, x)));
}
void c32_cross(cudaStream_t st, int ne, int N, int Ng, const float* u, const float* v, double* part) {
  STDG_C32_NG_SWITCH(Ng, (k_c32_cross<G><<<kC32Blocks, kC32Threads, 0, st>>>(ne, N, u, v, part)));
}
void c32_update(cudaStream_t st, int ne, int N, int Ng, const double* M, float* y, float* r, const float* p,
                const float* q, const Mix32& W, double* part, int want) {
  STDG_C32_NG_SWITCH(Ng, (k_c32_update<G><<<kC32Blocks, kC32Threads, 0, st>>>(ne, N, M, y, r, p, q, W, part, want)));
}
void c32_dir(cudaStream_t st, int ne, int N, int Ng, const double* M, const float* z, float* p) {
  STDG_C32_NG_SWITCH(Ng, (k_c32_dir<G><<<kC32Blocks, kC32Threads, 0, st>>>(ne, N, M, z, p)));
}

}  // namespace stdg
