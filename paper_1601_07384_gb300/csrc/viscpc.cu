// Block-Jacobi preconditioner of the viscous systems (Eq. A1_mod) by fast diagonalisation.
//
// With the orthonormal bases the diagonal block of tet i of the viscous operator is
//     D_i = d_i K (x) I_N + c I_Ng (x) G_i,      d_i = |det J_i|, c = nu dt,
// acting on the time-major coefficients x[a N + k]: K (the time matrix of Eq. MD_2) on the time index,
// and G_i = Sum over the tet's faces of Q^T Q (the spatial diagonal block of the viscous five-point
// operator, symmetric positive definite) on the space index.  With G_i = U Lambda U^T,
//     D_i^-1 = (I (x) U) diag_k (d_i K + c lambda_k I)^-1 (I (x) U^T),
// so each tet stores U (N x N, binary32) and Lambda (N) instead of the Nst x Nst inverse, and the
// apply costs two N x N products per time column plus N solves of size Ng.  U is found once per
// solver by the cyclic Jacobi eigenvalue method (rotations annihilating one off-diagonal pair at a
// time, Golub & Van Loan Sec. 8.5), one warp per tet in shared memory.  c enters only the small
// solves, so a new viscosity needs no new setup.  d_i K + c lambda_k I has a positive definite
// symmetric part (K + K^T = gamma(1) gamma(1)^T + gamma(0) gamma(0)^T), so its LU factorisation
// needs no pivoting.
#include <algorithm>
#include <cmath>

#include "solver.h"

namespace stdg {

namespace {

constexpr int kEigWarps = 4;                 // tets per block of the eigensolver
constexpr int kEigSweeps = 16;               // cyclic sweeps (each annihilates every pair once)
constexpr int kEigLd = kMaxN + 1;

// G_i = Bvisc_i - B_i; eigenvectors (columns of U) and eigenvalues, one warp per tet.  Binary32: the
// preconditioner needs a fixed approximate inverse, and binary64 rotations on sm_103a's FP64 pipe
// made this setup ~200 ms at 10,368 tets, p = 4.
__global__ void __launch_bounds__(32 * kEigWarps) k_visc_eig(int ne, int N, const double* __restrict__ Bdiag,
                                                             const double* __restrict__ Bvisc, float* __restrict__ Uout,
                                                             float* __restrict__ lam) {
  extern __shared__ float sm[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* A = sm + (size_t)w * 2 * kMaxN * kEigLd;
  float* V = A + kMaxN * kEigLd;
  __shared__ float cs_s[kEigWarps][2];
  const size_t NN = (size_t)N * N;
  for (int i = blockIdx.x * kEigWarps + w; i < ne; i += gridDim.x * kEigWarps) {
    for (int e = lane; e < N * N; e += 32) {
      const int r = e / N, c = e - r * N;
      A[r * kEigLd + c] = (float)(Bvisc[(size_t)i * NN + e] - Bdiag[(size_t)i * NN + e]);
      V[r * kEigLd + c] = r == c ? 1.0f : 0.0f;
    }
    __syncwarp();
    // symmetrise (the assembled block is symmetric up to rounding)
    for (int e = lane; e < N * N; e += 32) {
      const int r = e / N, c = e - r * N;
      if (r < c) {
        const float m = 0.5f * (A[r * kEigLd + c] + A[c * kEigLd + r]);
        A[r * kEigLd + c] = m;
        A[c * kEigLd + r] = m;
      }
    }
    __syncwarp();
    for (int sweep = 0; sweep < kEigSweeps; ++sweep) {
      float off = 0.0f, dia = 0.0f;
      for (int e = lane; e < N * N; e += 32) {
        const int r = e / N, c = e - r * N;
        const float v = A[r * kEigLd + c];
        if (r != c) off += v * v; else dia += v * v;
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        dia += __shfl_xor_sync(0xffffffffu, dia, o);
      }
      if (off <= 1e-11f * dia) break;
      for (int p = 0; p < N - 1; ++p)
        for (int q = p + 1; q < N; ++q) {
          if (lane == 0) {
            const float apq = A[p * kEigLd + q];
            float c = 1.0f, s = 0.0f;
            // skip pairs already negligible against their diagonal entries
            if (fabsf(apq) > 1e-9f * (fabsf(A[p * kEigLd + p]) + fabsf(A[q * kEigLd + q]))) {
              const float tau = (A[q * kEigLd + q] - A[p * kEigLd + p]) / (2.0f * apq);
              const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
              c = 1.0f / sqrtf(1.0f + t * t);
              s = t * c;
            }
            cs_s[w][0] = c; cs_s[w][1] = s;
          }
          __syncwarp();
          const float c = cs_s[w][0], s = cs_s[w][1];
          if (s != 0.0f) {
            // A <- A J (columns p, q), V <- V J
            for (int k = lane; k < N; k += 32) {
              const float akp = A[k * kEigLd + p], akq = A[k * kEigLd + q];
              A[k * kEigLd + p] = c * akp - s * akq;
              A[k * kEigLd + q] = s * akp + c * akq;
              const float vkp = V[k * kEigLd + p], vkq = V[k * kEigLd + q];
              V[k * kEigLd + p] = c * vkp - s * vkq;
              V[k * kEigLd + q] = s * vkp + c * vkq;
            }
            __syncwarp();
            // A <- J^T A (rows p, q)
            for (int k = lane; k < N; k += 32) {
              const float apk = A[p * kEigLd + k], aqk = A[q * kEigLd + k];
              A[p * kEigLd + k] = c * apk - s * aqk;
              A[q * kEigLd + k] = s * apk + c * aqk;
            }
          }
          __syncwarp();
        }
    }
    for (int e = lane; e < N * N; e += 32) {
      const int r = e / N, c = e - r * N;
      Uout[(size_t)i * NN + e] = V[r * kEigLd + c];     // U[l][k]: row l, eigenvector k
    }
    for (int k = lane; k < N; k += 32) lam[(size_t)i * N + k] = fmaxf(A[k * kEigLd + k], 0.0f);
    __syncwarp();
  }
}

struct SmallK { float v[kMaxNg * kMaxNg]; };

// z_i = D_i^-1 r_i (accum: z_i += D_i^-1 r_i), thread per (tet, spatial index), all time columns;
// several tets per block pass with their rows staged in shared memory.  All arithmetic is binary32
// (in binary64 the products and the divides of the small solves are FP64-pipe-bound on sm_103a);
// the result is a fixed linear map of r, as right preconditioning requires.
template <int NC>
__global__ void __launch_bounds__(256) k_visc_fd(int ne, int Nrt, int Ng, const float* __restrict__ U,
                                                 const float* __restrict__ lam, const double* __restrict__ detJ,
                                                 SmallK K, float c, const double* __restrict__ r,
                                                 double* __restrict__ z, int accum) {
  extern __shared__ float vs[];
  const int N = NC ? NC : Nrt;
  const int Nst = N * Ng;
  const int TB = blockDim.x / N;
  const size_t NN = (size_t)N * N;
  const int tl = threadIdx.x / N, k = threadIdx.x - tl * N;
  for (int i0 = blockIdx.x * TB; i0 < ne; i0 += gridDim.x * TB) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < TB * Nst; idx += blockDim.x)
      vs[idx] = i0 + idx / Nst < ne ? (float)r[(size_t)i0 * Nst + idx] : 0.0f;
    __syncthreads();
    const int i = i0 + tl;
    float y[kMaxNg] = {0, 0, 0, 0, 0};
    if (tl < TB && i < ne) {
      // w[a] = Sum_l U[l][k] r[a][l]
      const float* Uc = U + (size_t)i * NN + k;
      const float* rr = vs + tl * Nst;
      float wf[kMaxNg] = {0, 0, 0, 0, 0};
#pragma unroll 4
      for (int l = 0; l < N; ++l) {
        const float u = Uc[(size_t)l * N];
#pragma unroll
        for (int a = 0; a < kMaxNg; ++a)
          if (a < Ng) wf[a] = fmaf(u, rr[a * N + l], wf[a]);
      }
      float* w = wf;
      // (d K + c lambda_k I) y = w, LU without pivoting
      const float d = (float)fabs(detJ[i]), cl = c * lam[(size_t)i * N + k];
      float M[kMaxNg][kMaxNg];
#pragma unroll
      for (int a = 0; a < kMaxNg; ++a)
#pragma unroll
        for (int b = 0; b < kMaxNg; ++b) M[a][b] = (a < Ng && b < Ng) ? d * K.v[a * Ng + b] + (a == b ? cl : 0.0f) : 0.0f;
#pragma unroll
      for (int p = 0; p < kMaxNg; ++p)
        if (p < Ng) {
          const float ip = 1.0f / M[p][p];
#pragma unroll
          for (int a = p + 1; a < kMaxNg; ++a)
            if (a < Ng) {
              const float f = M[a][p] * ip;
#pragma unroll
              for (int b = p + 1; b < kMaxNg; ++b)
                if (b < Ng) M[a][b] -= f * M[p][b];
              w[a] -= f * w[p];
            }
        }
#pragma unroll
      for (int a = kMaxNg - 1; a >= 0; --a)
        if (a < Ng) {
          float v = w[a];
#pragma unroll
          for (int b = a + 1; b < kMaxNg; ++b)
            if (b < Ng) v -= M[a][b] * y[b];
          y[a] = v / M[a][a];
        }
    }
    __syncthreads();
    if (tl < TB && i < ne)
#pragma unroll
      for (int a = 0; a < kMaxNg; ++a)
        if (a < Ng) vs[tl * Nst + a * N + k] = y[a];
    __syncthreads();
    if (tl < TB && i < ne) {
      // z[a][k] = Sum_l U[k][l] y[a][l]
      const float* Ur = U + (size_t)i * NN + (size_t)k * N;
      const float* yy = vs + tl * Nst;
      float zz[kMaxNg] = {0, 0, 0, 0, 0};
#pragma unroll 4
      for (int l = 0; l < N; ++l) {
        const float u = Ur[l];
#pragma unroll
        for (int a = 0; a < kMaxNg; ++a)
          if (a < Ng) zz[a] = fmaf(u, yy[a * N + l], zz[a]);
      }
#pragma unroll
      for (int a = 0; a < kMaxNg; ++a)
        if (a < Ng) {
          const size_t o = (size_t)i * Nst + a * N + k;
          z[o] = accum ? z[o] + (double)zz[a] : (double)zz[a];
        }
    }
  }
}

}  // namespace

stdg_status visc_pc_ensure(stdg_solver* s) {
  if (s->vpcU) return STDG_OK;
  const size_t NN = (size_t)s->N * s->N;
  stdg_status e = dev_alloc(s, (void**)&s->vpcU, (size_t)s->ne * NN * sizeof(float));
  if (e == STDG_OK) e = dev_alloc(s, (void**)&s->vpcLam, (size_t)s->ne * s->N * sizeof(float));
  if (e != STDG_OK) return e;
  const size_t smem = (size_t)kEigWarps * 2 * kMaxN * kEigLd * sizeof(float);
  STDG_CUDA(cudaFuncSetAttribute(k_visc_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int blocks = (int)std::min<int64_t>((s->ne + kEigWarps - 1) / kEigWarps, 152 * 16);
  ++s->nlaunch;
  k_visc_eig<<<blocks, 32 * kEigWarps, smem, s->stream>>>((int)s->ne, s->N, s->Bdiag, s->Bvisc, s->vpcU, s->vpcLam);
  STDG_LAUNCH_CHECK();
  return STDG_OK;
}

// z = D^-1 r (accum: z += D^-1 r) for the viscous operator with viscosity nu.
stdg_status visc_pc_apply(stdg_solver* s, double nu, const double* r, double* z, int accum) {
  SmallK K{};
  for (int c = 0; c < s->Ng * s->Ng; ++c) K.v[c] = (float)s->K[c];
  const int N = s->N, TB = 256 / N;
  const size_t smem = (size_t)TB * N * s->Ng * sizeof(float);
  const float c = (float)(nu * s->dt);
  const int blocks = 1216;
  ++s->nlaunch;
  switch (N) {
    case 20: k_visc_fd<20><<<blocks, 256, smem, s->stream>>>((int)s->ne, N, s->Ng, s->vpcU, s->vpcLam, s->dm.detJ, K, c, r, z, accum); break;
    case 35: k_visc_fd<35><<<blocks, 256, smem, s->stream>>>((int)s->ne, N, s->Ng, s->vpcU, s->vpcLam, s->dm.detJ, K, c, r, z, accum); break;
    case 10: k_visc_fd<10><<<blocks, 256, smem, s->stream>>>((int)s->ne, N, s->Ng, s->vpcU, s->vpcLam, s->dm.detJ, K, c, r, z, accum); break;
    default: k_visc_fd<0><<<blocks, 256, smem, s->stream>>>((int)s->ne, N, s->Ng, s->vpcU, s->vpcLam, s->dm.detJ, K, c, r, z, accum); break;
  }
  STDG_LAUNCH_CHECK();
  return STDG_OK;
}

}  // namespace stdg
