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
#include <complex>
#include <vector>

#include <type_traits>

#include "lp_ptx.cuh"
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
// several tets per block pass, their rows and their U staged in shared memory (U with row pitch
// N + 1, so both the column reads of U^T r and the row reads of U y are free of bank conflicts).
// All arithmetic is binary32 (in binary64 the products and the divides of the small solves are
// FP64-pipe-bound on sm_103a); the result is a fixed linear map of r, as preconditioning requires.
// K may be any Ng x Ng matrix whose symmetric part is positive semidefinite (the time matrix, or
// its real block-diagonal form).
template <int NC, typename TI, typename TO>
__global__ void __launch_bounds__(256) k_visc_fd(int ne, int Nrt, int Ng, const float* __restrict__ U,
                                                 const float* __restrict__ lam, const double* __restrict__ detJ,
                                                 SmallK K, float c, const TI* __restrict__ r,
                                                 TO* __restrict__ z, int accum) {
  extern __shared__ float vs[];
  const int N = NC ? NC : Nrt;
  const int Nst = N * Ng, NU = N * (N + 1);
  const int TB = blockDim.x / N;
  const size_t NN = (size_t)N * N;
  float* us = vs + TB * Nst;               // TB x N x (N + 1)
  const int tl = threadIdx.x / N, k = threadIdx.x - tl * N;
  for (int i0 = blockIdx.x * TB; i0 < ne; i0 += gridDim.x * TB) {
    const int nt = min(TB, ne - i0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nt * Nst; idx += blockDim.x) vs[idx] = (float)r[(size_t)i0 * Nst + idx];
    for (int idx = threadIdx.x; idx < nt * (int)NN; idx += blockDim.x) {
      const int t = idx / (int)NN, e = idx - t * (int)NN, row = e / N;
      us[t * NU + row * (N + 1) + (e - row * N)] = U[(size_t)i0 * NN + idx];
    }
    __syncthreads();
    const int i = i0 + tl;
    const bool act = tl < nt;
    float y[kMaxNg] = {0, 0, 0, 0, 0};
    if (act) {
      // w[a] = Sum_l U[l][k] r[a][l]
      const float* Uc = us + tl * NU + k;
      const float* rr = vs + tl * Nst;
      float w[kMaxNg] = {0, 0, 0, 0, 0};
#pragma unroll 4
      for (int l = 0; l < N; ++l) {
        const float u = Uc[l * (N + 1)];
#pragma unroll
        for (int a = 0; a < kMaxNg; ++a)
          if (a < Ng) w[a] = fmaf(u, rr[a * N + l], w[a]);
      }
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
    if (act)
#pragma unroll
      for (int a = 0; a < kMaxNg; ++a)
        if (a < Ng) vs[tl * Nst + a * N + k] = y[a];
    __syncthreads();
    if (act) {
      // z[a][k] = Sum_l U[k][l] y[a][l]
      const float* Ur = us + tl * NU + k * (N + 1);
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
          z[o] = accum ? z[o] + (TO)zz[a] : (TO)zz[a];
        }
    }
  }
}

// The same with N and Ng at compile time (the solve's N, the time degree's Ng): the small solve is
// unrolled with constant indices and U is staged by a plain contiguous copy (the tets of a pass are
// consecutive), read by rows from its unpadded layout.
template <int N, int NG, typename TI, typename TO>
__global__ void __launch_bounds__(256) k_visc_fd_t(int ne, const float* __restrict__ U, const float* __restrict__ lam,
                                                   const double* __restrict__ detJ, SmallK K, float c,
                                                   const TI* __restrict__ r, TO* __restrict__ z, int accum) {
  constexpr int Nst = N * NG, NN = N * N, TB = 256 / N;
  __shared__ __align__(16) float vs[TB * Nst];
  __shared__ __align__(16) float us[TB * NN];      // read as float4 when NN % 4 == 0
  const int tl = threadIdx.x / N, k = threadIdx.x - tl * N;
  float Kc[NG][NG];
#pragma unroll
  for (int a = 0; a < NG; ++a)
#pragma unroll
    for (int b = 0; b < NG; ++b) Kc[a][b] = K.v[a * NG + b];
  for (int i0 = blockIdx.x * TB; i0 < ne; i0 += gridDim.x * TB) {
    const int nt = min(TB, ne - i0);
    __syncthreads();
    // the pass's U blocks (and binary32 rows) by cp.async: every thread issues all its copies before
    // waiting once (copies through registers, one load after another, left the kernel waiting on
    // memory latency: N^2 = 1225 at p = 4 is not a multiple of 4, so those went one word at a time)
    const float* Ug = U + (size_t)i0 * NN;
    if constexpr (NN % 4 == 0) {
      for (int idx = threadIdx.x; idx < nt * NN / 4; idx += blockDim.x) cp_async<16>(us + 4 * idx, Ug + 4 * idx);
    } else {
      for (int idx = threadIdx.x; idx < nt * NN; idx += blockDim.x) cp_async<4>(us + idx, Ug + idx);
    }
    if constexpr (std::is_same<TI, float>::value) {
      for (int idx = threadIdx.x; idx < nt * Nst; idx += blockDim.x) cp_async<4>(vs + idx, r + (size_t)i0 * Nst + idx);
    } else {
      for (int idx = threadIdx.x; idx < nt * Nst; idx += blockDim.x) vs[idx] = (float)r[(size_t)i0 * Nst + idx];
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int i = i0 + tl;
    const bool act = tl < nt;
    float y[NG];
    if (act) {
      const float* Uc = us + tl * NN + k;
      const float* rr = vs + tl * Nst;
      float w[NG];
#pragma unroll
      for (int a = 0; a < NG; ++a) w[a] = 0.0f;
#pragma unroll 5
      for (int l = 0; l < N; ++l) {
        const float u = Uc[l * N];
#pragma unroll
        for (int a = 0; a < NG; ++a) w[a] = fmaf(u, rr[a * N + l], w[a]);
      }
      const float d = (float)detJ[i], cl = c * lam[(size_t)i * N + k];
      float M[NG][NG];
#pragma unroll
      for (int a = 0; a < NG; ++a)
#pragma unroll
        for (int b = 0; b < NG; ++b) M[a][b] = d * Kc[a][b] + (a == b ? cl : 0.0f);
#pragma unroll
      for (int p = 0; p < NG; ++p) {
        const float ip = 1.0f / M[p][p];
#pragma unroll
        for (int a = p + 1; a < NG; ++a) {
          const float f = M[a][p] * ip;
#pragma unroll
          for (int b = p + 1; b < NG; ++b) M[a][b] -= f * M[p][b];
          w[a] -= f * w[p];
        }
      }
#pragma unroll
      for (int a = NG - 1; a >= 0; --a) {
        float v = w[a];
#pragma unroll
        for (int b = a + 1; b < NG; ++b) v -= M[a][b] * y[b];
        y[a] = v / M[a][a];
      }
    }
    __syncthreads();
    if (act)
#pragma unroll
      for (int a = 0; a < NG; ++a) vs[tl * Nst + a * N + k] = y[a];
    __syncthreads();
    if (act) {
      const float* Ur = us + tl * NN + k * N;
      const float* yy = vs + tl * Nst;
      float zz[NG];
#pragma unroll
      for (int a = 0; a < NG; ++a) zz[a] = 0.0f;
#pragma unroll 5
      for (int l = 0; l < N; ++l) {
        const float u = Ur[l];
#pragma unroll
        for (int a = 0; a < NG; ++a) zz[a] = fmaf(u, yy[a * N + l], zz[a]);
      }
#pragma unroll
      for (int a = 0; a < NG; ++a) {
        const size_t o = (size_t)i * Nst + a * N + k;
        z[o] = accum ? z[o] + (TO)zz[a] : (TO)zz[a];
      }
    }
  }
}

// Resident blocks of a kernel across the device (its grid-stride loop then splits the work evenly: a
// fixed 8 blocks per SM with 5 resident ran 1.6 waves, the last at 60 % occupancy).  Host-side query,
// no stream work (safe while a graph is being captured); cached per kernel.
template <typename K>
static int resident_grid(K kern, int threads, size_t smem) {
  static int cached = 0;
  if (cached) return cached;
  int dev = 0, nsm = 152, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess || per < 1) per = 1;
  cached = nsm * per;
  return cached;
}

template <int N, int NG, typename TI, typename TO>
static void launch_fd_ng(cudaStream_t st, int ne, const float* U, const float* lam, const double* detJ,
                         const SmallK& K, float c, const TI* r, TO* z, int accum) {
  const int blocks = resident_grid(k_visc_fd_t<N, NG, TI, TO>, 256, 0);
  k_visc_fd_t<N, NG, TI, TO><<<blocks, 256, 0, st>>>(ne, U, lam, detJ, K, c, r, z, accum);
}

template <int N, typename TI, typename TO>
static void launch_fd_t(int Ng, int, cudaStream_t st, int ne, const float* U, const float* lam,
                        const double* detJ, const SmallK& K, float c, const TI* r, TO* z, int accum) {
  switch (Ng) {
    case 1: launch_fd_ng<N, 1>(st, ne, U, lam, detJ, K, c, r, z, accum); break;
    case 2: launch_fd_ng<N, 2>(st, ne, U, lam, detJ, K, c, r, z, accum); break;
    case 3: launch_fd_ng<N, 3>(st, ne, U, lam, detJ, K, c, r, z, accum); break;
    case 4: launch_fd_ng<N, 4>(st, ne, U, lam, detJ, K, c, r, z, accum); break;
    default: launch_fd_ng<N, 5>(st, ne, U, lam, detJ, K, c, r, z, accum); break;
  }
}

}  // namespace

// Real block-diagonal form of the time matrix, K = W R W^-1: R has a 2 x 2 block [[a, b], [-b, a]]
// for every complex eigenvalue pair a +- ib (columns vr, vi of W: the real and imaginary parts of
// the eigenvector of a + ib) and a 1 x 1 block for every real eigenvalue.  pair[c] = 1 marks the
// first column of a 2 x 2 block.  Eigenvalues from the characteristic polynomial (Faddeev-LeVerrier
// coefficients, Durand-Kerner iteration), eigenvectors by complex elimination; the result is checked
// (||K W - W R||, cond(W) <= 1e6) and false is returned if it fails.  Ng <= 5.
bool time_blockdiag(const double* K, int Ng, double* W, double* Winv, double* R, int* pair) {
  using cd = std::complex<double>;
  const int n = Ng;
  // characteristic polynomial det(lambda I - K) = lambda^n + c[1] lambda^(n-1) + ... + c[n]
  std::vector<double> c(n + 1, 0.0), M(n * n, 0.0), KM(n * n);
  c[0] = 1.0;
  for (int k = 1; k <= n; ++k) {
    // M_k = K M_{k-1} + c_{k-1} I,  c_k = -tr(K M_k) / k
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = 0.0;
        for (int l = 0; l < n; ++l) v += K[i * n + l] * M[l * n + j];
        KM[i * n + j] = v;
      }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) M[i * n + j] = KM[i * n + j] + (i == j ? c[k - 1] : 0.0);
    double tr = 0.0;
    for (int i = 0; i < n; ++i)
      for (int l = 0; l < n; ++l) tr += K[i * n + l] * M[l * n + i];
    c[k] = -tr / k;
  }
  auto poly = [&](cd z) { cd v = 1.0; for (int k = 1; k <= n; ++k) v = v * z + c[k]; return v; };
  double rad = 1.0;
  for (int k = 1; k <= n; ++k) rad = std::max(rad, 1.0 + std::fabs(c[k]));
  std::vector<cd> z(n);
  for (int k = 0; k < n; ++k) z[k] = std::polar(0.5 * rad, 0.4 + 6.283185307179586 * k / n);
  for (int it = 0; it < 500; ++it) {
    double moved = 0.0;
    for (int k = 0; k < n; ++k) {
      cd den = 1.0;
      for (int j = 0; j < n; ++j) if (j != k) den *= (z[k] - z[j]);
      if (std::abs(den) == 0.0) return false;
      const cd d = poly(z[k]) / den;
      z[k] -= d;
      moved = std::max(moved, std::abs(d) / std::max(1.0, std::abs(z[k])));
    }
    if (moved < 1e-15) break;
  }
  // pair up: real roots, then one representative (imaginary part > 0) per conjugate pair
  std::vector<cd> reps;
  std::vector<int> used(n, 0);
  const double tiny = 1e-9 * rad;
  for (int k = 0; k < n; ++k)
    if (std::fabs(z[k].imag()) <= tiny) reps.push_back(cd(z[k].real(), 0.0)), used[k] = 1;
  for (int k = 0; k < n; ++k)
    if (!used[k] && z[k].imag() > 0.0) reps.push_back(z[k]);
  int cols = 0;
  for (const cd& l : reps) cols += l.imag() == 0.0 ? 1 : 2;
  if (cols != n) return false;
  std::vector<double> Wm(n * n, 0.0), Rm(n * n, 0.0);
  int col = 0;
  for (const cd& l : reps) {
    // null vector of (K - l I): Gaussian elimination with full pivoting, last free variable = 1
    std::vector<cd> A(n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[i * n + j] = cd(K[i * n + j]) - (i == j ? l : cd(0.0));
    std::vector<int> perm(n);
    for (int j = 0; j < n; ++j) perm[j] = j;
    for (int k = 0; k < n - 1; ++k) {
      int pi = k, pj = k;
      for (int i = k; i < n; ++i)
        for (int j = k; j < n; ++j)
          if (std::abs(A[i * n + j]) > std::abs(A[pi * n + pj])) pi = i, pj = j;
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[pi * n + j]);
      for (int i = 0; i < n; ++i) std::swap(A[i * n + k], A[i * n + pj]);
      std::swap(perm[k], perm[pj]);
      if (std::abs(A[k * n + k]) == 0.0) return false;
      for (int i = k + 1; i < n; ++i) {
        const cd f = A[i * n + k] / A[k * n + k];
        for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      }
    }
    std::vector<cd> y(n);
    y[n - 1] = 1.0;
    for (int k = n - 2; k >= 0; --k) {
      cd v = 0.0;
      for (int j = k + 1; j < n; ++j) v -= A[k * n + j] * y[j];
      y[k] = v / A[k * n + k];
    }
    std::vector<cd> v(n);
    for (int j = 0; j < n; ++j) v[perm[j]] = y[j];
    double nrm = 0.0;
    for (const cd& e : v) nrm += std::norm(e);
    nrm = std::sqrt(nrm);
    for (cd& e : v) e /= nrm;
    if (l.imag() == 0.0) {
      for (int i = 0; i < n; ++i) Wm[i * n + col] = v[i].real();
      Rm[col * n + col] = l.real();
      pair[col] = 0;
      ++col;
    } else {
      for (int i = 0; i < n; ++i) { Wm[i * n + col] = v[i].real(); Wm[i * n + col + 1] = v[i].imag(); }
      Rm[col * n + col] = l.real();       Rm[col * n + col + 1] = l.imag();
      Rm[(col + 1) * n + col] = -l.imag(); Rm[(col + 1) * n + col + 1] = l.real();
      pair[col] = 1; pair[col + 1] = 0;
      col += 2;
    }
  }
  // W^-1 by Gauss-Jordan with partial pivoting
  std::vector<double> A(Wm), I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int pi = k;
    for (int i = k + 1; i < n; ++i) if (std::fabs(A[i * n + k]) > std::fabs(A[pi * n + k])) pi = i;
    if (std::fabs(A[pi * n + k]) < 1e-12) return false;
    for (int j = 0; j < n; ++j) { std::swap(A[k * n + j], A[pi * n + j]); std::swap(I[k * n + j], I[pi * n + j]); }
    const double d = A[k * n + k];
    for (int j = 0; j < n; ++j) { A[k * n + j] /= d; I[k * n + j] /= d; }
    for (int i = 0; i < n; ++i)
      if (i != k) {
        const double f = A[i * n + k];
        for (int j = 0; j < n; ++j) { A[i * n + j] -= f * A[k * n + j]; I[i * n + j] -= f * I[k * n + j]; }
      }
  }
  // check K W = W R
  double err = 0.0, ref = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double kw = 0.0, wr = 0.0;
      for (int l = 0; l < n; ++l) { kw += K[i * n + l] * Wm[l * n + j]; wr += Wm[i * n + l] * Rm[l * n + j]; }
      err = std::max(err, std::fabs(kw - wr));
      ref = std::max(ref, std::fabs(kw));
    }
  if (!(err <= 1e-10 * std::max(ref, 1.0))) return false;
  double nw = 0.0, ni = 0.0;                      // infinity-norm condition number of W
  for (int i = 0; i < n; ++i) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < n; ++j) { a += std::fabs(Wm[i * n + j]); b += std::fabs(I[i * n + j]); }
    nw = std::max(nw, a); ni = std::max(ni, b);
  }
  if (!(nw * ni <= 1e6)) return false;
  for (int q = 0; q < n * n; ++q) { W[q] = Wm[q]; Winv[q] = I[q]; R[q] = Rm[q]; }
  return true;
}

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

// z = D^-1 r (accum: z += D^-1 r) for the viscous operator with viscosity nu; with Kt, for the
// operator whose time matrix is Kt instead of K (the block-diagonal form of the decoupled solve).
template <typename TI, typename TO>
static stdg_status visc_pc_launch(stdg_solver* s, double nu, const TI* r, TO* z, int accum, const double* Kt) {
  SmallK K{};
  for (int c = 0; c < s->Ng * s->Ng; ++c) K.v[c] = (float)(Kt ? Kt[c] : s->K[c]);
  const int N = s->N, TB = 256 / N;
  const size_t smem = ((size_t)TB * N * s->Ng + (size_t)TB * N * (N + 1)) * sizeof(float);
  const float c = (float)(nu * s->dt);
  const int blocks = 1216;
  ++s->nlaunch;
  switch (N) {
    case 20: launch_fd_t<20>(s->Ng, blocks, s->stream, (int)s->ne, s->vpcU, s->vpcLam, s->dm.detJ, K, c, r, z, accum); break;
    case 35: launch_fd_t<35>(s->Ng, blocks, s->stream, (int)s->ne, s->vpcU, s->vpcLam, s->dm.detJ, K, c, r, z, accum); break;
    case 10: launch_fd_t<10>(s->Ng, blocks, s->stream, (int)s->ne, s->vpcU, s->vpcLam, s->dm.detJ, K, c, r, z, accum); break;
    default:
      k_visc_fd<0, TI, TO><<<blocks, 256, smem, s->stream>>>((int)s->ne, N, s->Ng, s->vpcU, s->vpcLam, s->dm.detJ, K, c, r, z,
                                                              accum);
      break;
  }
  STDG_LAUNCH_CHECK();
  return STDG_OK;
}

stdg_status visc_pc_apply(stdg_solver* s, double nu, const double* r, double* z, int accum, const double* Kt) {
  return visc_pc_launch(s, nu, r, z, accum, Kt);
}

// binary32 vectors in and out (the inner solves of the mixed-precision viscous refinement)
stdg_status visc_pc_apply32(stdg_solver* s, double nu, const float* r, float* z, const double* Kt) {
  return visc_pc_launch(s, nu, r, z, 0, Kt);
}

}  // namespace stdg

extern "C" stdg_status stdg_time_blockdiag(const double* K, int Ng, double* W, double* Winv, double* R, int* pair) {
  if (!K || !W || !Winv || !R || !pair || Ng < 1 || Ng > stdg::kMaxNg) {
    stdg::set_error("stdg_time_blockdiag: NULL argument or Ng outside 1..%d", stdg::kMaxNg);
    return STDG_EINVAL;
  }
  if (!stdg::time_blockdiag(K, Ng, W, Winv, R, pair)) {
    stdg::set_error("stdg_time_blockdiag: no well-conditioned real block-diagonal form");
    return STDG_EUNSUPPORTED;
  }
  return STDG_OK;
}
