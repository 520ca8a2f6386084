// The support steps of a Picard iteration at the benchmarked degrees (N, Ng compile-time), in
// binary64-accurate pair arithmetic on the binary32 pipe instead of binary64 multiply-adds:
//   averaging        out[c][i][a][k] = 1/|J_i| Sum_f Sum_l Mij[j][s][k][l] in[j][c][a][l]   (Eq. A3_mod)
//   face gradient    G[j][c][a][m]   = dt Sum_b Kinv[a][b] Sum_s Sum_l Q[j][s][c][m][l] p[s(j)][b][l]
//   velocity update  V[j][c][a][m]   = F[j][c][a][m] - dt Sum_b Kinv[a][b] Sum_s (Q dp) as above (Eq. A3_mod)
// Each binary64 matrix entry is loaded once, split into a (hi, lo) pair by integer operations and
// used for all the component and time-column sums of its row at once (3 Ng or Ng of them, two per
// packed binary32 operation); the vectors are split once into shared memory.  The binary64 kernels
// in step.cu / operators.cu take the same sums entry by entry on the binary64 pipe (1/64 of the
// binary32 rate on sm_103a): each entry there is reused 3 Ng times, so they are bound by that pipe, at
// about 20 times the time their bytes take.  A pair carries about 48 significant bits against
// binary64's 53, so results agree with the binary64 kernels to about 1e-14 relative.  The go back F
// and the pressure right-hand side b = D F stay binary64: b is a discrete divergence of a nearly
// solenoidal field, its cancellation amplifies that difference by orders of magnitude, and the
// pressure system amplifies it again (pair versions moved the p = 4 step from 2e-11 to 1.3e-10 of the
// oracle's pressure).
#include <cstdlib>
#include <cstring>

#include "pair.cuh"
#include "solver.h"

namespace stdg {
namespace {

constexpr int kSupThreads = 128;

// acc[r] += m v[r] for the R vectors v[r] = vrow[r * N] (pairs in shared memory), m a pair; packed
// over consecutive r
template <int N, int R>
__device__ __forceinline__ void sup_row(float2 m, const float2* vrow, float2 (&S)[(R + 1) / 2],
                                        float2 (&C)[(R + 1) / 2]) {
  const float2 mh2 = make_float2(m.x, m.x), nm2 = make_float2(-m.x, -m.x), ml2 = make_float2(m.y, m.y);
#pragma unroll
  for (int r2 = 0; r2 < (R + 1) / 2; ++r2) {
    const float2 v0 = vrow[(2 * r2) * N];
    const float2 v1 = 2 * r2 + 1 < R ? vrow[(2 * r2 + 1) * N] : make_float2(0.0f, 0.0f);
    pair_fma2(mh2, nm2, ml2, make_float2(v0.x, v1.x), make_float2(v0.y, v1.y), S[r2], C[r2]);
  }
}

template <int R>
__device__ __forceinline__ double sup_value(const float2 (&S)[(R + 1) / 2], const float2 (&C)[(R + 1) / 2], int r) {
  return (r & 1) ? pair_value(S[r >> 1].y, C[r >> 1].y) : pair_value(S[r >> 1].x, C[r >> 1].x);
}

template <int R>
__device__ __forceinline__ void sup_zero(float2 (&S)[(R + 1) / 2], float2 (&C)[(R + 1) / 2]) {
#pragma unroll
  for (int r2 = 0; r2 < (R + 1) / 2; ++r2) S[r2] = C[r2] = make_float2(0.0f, 0.0f);
}

// averaging: thread (tet, k), the 3 Ng sums of row k; the face's vectors staged per face
template <int N, int NG>
__global__ void __launch_bounds__(kSupThreads) k_average_p(int ne, const int* __restrict__ t2f,
                                                           const int* __restrict__ left,
                                                           const double* __restrict__ detJ,
                                                           const double* __restrict__ Mij,
                                                           const double* __restrict__ in, double* __restrict__ out) {
  constexpr int R = 3 * NG, Nst = N * NG, TB = kSupThreads / N;
  __shared__ float2 vs[TB][R * N];
  const int tl = threadIdx.x / N, k = threadIdx.x - tl * N;
  for (int i0 = blockIdx.x * TB; i0 < ne; i0 += gridDim.x * TB) {
    const int i = i0 + tl;
    const bool act = tl < TB && i < ne;
    float2 S[(R + 1) / 2], C[(R + 1) / 2];
    sup_zero<R>(S, C);
    for (int f = 0; f < 4; ++f) {
      __syncthreads();
      for (int idx = threadIdx.x; idx < TB * R * N; idx += kSupThreads) {
        const int t = idx / (R * N), rem = idx - t * R * N;
        if (i0 + t < ne) vs[t][rem] = df_split(in[(size_t)t2f[4 * (i0 + t) + f] * 3 * Nst + rem]);
      }
      __syncthreads();
      if (act) {
        const int j = t2f[4 * i + f], sd = left[j] == i ? 0 : 1;
        const double* M = Mij + (((size_t)j * 2 + sd) * N + k) * N;
#pragma unroll 5
        for (int l = 0; l < N; ++l) sup_row<N, R>(df_split(M[l]), &vs[tl][l], S, C);
      }
    }
    if (act) {
      const double inv = 1.0 / detJ[i];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r / NG, a = r - c * NG;
        out[((size_t)c * ne + i) * Nst + a * N + k] = sup_value<R>(S, C, r) * inv;
      }
    }
  }
}

struct SupK { float2 v[kMaxNg * kMaxNg]; };   // Kinv as pairs

// g[c][b] = Sum_s Sum_l Q[j][s][c][m][l] p[s(j)][b][l] for thread (face, m): 3 x Ng sums, packed over b
// (the same Q entry multiplies every b); interior faces both sides, boundary faces the single side's
// volume part (Q block 3 + c with the left tet)
template <int N, int NG>
__device__ __forceinline__ void sup_face_qp(int j, int m, bool interior, const double* __restrict__ Q,
                                            const float2 (*ps)[NG * N], float2 (&S)[3][(NG + 1) / 2],
                                            float2 (&C)[3][(NG + 1) / 2]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) sup_zero<NG>(S[c], C[c]);
  const int s0 = interior ? 0 : 1;
#pragma unroll 1
  for (int sd = s0; sd < 2; ++sd) {
    const float2* pv = ps[interior ? sd : 0];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double* q = Q + (((size_t)j * 6 + sd * 3 + c) * N + m) * N;
#pragma unroll 5
      for (int l = 0; l < N; ++l) sup_row<N, NG>(df_split(q[l]), pv + l, S[c], C[c]);
    }
  }
}

// the time mixing out[c][a] = Sum_b Kinv[a][b] g[c][b] of the pair sums above, as binary64 values
template <int NG>
__device__ __forceinline__ void sup_mix(const SupK& K, const float2 (&S)[3][(NG + 1) / 2],
                                        const float2 (&C)[3][(NG + 1) / 2], double (&o)[3][NG]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 gv[NG];
#pragma unroll
    for (int b = 0; b < NG; ++b)
      gv[b] = (b & 1) ? pair_norm(S[c][b >> 1].y, C[c][b >> 1].y) : pair_norm(S[c][b >> 1].x, C[c][b >> 1].x);
#pragma unroll
    for (int a = 0; a < NG; ++a) {
      float s = 0.0f, e = 0.0f;
#pragma unroll
      for (int b = 0; b < NG; ++b) pair_fma(K.v[a * NG + b], gv[b], s, e);
      o[c][a] = pair_value(s, e);
    }
  }
}

// face gradient: thread (face, m)
template <int N, int NG>
__global__ void __launch_bounds__(kSupThreads) k_face_grad_p(int nf, const int* __restrict__ left,
                                                             const int* __restrict__ right, const double* __restrict__ Q,
                                                             const double* __restrict__ Pp, double dt, SupK K,
                                                             double* __restrict__ G) {
  constexpr int Nst = N * NG, TB = kSupThreads / N;
  __shared__ float2 ps[TB][2][Nst];
  const int tl = threadIdx.x / N, m = threadIdx.x - tl * N;
  for (int j0 = blockIdx.x * TB; j0 < nf; j0 += gridDim.x * TB) {
    const int j = j0 + tl;
    const bool act = tl < TB && j < nf;
    __syncthreads();
    for (int idx = threadIdx.x; idx < TB * 2 * Nst; idx += kSupThreads) {
      const int t = idx / (2 * Nst), rem = idx - t * 2 * Nst, sd = rem / Nst, o = rem - sd * Nst;
      if (j0 + t >= nf) continue;
      const int tet = sd ? right[j0 + t] : left[j0 + t];
      if (tet >= 0) ps[t][sd][o] = df_split(Pp[(size_t)tet * Nst + o]);
    }
    __syncthreads();
    if (!act) continue;
    float2 S[3][(NG + 1) / 2], C[3][(NG + 1) / 2];
    sup_face_qp<N, NG>(j, m, right[j] >= 0, Q, ps[tl], S, C);
    double o[3][NG];
    sup_mix<NG>(K, S, C, o);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int a = 0; a < NG; ++a) G[(size_t)j * 3 * Nst + (c * NG + a) * N + m] = dt * o[c][a];
  }
}

// velocity update: thread (face, m); boundary faces V = F
template <int N, int NG>
__global__ void __launch_bounds__(kSupThreads) k_update_p(int nf, const int* __restrict__ left,
                                                          const int* __restrict__ right, const double* __restrict__ Q,
                                                          const double* __restrict__ F, const double* __restrict__ dp,
                                                          double dt, SupK K, double* __restrict__ V) {
  constexpr int Nst = N * NG, TB = kSupThreads / N;
  __shared__ float2 ps[TB][2][Nst];
  const int tl = threadIdx.x / N, m = threadIdx.x - tl * N;
  for (int j0 = blockIdx.x * TB; j0 < nf; j0 += gridDim.x * TB) {
    const int j = j0 + tl;
    const bool act = tl < TB && j < nf;
    __syncthreads();
    for (int idx = threadIdx.x; idx < TB * 2 * Nst; idx += kSupThreads) {
      const int t = idx / (2 * Nst), rem = idx - t * 2 * Nst, sd = rem / Nst, o = rem - sd * Nst;
      if (j0 + t >= nf) continue;
      const int tet = sd ? right[j0 + t] : left[j0 + t];
      if (tet >= 0) ps[t][sd][o] = df_split(dp[(size_t)tet * Nst + o]);
    }
    __syncthreads();
    if (!act) continue;
    const double* Fj = F + (size_t)j * 3 * Nst;
    double* Vj = V + (size_t)j * 3 * Nst;
    if (right[j] < 0) {
#pragma unroll
      for (int r = 0; r < 3 * NG; ++r) Vj[r * N + m] = Fj[r * N + m];
      continue;
    }
    float2 S[3][(NG + 1) / 2], C[3][(NG + 1) / 2];
    sup_face_qp<N, NG>(j, m, true, Q, ps[tl], S, C);
    double o[3][NG];
    sup_mix<NG>(K, S, C, o);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int a = 0; a < NG; ++a) Vj[(c * NG + a) * N + m] = Fj[(c * NG + a) * N + m] - dt * o[c][a];
  }
}

constexpr int kSupBlocks = 152 * 8;

static SupK sup_k(const double* Kinv, int Ng) {
  SupK k{};
  for (int q = 0; q < Ng * Ng; ++q) {
    const float h = (float)Kinv[q];
    k.v[q] = make_float2(h, (float)(Kinv[q] - (double)h));
  }
  return k;
}

}  // namespace

bool support_fp64() {
  static const bool v = std::getenv("STDG_SUPPORT") && std::strcmp(std::getenv("STDG_SUPPORT"), "fp64") == 0;
  return v;
}

// The launchers return cudaErrorNotSupported where (N, Ng) has no compile-time kernel; the callers
// then use the binary64 kernels.
#define STDG_SUP_DISPATCH(N_, NG_, CALL)                                                  \
  if (N_ == 35 && NG_ == 5) { constexpr int SN = 35, SG = 5; CALL; return cudaGetLastError(); } \
  if (N_ == 20 && NG_ == 2) { constexpr int SN = 20, SG = 2; CALL; return cudaGetLastError(); } \
  return cudaErrorNotSupported;

cudaError_t sup_average(cudaStream_t st, int ne, int N, int Ng, const int* t2f, const int* left, const double* detJ,
                        const double* Mij, const double* in, double* out) {
  STDG_SUP_DISPATCH(N, Ng, (k_average_p<SN, SG><<<kSupBlocks, kSupThreads, 0, st>>>(ne, t2f, left, detJ, Mij, in, out)))
}
cudaError_t sup_face_grad(cudaStream_t st, int nf, int N, int Ng, const int* left, const int* right, const double* Q,
                          const double* Pp, double dt, const double* Kinv, double* G) {
  const SupK k = sup_k(Kinv, Ng);
  STDG_SUP_DISPATCH(N, Ng, (k_face_grad_p<SN, SG><<<kSupBlocks, kSupThreads, 0, st>>>(nf, left, right, Q, Pp, dt, k, G)))
}
cudaError_t sup_update(cudaStream_t st, int nf, int N, int Ng, const int* left, const int* right, const double* Q,
                       const double* F, const double* dp, double dt, const double* Kinv, double* V) {
  const SupK k = sup_k(Kinv, Ng);
  STDG_SUP_DISPATCH(N, Ng, (k_update_p<SN, SG><<<kSupBlocks, kSupThreads, 0, st>>>(nf, left, right, Q, F, dp, dt, k, V)))
}
}  // namespace stdg
