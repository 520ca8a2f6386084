// Krylov solvers on the device (Sec. 2.4: matrix-free, unpreconditioned GMRES; Sec. 2.7: CG for
// p_t = 0).  Every reduction is two-stage over a fixed grid, so results are bitwise
// reproducible run to run.  Vectors use the pressure layout P[ne][Ng][N].
#include <string>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "solver.h"

namespace stdg {

constexpr int kRedBlocks = 1216;   // 8 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kMaxCols = 64;
constexpr int kLpBlocksK = 1216;   // partial rows the binary32 block-Jacobi kernels write (lowprec.cu)

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce `cnt` per-thread values (cnt <= 8) into part[blockIdx.x * stride + c].
__device__ inline void block_reduce_store(double* v, int cnt, double* part, int stride) {
  __shared__ double red[8][kRedThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < cnt; ++c) {
    double s = warp_sum(v[c]);
    if (lane == 0) red[c][w] = s;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) s += red[threadIdx.x][k];
    part[blockIdx.x * stride + threadIdx.x] = s;
  }
}

// per-time-column dot products: part[b][a] = Sum over this block's elements of column a
__global__ void __launch_bounds__(kRedThreads) k_coldot(int64_t n, int N, int Ng, const double* __restrict__ x,
                                                       const double* __restrict__ y, double* part) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)((e / N) % Ng);
    acc[a] = fma(x[e], y[e], acc[a]);
  }
  block_reduce_store(acc, Ng, part, Ng);
}

// x += alpha_a p; r -= alpha_a q; partials of r.r per column (slot a) and of ||(I (x) Tp) r||^2 (slot Ng)
struct TpArg { double v[kMaxNg * kMaxNg]; };
// want = 0 (block-Jacobi PCG between convergence checks): only the x and r updates; the binary64
// pipe is 1/64 of the binary32 rate on sm_103a, so the norms are not formed when nobody reads them.
__global__ void __launch_bounds__(kRedThreads) k_cg_update(int64_t ne, int N, int Ng, const double* __restrict__ alpha,
                                                          double* __restrict__ x, double* __restrict__ r,
                                                          const double* __restrict__ p, const double* __restrict__ q,
                                                          TpArg Tp, double* part, int want = 1) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double al[kMaxNg];
  for (int a = 0; a < Ng; ++a) al[a] = alpha[a];
  const int64_t npairs = ne * N;
  const int Nst = N * Ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npairs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int k = (int)(e % N);
    double rv[kMaxNg];
    for (int a = 0; a < Ng; ++a) {
      const int64_t o = i * Nst + a * N + k;
      x[o] = fma(al[a], p[o], x[o]);
      double rn = fma(-al[a], q[o], r[o]);
      r[o] = rn;
      rv[a] = rn;
      if (want) acc[a] = fma(rn, rn, acc[a]);
    }
    if (want)
      for (int a = 0; a < Ng; ++a) {
        double w = 0.0;
        for (int b = 0; b < Ng; ++b) w = fma(Tp.v[a * Ng + b], rv[b], w);
        acc[Ng] = fma(w, w, acc[Ng]);
      }
  }
  if (want) block_reduce_store(acc, Ng + 1, part, Ng + 1);
}

// z_i[a][k] = Sum_l Binv_i[k][l] r_i[a][l]  (block Jacobi); partials of r.z per column a.
// Fixed grid (kRedBlocks blocks striding over tets) so the partials stay deterministic.
__global__ void __launch_bounds__(128) k_bjacobi(int ne, int N, int Ng, const double* __restrict__ Binv,
                                                 const double* __restrict__ r, double* __restrict__ z,
                                                 double* part) {
  extern __shared__ double sm[];
  const int Nst = N * Ng;
  const size_t NN = (size_t)N * N;
  double* rs = sm;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x; i < ne; i += gridDim.x) {
    __syncthreads();
    for (int o = threadIdx.x; o < Nst; o += blockDim.x) rs[o] = r[(size_t)i * Nst + o];
    __syncthreads();
    for (int o = threadIdx.x; o < Nst; o += blockDim.x) {
      const int a = o / N, k = o % N;
      const double* B = Binv + (size_t)i * NN + k;     // symmetric: read column k (coalesced over k)
      double s = 0.0;
      for (int l = 0; l < N; ++l) s = fma(B[(size_t)l * N], rs[a * N + l], s);
      z[(size_t)i * Nst + o] = s;
      acc[a] = fma(s, rs[o], acc[a]);
    }
  }
  __shared__ double red[8][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int a = 0; a < Ng; ++a) {
    double v = warp_sum(acc[a]);
    if (lane == 0) red[a][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < Ng) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    part[(size_t)blockIdx.x * Ng + threadIdx.x] = s;
  }
}

// Same with binary32 inverses and binary32 products (the preconditioner need not be FP64; the
// CG iterates, residuals and scalars stay binary64).
__global__ void __launch_bounds__(256) k_bjacobi32(int ne, int N, int Ng, const float* __restrict__ Binv,
                                                   const double* __restrict__ r, double* __restrict__ z,
                                                   double* part) {
  extern __shared__ float rsf[];
  const int Nst = N * Ng;
  const int TB = blockDim.x / Nst;
  const size_t NN = (size_t)N * N;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int tl = threadIdx.x / Nst, o = threadIdx.x - tl * Nst, a = o / N, k = o - a * N;
  for (int i0 = blockIdx.x * TB; i0 < ne; i0 += gridDim.x * TB) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < TB * Nst; idx += blockDim.x) {
      const int i = i0 + idx / Nst;
      rsf[idx] = i < ne ? (float)r[(size_t)i0 * Nst + idx] : 0.0f;
    }
    __syncthreads();
    const int i = i0 + tl;
    if (tl < TB && i < ne) {
      const float* B = Binv + (size_t)i * NN + k;
      const float* rr = rsf + tl * Nst + a * N;
      float sacc = 0.0f;
      for (int l = 0; l < N; ++l) sacc = fmaf(B[(size_t)l * N], rr[l], sacc);
      z[(size_t)i * Nst + o] = (double)sacc;
      acc[a] = fma((double)sacc, r[(size_t)i * Nst + o], acc[a]);
    }
  }
  __shared__ double red[8][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = 0; q < Ng; ++q) {
    double v = warp_sum(acc[q]);
    if (lane == 0) red[q][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < Ng) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x][q];
    part[(size_t)blockIdx.x * Ng + threadIdx.x] = t;
  }
}

// beta_a = rznew_a / rz_a; rz <- rznew; res = sqrt(mix2)
__global__ void k_cg_beta2(int Ng, double* rz, const double* rznew, double* beta, double* res, const double* mix2) {
  int a = threadIdx.x;
  if (a < Ng) {
    beta[a] = (rz[a] != 0.0) ? rznew[a] / rz[a] : 0.0;
    rz[a] = rznew[a];
  }
  if (a == 0) res[0] = sqrt(mix2[0]);
}

// p = r + beta_a p
__global__ void k_cg_dir(int64_t n, int N, int Ng, const double* __restrict__ beta, const double* __restrict__ r,
                         double* __restrict__ p) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)((e / N) % Ng);
    p[e] = fma(beta[a], p[e], r[e]);
  }
}

// out[c] = Sum_b part[b * width + c] in fixed order (one block per column)
__global__ void k_final(int nparts, int width, const double* __restrict__ part, double* __restrict__ out,
                        const double* gate = nullptr) {
  if (gate && gate[0] == 0.0) {                   // gated off: the result is 0
    if (threadIdx.x == 0) out[blockIdx.x] = 0.0;
    return;
  }
  __shared__ double red[kRedThreads / 32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(size_t)b * width + c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) t += red[k];
    out[c] = t;
  }
}

// alpha_a = rr_a / pq_a ; (guarded)
__global__ void k_cg_alpha(int Ng, const double* rr, const double* pq, double* alpha) {
  int a = threadIdx.x;
  if (a < Ng) alpha[a] = (pq[a] != 0.0) ? rr[a] / pq[a] : 0.0;
}
// Guarded step length for the binary32 CG of the mixed-precision solve: a breakdown (p.Ap <= 0 or a
// non-finite step in any column: the rounded operator has lost definiteness along p) freezes the
// recurrence (alpha = 0) and raises flag[0] until the host restarts the direction.
__global__ void k_cg_alpha_guard(int Ng, const double* rr, const double* pq, double* alpha, double* flag) {
  const int a = threadIdx.x;
  double al = 0.0;
  bool bad = false;
  if (a < Ng) {
    al = rr[a] / pq[a];
    bad = flag[0] != 0.0 || !(pq[a] > 0.0) || !isfinite(al);
  }
  bad = __any_sync(0xffffffffu, bad);
  if (a < Ng) alpha[a] = bad ? 0.0 : al;
  if (a == 0 && bad) flag[0] = 1.0;
}
// One block: reduce the per-block p.q partials of every column in a fixed order, then the guarded
// step length of k_cg_alpha_guard (one launch instead of two per binary32 iteration).
__global__ void k_final_alpha_guard(int nparts, int Ng, const double* __restrict__ part, const double* rz,
                                    double* alpha, double* flag) {
  __shared__ double red[kMaxNg][kRedThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int a = 0; a < Ng; ++a) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(size_t)b * Ng + a];
    s = warp_sum(s);
    if (lane == 0) red[a][w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double al[kMaxNg];
    bool bad = flag[0] != 0.0;
    for (int a = 0; a < Ng; ++a) {
      double pq = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) pq += red[a][q];
      al[a] = rz[a] / pq;
      if (!(pq > 0.0) || !isfinite(al[a])) bad = true;
    }
    for (int a = 0; a < Ng; ++a) alpha[a] = bad ? 0.0 : al[a];
    if (bad) flag[0] = 1.0;
  }
}
// k_cg_beta2 for the mixed solve: the residual estimate reads -1 once the recurrence is frozen
__global__ void k_cg_beta_guard(int Ng, double* rz, const double* rznew, double* beta, double* res, const double* mix2,
                                const double* flag) {
  int a = threadIdx.x;
  if (a < Ng) {
    beta[a] = (rz[a] != 0.0) ? rznew[a] / rz[a] : 0.0;
    rz[a] = rznew[a];
  }
  if (a == 0) res[0] = flag[0] != 0.0 ? -1.0 : sqrt(mix2[0]);
}
// Preconditioner of the viscous systems (Eq. A1_mod): the inverse of their mass part,
// z_i = (mass |J_i| K)^-1 (x) I r_i (K^-1 passed in Kinv), with partials of r.z per column.
__global__ void __launch_bounds__(kRedThreads) k_visc_mass_inv(int64_t ne, int N, int Ng, TpArg Kinv, double mass,
                                                              const double* __restrict__ detJ,
                                                              const double* __restrict__ r, double* __restrict__ z,
                                                              double* part) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int Nst = N * Ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int k = (int)(e % N);
    const double c = 1.0 / (mass * detJ[i]);
    double rv[kMaxNg];
    for (int b = 0; b < Ng; ++b) rv[b] = r[i * Nst + b * N + k];
    for (int a = 0; a < Ng; ++a) {
      double s = 0.0;
      for (int b = 0; b < Ng; ++b) s = fma(Kinv.v[a * Ng + b], rv[b], s);
      s *= c;
      z[i * Nst + a * N + k] = s;
      if (part) acc[a] = fma(s, rv[a], acc[a]);
    }
  }
  if (part) block_reduce_store(acc, Ng, part, Ng);
}

// Classical Gram-Schmidt reorthogonalisation test ("twice is enough", Giraud et al. 2005): a second
// pass is needed only when the first removed more than half of ||w||^2, i.e. when
// ||w||^2 - Sum h^2 < ||w||^2 / 2 (cancellation then makes the left side small, so the test errs
// towards reorthogonalising).  gate[0] = 1 if the second pass runs.
__global__ void k_reorth_gate(int cnt, const double* h, const double* w2, double* gate) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < cnt; ++i) s = fma(h[i], h[i], s);
  gate[0] = (w2[0] - s < 0.5 * w2[0]) ? 1.0 : 0.0;
}

// alpha_a = rz_a / (Sum of the partials of p.q)_a, one block per column (fixed order: deterministic)
__global__ void k_final_alpha(int nparts, int Ng, const double* __restrict__ part, const double* rz, double* alpha) {
  const int a = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(size_t)b * Ng + a];
  __shared__ double red[kRedThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) t += red[q];
    alpha[a] = t != 0.0 ? rz[a] / t : 0.0;
  }
}
// rznew_a = Sum of the partials of r.z; beta_a = rznew_a / rz_a; rz_a = rznew_a
__global__ void k_final_beta(int nparts, int Ng, const double* __restrict__ part, double* rz, double* beta) {
  const int a = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(size_t)b * Ng + a];
  __shared__ double red[kRedThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) t += red[q];
    beta[a] = rz[a] != 0.0 ? t / rz[a] : 0.0;
    rz[a] = t;
  }
}
// res = sqrt of the reduced ||(I (x) Tp) r||^2 partials (slot Ng of width Ng + 1)
__global__ void k_final_res(int nparts, int width, int slot, const double* __restrict__ part, double* res) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(size_t)b * width + slot];
  __shared__ double red[kRedThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) t += red[q];
    res[0] = sqrt(t);
  }
}
// flexible CG with m stored directions: per direction j (blockIdx.y) and column a, partials of z.Q_j
__global__ void __launch_bounds__(kRedThreads) k_fcg_dots(int64_t n, int N, int Ng, int m, const double* __restrict__ Qb,
                                                         const double* __restrict__ z, double* part) {
  const int j = blockIdx.y;
  const double* Q = Qb + (size_t)j * n;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc[(e / N) % Ng] = fma(z[e], Q[e], acc[(e / N) % Ng]);
  __shared__ double red[8][kRedThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < Ng; ++c) {
    double s = warp_sum(acc[c]);
    if (lane == 0) red[c][w] = s;
  }
  __syncthreads();
  if (threadIdx.x < Ng) {
    double s = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) s += red[threadIdx.x][q];
    part[(size_t)blockIdx.x * m * Ng + j * Ng + threadIdx.x] = s;
  }
}
// c[j][a] = -(z.Q_j)_a / (P_j.Q_j)_a
__global__ void k_fcg_coef(int cnt, const double* zq, const double* pq, double* c) {
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) c[t] = pq[t] != 0.0 ? -zq[t] / pq[t] : 0.0;
}
// p = z + Sum_j c[j][a] P_j  (column a of each entry)
__global__ void k_fcg_dir(int64_t n, int N, int Ng, int m, const double* __restrict__ c, const double* __restrict__ Pb,
                          const double* __restrict__ z, double* __restrict__ p) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)((e / N) % Ng);
    double v = z[e];
    for (int j = 0; j < m; ++j) v = fma(c[j * Ng + a], Pb[(size_t)j * n + e], v);
    p[e] = v;
  }
}
// beta_a = rrnew_a / rr_a; rr <- rrnew; res = sqrt(tp2)
__global__ void k_cg_beta(int Ng, double* rr, const double* rrnew, double* beta, double* res) {
  int a = threadIdx.x;
  if (a < Ng) {
    beta[a] = (rr[a] != 0.0) ? rrnew[a] / rr[a] : 0.0;
    rr[a] = rrnew[a];
  }
  if (a == 0) res[0] = sqrt(rrnew[Ng]);
}

// y_a-mixing: out[i][a][k] = coef Sum_b M[a][b] in[i][b][k]
__global__ void k_timemix(int64_t ne, int N, int Ng, TpArg M, double coef, const double* __restrict__ in,
                          double* __restrict__ out) {
  const int Nst = N * Ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int k = (int)(e % N);
    double v[kMaxNg];
    for (int b = 0; b < Ng; ++b) v[b] = in[i * Nst + b * N + k];
    for (int a = 0; a < Ng; ++a) {
      double s = 0.0;
      for (int b = 0; b < Ng; ++b) s = fma(M.v[a * Ng + b], v[b], s);
      out[i * Nst + a * N + k] = coef * s;
    }
  }
}

// GMRES helpers -------------------------------------------------------------------------------
// part[v][b]: dot of basis vector v with w over this block's range
__global__ void __launch_bounds__(kRedThreads) k_multidot(int64_t n, const double* __restrict__ Vb,
                                                         const double* __restrict__ w, double* part,
                                                         const double* gate = nullptr) {
  if (gate && gate[0] == 0.0) return;             // second Gram-Schmidt pass not needed
  const int v = blockIdx.y;
  const double* vv = Vb + (size_t)v * n;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc = fma(vv[e], w[e], acc);
  __shared__ double red[kRedThreads / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) s += red[k];
    part[(size_t)blockIdx.x * gridDim.y + v] = s;
  }
}
// w += sign Sum_v h[v] V[v]
__global__ void k_multiaxpy(int64_t n, int nv, const double* __restrict__ Vb, const double* __restrict__ h,
                            double sign, double* __restrict__ w, const double* gate = nullptr) {
  if (gate && gate[0] == 0.0) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int v = 0; v < nv; ++v) s = fma(h[v], Vb[(size_t)v * n + e], s);
    w[e] = fma(sign, s, w[e]);
  }
}
__global__ void __launch_bounds__(kRedThreads) k_sumsq(int64_t n, const double* __restrict__ x, double* part) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[e], x[e], acc);
  block_reduce_store(&acc, 1, part, 1);
}
__global__ void k_scale_copy(int64_t n, const double* __restrict__ in, const double* __restrict__ sc, int mode,
                             double* __restrict__ out) {
  // mode 0: out = in / sqrt(sc[0]);  mode 1: out = in - out (residual r = b - Ax, out holds Ax)
  double f = (mode == 0) ? 1.0 / sqrt(sc[0]) : 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (mode == 0) ? in[e] * f : in[e] - out[e];
}

// Every device array of a solver comes from here: the caller's allocator when one was given at
// creation, else cudaMalloc.  The arrays are released together by stdg_solver_destroy.
stdg_status dev_alloc(stdg_solver* s, void** p, size_t bytes) {
  const size_t b = bytes ? bytes : 16;
  *p = nullptr;
  if (s->alloc_fn) {
    *p = s->alloc_fn(b, (void*)s->stream, s->alloc_user);
    if (!*p) {
      set_error("device allocation of %zu bytes failed (caller's allocator)", b);
      return STDG_ENOMEM;
    }
  } else {
    cudaError_t e = cudaMalloc(p, b);
    if (e != cudaSuccess) {
      *p = nullptr;
      set_error("cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
      return STDG_ENOMEM;
    }
  }
  s->allocs.push_back({*p, b});
  return STDG_OK;
}

cudaError_t dev_alloc_cuda(stdg_solver* s, void** p, size_t bytes) {
  return dev_alloc(s, p, bytes) == STDG_OK ? cudaSuccess : cudaErrorMemoryAllocation;
}

// Release one array obtained from dev_alloc before the solver is destroyed (stream-ordered use of it
// must have finished: the caller synchronises first).
void dev_free(stdg_solver* s, void* p) {
  for (size_t k = 0; k < s->allocs.size(); ++k)
    if (s->allocs[k].p == p) {
      if (s->free_fn) s->free_fn(p, s->allocs[k].bytes, (void*)s->stream, s->alloc_user);
      else cudaFree(p);
      s->allocs.erase(s->allocs.begin() + (long)k);
      return;
    }
}

stdg_status ensure_krylov(stdg_solver* s) {
  if (s->kb) return STDG_OK;
  const size_t n = (size_t)s->ne * s->Nst * sizeof(double);
  stdg_status st;
  for (double** v : {&s->kb, &s->kx, &s->kr, &s->kp, &s->kq, &s->kz})
    if ((st = dev_alloc(s, (void**)v, n)) != STDG_OK) return st;
  if ((st = dev_alloc(s, (void**)&s->part, (size_t)kRedBlocks * kMaxCols * sizeof(double))) != STDG_OK) return st;
  if ((st = dev_alloc(s, (void**)&s->scal, 1024 * sizeof(double))) != STDG_OK) return st;
  if (cudaMallocHost((void**)&s->hostbuf, 1024 * sizeof(double)) != cudaSuccess) {
    set_error("cudaMallocHost failed");
    return STDG_ENOMEM;
  }
  return STDG_OK;
}

static stdg_status ensure_basis(stdg_solver* s, int cols) {
  if (s->basis && s->basis_cols >= cols) return STDG_OK;
  const size_t n = (size_t)s->ne * s->Nst;
  return dev_alloc(s, (void**)&s->basis, (size_t)cols * n * sizeof(double)) == STDG_OK
             ? (s->basis_cols = cols, STDG_OK)
             : STDG_ENOMEM;
}

static double host_norm(stdg_solver* s, const double* v, int64_t n) {
  ++s->nlaunch;
  k_sumsq<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, v, s->part);
  ++s->nlaunch;
  k_final<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, 1, s->part, s->scal + 900);
  cudaMemcpyAsync(s->hostbuf + 900, s->scal + 900, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  cudaStreamSynchronize(s->stream);
  return std::sqrt(s->hostbuf[900]);
}

void prof_fold(stdg_solver* s) {
  if (s->ev_used == 0) return;
  cudaEventSynchronize(s->ev[2 * s->ev_used - 1]);
  for (int k = 0; k < s->ev_used; ++k) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->ev[2 * k], s->ev[2 * k + 1]);
    s->op_ms += ms;
    s->kind_ms[s->ev_kind[k]] += ms;
    s->kind_n[s->ev_kind[k]] += 1;
  }
  s->ev_used = 0;
}

// the binary64-accurate pair kernel serves this operator (the pressure operator; with the warp
// kernels also the viscous operator of Eq. A1_mod) in every precision mode but plain FP64
static bool df_serves(const stdg_solver* s, const ApplyArgs& a) {
  if (s->opt.precision == STDG_PREC_FP64) return false;     // DF32 and the mixed modes (outer and viscous)
  if (a.Bextra == nullptr && a.mass_coef == 0.0) return s->dfB || s->wdB;
  return s->wdBv && a.Bextra == s->Bvisc && a.extra_coef == -1.0 && a.tacc_identity && !a.pinned;
}

// y = op x with the binary64-accurate kernel for this operator (the pair kernel where it serves,
// else the binary64 kernel), or with the binary64 kernel alone when fp64_only
static stdg_status op_apply(stdg_solver* s, const ApplyArgs& a, const double* x, double* y, bool fp64_only = false) {
  const bool prof = s->prof && !s->ev.empty() && !s->capturing;
  const bool use_df = !fp64_only && df_serves(s, a);
  if (prof) {
    if (2 * s->ev_used >= (int)s->ev.size()) prof_fold(s);
    s->ev_kind[s->ev_used] = use_df ? 1 : 0;
    cudaEventRecord(s->ev[2 * s->ev_used], s->stream);
  }
  ++s->nlaunch;
  ++s->op_launches;
  // binary64-accurate operator from binary32 pairs when requested (pressure operator only)
  cudaError_t e = !use_df ? launch_apply(a, x, y, s->stream)
                 : a.Bextra ? launch_apply_warp_df_visc(s, x, y, a.scale, a.mass_coef, a.Kmass)
                            : launch_apply_df(s, x, y, a.pinned, a.tacc_identity, a.scale, a.pin_diag);
  if (prof) {
    cudaEventRecord(s->ev[2 * s->ev_used + 1], s->stream);
    ++s->ev_used;
  }
  if (e != cudaSuccess) { set_error("operator launch failed: %s", cudaGetErrorString(e)); return STDG_ECUDA; }
  return STDG_OK;
}

static ApplyArgs pressure_op(stdg_solver* s, int pinned, int kron, double scale, double pin_diag) {
  ApplyArgs a{};
  a.ne = (int)s->ne; a.N = s->N; a.Ng = s->Ng;
  a.t2f = s->dm.t2f; a.t2n = s->dm.t2n; a.left = s->dm.left;
  a.Bdiag = s->Bdiag; a.Aoff = s->Aoff; a.Bextra = nullptr; a.detJ = s->dm.detJ;
  a.extra_coef = 0.0; a.scale = scale; a.mass_coef = 0.0; a.pin_diag = pin_diag;
  a.tacc_identity = kron; a.pinned = pinned;
  for (int q = 0; q < s->Ng * s->Ng; ++q) a.Tacc[q] = s->tm.Tp[q];
  return a;
}

stdg_status apply_pressure(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale,
                           double pin_diag) {
  return op_apply(s, pressure_op(s, pinned, kron, scale, pin_diag), x, y);
}

// A batch of B iterations of `body` captured once into a CUDA graph and replayed on the solver's
// internal stream, ordered after and before the caller's stream by events (the caller's stream may
// be a legacy stream that cannot be captured).
struct GraphLoop {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int B = 0;
  bool prof = false;
  ~GraphLoop() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

static stdg_status graph_streams(stdg_solver* s, int B) {
  if (!s->cstream) {
    if (cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->sync_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->sync_ev[1], cudaEventDisableTiming) != cudaSuccess) {
      set_error("internal stream creation failed");
      return STDG_ECUDA;
    }
  }
  if ((int)s->gev.size() < 2 * B) {
    for (cudaEvent_t e : s->gev) cudaEventDestroy(e);
    s->gev.assign(2 * B, nullptr);
    for (auto& e : s->gev)
      if (cudaEventCreate(&e) != cudaSuccess) { set_error("cudaEventCreate failed"); return STDG_ECUDA; }
  }
  return STDG_OK;
}

template <typename Body>
static stdg_status graph_capture(stdg_solver* s, int B, Body body, GraphLoop& g) {
  stdg_status st = graph_streams(s, B);
  if (st != STDG_OK) return st;
  cudaStream_t user = s->stream;
  s->stream = s->cstream;
  g.prof = s->prof;
  g.B = B;
  s->capturing = true;
  if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    s->capturing = false; s->stream = user;
    set_error("stream capture failed to start");
    return STDG_ECUDA;
  }
  for (int j = 0; j < B && st == STDG_OK; ++j) st = body(j, g.prof ? &s->gev[2 * j] : nullptr);
  cudaError_t ce = cudaStreamEndCapture(s->stream, &g.graph);
  s->capturing = false;
  s->stream = user;
  if (st != STDG_OK) return st;
  if (ce != cudaSuccess || cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) {
    set_error("graph capture/instantiation failed: %s", cudaGetErrorString(ce));
    return STDG_ECUDA;
  }
  return STDG_OK;
}

static stdg_status graph_launch(stdg_solver* s, GraphLoop& g, int kernels_per_iter, int kind) {
  cudaEventRecord(s->sync_ev[0], s->stream);
  cudaStreamWaitEvent(s->cstream, s->sync_ev[0], 0);
  if (cudaGraphLaunch(g.exec, s->cstream) != cudaSuccess) {
    set_error("graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return STDG_ECUDA;
  }
  cudaEventRecord(s->sync_ev[1], s->cstream);
  cudaStreamWaitEvent(s->stream, s->sync_ev[1], 0);
  s->nlaunch += (int64_t)g.B * kernels_per_iter;
  s->op_launches += g.B;
  if (g.prof) {
    if (cudaStreamSynchronize(s->cstream) != cudaSuccess) { set_error("graph launch failed"); return STDG_ECUDA; }
    for (int j = 0; j < g.B; ++j) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, s->gev[2 * j], s->gev[2 * j + 1]);
      s->op_ms += ms;
      s->kind_ms[kind] += ms;
      s->kind_n[kind] += 1;
    }
  }
  return STDG_OK;
}

// Run `body` (one Krylov iteration that ends by copying its residual to host_slot) in batches of
// B iterations captured once into a CUDA graph and replayed on an internal stream; the caller's
// stream is ordered before and after by events.  Up to B-1 iterations may run past convergence;
// they are counted.  Operator launches inside the graph are timed by dedicated event nodes.
template <typename Body>
static stdg_status run_batched(stdg_solver* s, int B, int kernels_per_iter, int max_it, double tol_abs, Body body,
                               int* iters, double* rabs_out, int kind, bool last_only = false) {
  if (!s->cstream) {
    if (cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->sync_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->sync_ev[1], cudaEventDisableTiming) != cudaSuccess) {
      set_error("internal stream creation failed");
      return STDG_ECUDA;
    }
  }
  if ((int)s->gev.size() < 2 * B) {
    for (cudaEvent_t e : s->gev) cudaEventDestroy(e);
    s->gev.assign(2 * B, nullptr);
    for (auto& e : s->gev)
      if (cudaEventCreate(&e) != cudaSuccess) { set_error("cudaEventCreate failed"); return STDG_ECUDA; }
  }
  cudaStream_t user = s->stream;
  cudaEventRecord(s->sync_ev[0], user);
  cudaStreamWaitEvent(s->cstream, s->sync_ev[0], 0);
  s->stream = s->cstream;
  const bool prof = s->prof;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  stdg_status st = STDG_OK;
  s->capturing = true;
  if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    s->capturing = false; s->stream = user;
    set_error("stream capture failed to start");
    return STDG_ECUDA;
  }
  for (int j = 0; j < B && st == STDG_OK; ++j) st = body(j, prof ? &s->gev[2 * j] : nullptr);
  cudaError_t ce = cudaStreamEndCapture(s->stream, &graph);
  s->capturing = false;
  if (st == STDG_OK && (ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)) {
    set_error("graph capture/instantiation failed: %s", cudaGetErrorString(ce));
    st = STDG_ECUDA;
  }
  int it = 0;
  double rabs = INFINITY;
  while (st == STDG_OK && it < max_it) {
    if (cudaGraphLaunch(exec, s->stream) != cudaSuccess || cudaStreamSynchronize(s->stream) != cudaSuccess) {
      set_error("graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
      st = STDG_ECUDA;
      break;
    }
    it += B;
    s->nlaunch += (int64_t)B * kernels_per_iter;
    s->op_launches += B;
    if (prof) {
      for (int j = 0; j < B; ++j) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->gev[2 * j], s->gev[2 * j + 1]);
        s->op_ms += ms;
        s->kind_ms[kind] += ms;
        s->kind_n[kind] += 1;
      }
    }
    bool done = false;
    for (int j = last_only ? B - 1 : 0; j < B; ++j) {
      rabs = s->hostbuf[j];
      if (!std::isfinite(rabs)) { set_error("Krylov: non-finite residual"); st = STDG_ENAN; break; }
      if (rabs <= tol_abs) { done = true; }
    }
    rabs = s->hostbuf[B - 1];
    if (done) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaEventRecord(s->sync_ev[1], s->stream);
  s->stream = user;
  cudaStreamWaitEvent(user, s->sync_ev[1], 0);
  *iters = it;
  *rabs_out = rabs;
  return st;
}

static stdg_status ensure_block_inverse(stdg_solver* s) {
  if (s->Binv) return STDG_OK;
  const size_t cnt = (size_t)s->ne * s->N * s->N;
  stdg_status e = dev_alloc(s, (void**)&s->Binv, cnt * sizeof(double));
  if (e != STDG_OK) return e;
  if ((e = dev_alloc(s, (void**)&s->lpBinv, cnt * sizeof(float))) != STDG_OK) return e;
  s->nlaunch += 2;
  cudaError_t ce = launch_block_inverse((int)s->ne, s->N, s->Bdiag, s->Binv, s->stream);
  if (ce == cudaSuccess) { lp_kernels().f32(s->stream, (int64_t)cnt, s->Binv, s->lpBinv); ce = cudaGetLastError(); }
  if (ce != cudaSuccess) { set_error("block inverse launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  return STDG_OK;
}

// Block CG for an operator that is symmetric positive definite on each time column, optionally
// preconditioned by block Jacobi (precond 1: per-tet inverses of the pinned diagonal blocks of -A), or
// by block Jacobi plus the agglomeration coarse correction of mg.cu (precond 2).
// x holds the initial guess unless zero_x0.  Stops when ||(I (x) mix) r|| <= tol_abs.
static stdg_status cg_block(stdg_solver* s, const ApplyArgs& op, const double* rhs, double* x, bool zero_x0,
                            const TpArg& mix, double tol_abs, int* iters, double* res_abs, int precond = 0) {
  const int N = s->N, Ng = s->Ng;
  const int64_t n = s->ne * (int64_t)s->Nst;
  double* r = s->kr; double* p = s->kp; double* q = s->kq; double* z = s->kz;
  double* rz = s->scal; double* pq = s->scal + 8; double* alpha = s->scal + 16; double* beta = s->scal + 24;
  double* rrnew = s->scal + 32; double* res = s->scal + 48; double* rznew = s->scal + 56;
  const int bj_tb = s->Nst > 256 ? 1 : 256 / s->Nst;
  const int bj_threads = bj_tb * s->Nst > 256 ? s->Nst : 256;
  const size_t bj_smem = (size_t)bj_tb * s->Nst * sizeof(float);
  if (precond) {
    stdg_status e = ensure_block_inverse(s);
    if (e == STDG_OK && precond == 2) e = mg_ensure(s);
    if (e != STDG_OK) return e;
  }
  // block Jacobi writes kRedBlocks rows of r.z partials, the coarse correction its own rows after them
  const bool mg = precond == 2;
  const int nrz = kRedBlocks + (mg ? mg_partial_blocks() : 0);
  double* mgpart = s->part + (size_t)kRedBlocks * Ng;
  if (zero_x0) {
    cudaMemsetAsync(x, 0, n * sizeof(double), s->stream);
    cudaMemcpyAsync(r, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
  } else {
    stdg_status e = op_apply(s, op, x, r);
    if (e != STDG_OK) return e;
    ++s->nlaunch;
    k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, rhs, nullptr, 1, r);
  }
  if (precond) {
    ++s->nlaunch;
    k_bjacobi32<<<kRedBlocks, bj_threads, bj_smem, s->stream>>>((int)s->ne, N, Ng, s->lpBinv, r, z, s->part);
    if (mg) { mg_apply_f64(s, r, z, mgpart); s->nlaunch += mg_launches(s); }
    cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
  } else {
    cudaMemcpyAsync(p, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    ++s->nlaunch;
    k_coldot<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, r, r, s->part);
  }
  ++s->nlaunch;
  k_final<<<Ng, kRedThreads, 0, s->stream>>>(precond ? nrz : kRedBlocks, Ng, s->part, rz);
  // one CG iteration; ends by copying the full-system residual norm to the host.  With the
  // preconditioner, inside a captured batch only the batch's last iteration forms the norm (the
  // host reads only that one), and the step length / beta come from fused reduction kernels.
  const int Bb = s->opt.graph_batch > 1 ? s->opt.graph_batch : 1;
  auto body = [&](int slot, cudaEvent_t* evs) -> stdg_status {
    if (evs) cudaEventRecordWithFlags(evs[0], s->stream, cudaEventRecordExternal);
    stdg_status e = op_apply(s, op, p, q);
    if (evs) cudaEventRecordWithFlags(evs[1], s->stream, cudaEventRecordExternal);
    if (e != STDG_OK) return e;
    k_coldot<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, p, q, s->part);
    if (precond) {
      const int want = slot == Bb - 1;
      k_final_alpha<<<Ng, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng, s->part, rz, alpha);
      k_cg_update<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, alpha, x, r, p, q, mix, s->part, want);
      if (want) k_final_res<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng + 1, Ng, s->part, res);
      k_bjacobi32<<<kRedBlocks, bj_threads, bj_smem, s->stream>>>((int)s->ne, N, Ng, s->lpBinv, r, z, s->part);
      if (mg) mg_apply_f64(s, r, z, mgpart);
      k_final_beta<<<Ng, kRedThreads, 0, s->stream>>>(nrz, Ng, s->part, rz, beta);
      k_cg_dir<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, beta, z, p);
      if (want) cudaMemcpyAsync(s->hostbuf + slot, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
      return STDG_OK;
    }
    k_final<<<Ng, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng, s->part, pq);
    k_cg_alpha<<<1, 32, 0, s->stream>>>(Ng, rz, pq, alpha);
    k_cg_update<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, alpha, x, r, p, q, mix, s->part);
    k_final<<<Ng + 1, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng + 1, s->part, rrnew);
    k_cg_beta2<<<1, 32, 0, s->stream>>>(Ng, rz, rrnew, beta, res, rrnew + Ng);
    k_cg_dir<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, beta, r, p);
    cudaMemcpyAsync(s->hostbuf + slot, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    return STDG_OK;
  };
  const int kpi = precond ? 7 + mg_launches(s) : 8;
  int it = 0;
  double rabs = INFINITY;
  const int maxit = s->opt.max_iters;
  if (s->opt.graph_batch > 1) {
    const int kind = df_serves(s, op) ? 1 : 0;
    stdg_status e = run_batched(s, s->opt.graph_batch, kpi, maxit, tol_abs, body, &it, &rabs, kind, precond);
    if (e != STDG_OK) return e;
  } else {
    while (it < maxit) {
      stdg_status e = body(0, nullptr);
      if (e != STDG_OK) return e;
      s->nlaunch += kpi;
      ++it;
      if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("CG: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
      rabs = s->hostbuf[0];
      if (!std::isfinite(rabs)) { set_error("CG: non-finite residual"); return STDG_ENAN; }
      if (s->snap_every > 0 && it % s->snap_every == 0 && s->nsnap < s->snap_cap && rabs > tol_abs)
        cudaMemcpyAsync(s->snaps + (size_t)(s->nsnap++) * n, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
      if (rabs <= tol_abs) break;
    }
  }
  *iters = it;
  *res_abs = rabs;
  if (rabs > tol_abs) { set_error("CG reached max_iters (%d)", it); return STDG_ENOCONV; }
  return STDG_OK;
}

// Restarted GMRES(m), classical Gram-Schmidt applied twice, Givens rotations on the host.
// x holds the initial guess unless zero_x0.  Stops when ||b - A x|| <= tol_abs.
// Restarted GMRES(m).  With pc_nu >= 0 it is right-preconditioned by the viscous block Jacobi of
// viscpc.cu (viscosity pc_nu): Arnoldi on A D^-1, x += D^-1 V y at the end of each cycle; the
// residual it monitors and returns is still that of A x = b.
static stdg_status gmres(stdg_solver* s, const ApplyArgs& op, const double* b, double* x, bool zero_x0,
                         double tol_abs, int* iters, int* nrestarts, double* res_abs, int restart = 0,
                         double pc_nu = -1.0) {
  const int m = restart > 0 ? restart : s->opt.restart;
  const int64_t n = s->ne * (int64_t)s->Nst;
  const bool pc = pc_nu >= 0.0;
  stdg_status e = ensure_basis(s, m + 1);
  if (e == STDG_OK && pc) e = visc_pc_ensure(s);
  if (e != STDG_OK) return e;
  if (zero_x0) cudaMemsetAsync(x, 0, n * sizeof(double), s->stream);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  double* hd = s->scal + 100;     // h (pass 1) at [0..m], h (pass 2) at [128..], norm^2 at [256]
  int it = 0, restarts = 0;
  double beta = INFINITY;
  const int maxit = s->opt.max_iters;
  while (true) {
    e = op_apply(s, op, x, s->kq);
    if (e != STDG_OK) return e;
    ++s->nlaunch;
    k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, b, nullptr, 1, s->kq);
    beta = host_norm(s, s->kq, n);
    if (!std::isfinite(beta)) { set_error("GMRES: non-finite residual"); return STDG_ENAN; }
    if (beta <= tol_abs || it >= maxit) break;
    s->hostbuf[901] = beta * beta;
    cudaMemcpyAsync(s->scal + 901, s->hostbuf + 901, sizeof(double), cudaMemcpyHostToDevice, s->stream);
    ++s->nlaunch;
    k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, s->kq, s->scal + 901, 0, s->basis);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (k = 0; k < m; ++k) {
      double* w = s->basis + (size_t)(k + 1) * n;
      if (pc) {
        if ((e = visc_pc_apply(s, pc_nu, s->basis + (size_t)k * n, s->kz, 0)) != STDG_OK) return e;
        e = op_apply(s, op, s->kz, w);
      } else {
        e = op_apply(s, op, s->basis + (size_t)k * n, w);
      }
      if (e != STDG_OK) return e;
      // classical Gram-Schmidt, second pass only when the first cancelled (gate at hd[260])
      k_sumsq<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, w, s->part);
      k_final<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, 1, s->part, hd + 258);
      for (int pass = 0; pass < 2; ++pass) {
        double* hp = hd + pass * 128;
        const double* gate = pass == 0 ? nullptr : hd + 260;
        if (pass == 1) k_reorth_gate<<<1, 32, 0, s->stream>>>(k + 1, hd, hd + 258, hd + 260);
        k_multidot<<<dim3(kRedBlocks, k + 1), kRedThreads, 0, s->stream>>>(n, s->basis, w, s->part, gate);
        k_final<<<k + 1, kRedThreads, 0, s->stream>>>(kRedBlocks, k + 1, s->part, hp, gate);
        k_multiaxpy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, k + 1, s->basis, hp, -1.0, w, gate);
      }
      s->nlaunch += 9;
      ++s->nlaunch;
      k_sumsq<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, w, s->part);
      ++s->nlaunch;
      k_final<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, 1, s->part, hd + 256);
      ++s->nlaunch;
      k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, w, hd + 256, 0, w);
      cudaMemcpyAsync(s->hostbuf, hd, 257 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
      if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("GMRES: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
      for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = s->hostbuf[i] + s->hostbuf[128 + i];
      H[(size_t)(k + 1) * m + k] = std::sqrt(s->hostbuf[256]);
      for (int i = 0; i < k; ++i) {
        double t1 = cs[i] * H[(size_t)i * m + k] + sn[i] * H[(size_t)(i + 1) * m + k];
        H[(size_t)(i + 1) * m + k] = -sn[i] * H[(size_t)i * m + k] + cs[i] * H[(size_t)(i + 1) * m + k];
        H[(size_t)i * m + k] = t1;
      }
      double den = std::hypot(H[(size_t)k * m + k], H[(size_t)(k + 1) * m + k]);
      cs[k] = H[(size_t)k * m + k] / den;
      sn[k] = H[(size_t)(k + 1) * m + k] / den;
      H[(size_t)k * m + k] = den;
      H[(size_t)(k + 1) * m + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      ++it;
      if (!std::isfinite(g[k + 1])) { set_error("GMRES: non-finite residual estimate"); return STDG_ENAN; }
      if (std::fabs(g[k + 1]) <= tol_abs || it >= maxit) { ++k; break; }
    }
    if (k > m) k = m;
    for (int i = k - 1; i >= 0; --i) {
      double sum = g[i];
      for (int jj = i + 1; jj < k; ++jj) sum -= H[(size_t)i * m + jj] * y[jj];
      y[i] = sum / H[(size_t)i * m + i];
    }
    std::memcpy(s->hostbuf, y.data(), k * sizeof(double));
    cudaMemcpyAsync(hd, s->hostbuf, k * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    ++s->nlaunch;
    if (pc) {
      cudaMemsetAsync(s->kp, 0, n * sizeof(double), s->stream);
      k_multiaxpy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, k, s->basis, hd, 1.0, s->kp);
      if ((e = visc_pc_apply(s, pc_nu, s->kp, x, 1)) != STDG_OK) return e;
    } else {
      k_multiaxpy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, k, s->basis, hd, 1.0, x);
    }
    ++restarts;
  }
  *iters = it; *nrestarts = restarts; *res_abs = beta;
  if (beta > tol_abs) { set_error("GMRES reached max_iters (%d)", it); return STDG_ENOCONV; }
  return STDG_OK;
}

// Flexible GMRES(m) with a right preconditioner z_j = M_j(v_j) that may change between iterations:
// x = x0 + Z y minimises ||b - A x|| over span(Z).  M_j is block Jacobi.  With use_gnn every cycle
// gets one more direction after the m block-Jacobi ones: block Jacobi plus the learned correction,
// applied to v_0, the normalised true residual of the cycle (the input the network was trained on,
// pairs of residuals and errors; later Arnoldi vectors are not residuals of any iterate).  The
// cycle's search space then contains the block-Jacobi cycle's, so its residual is never larger
// than that cycle's would be from the same start, whatever the network returns.
static stdg_status fgmres(stdg_solver* s, const ApplyArgs& op, const double* b, double* x, bool zero_x0,
                          double tol_abs, int* iters, int* nrestarts, double* res_abs, int use_gnn, bool visc = false) {
  TpArg Kinv{};
  for (int c = 0; c < s->Ng * s->Ng; ++c) Kinv.v[c] = s->Kinv[c];
  const int m0 = s->opt.restart;
  const int m = m0 + (use_gnn ? 1 : 0);            // directions per cycle
  const int64_t n = s->ne * (int64_t)s->Nst;
  stdg_status e = ensure_basis(s, m + 1);
  if (e != STDG_OK) return e;
  if (!s->kzz && (e = dev_alloc(s, (void**)&s->kzz, (size_t)(m0 + 1) * n * sizeof(double))) != STDG_OK) return e;
  if (zero_x0) cudaMemsetAsync(x, 0, n * sizeof(double), s->stream);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  double* hd = s->scal + 100;     // h (pass 1) at [0..m], h (pass 2) at [128..], norm^2 at [256]
  int it = 0, restarts = 0;
  double beta = INFINITY;
  const int maxit = s->opt.max_iters;
  while (true) {
    e = op_apply(s, op, x, s->kq);
    if (e != STDG_OK) return e;
    ++s->nlaunch;
    k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, b, nullptr, 1, s->kq);
    beta = host_norm(s, s->kq, n);
    if (!std::isfinite(beta)) { set_error("GMRES: non-finite residual"); return STDG_ENAN; }
    if (beta <= tol_abs || it >= maxit) break;
    s->hostbuf[901] = beta * beta;
    cudaMemcpyAsync(s->scal + 901, s->hostbuf + 901, sizeof(double), cudaMemcpyHostToDevice, s->stream);
    ++s->nlaunch;
    k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, s->kq, s->scal + 901, 0, s->basis);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (k = 0; k < m; ++k) {
      double* w = s->basis + (size_t)(k + 1) * n;
      double* zk = s->kzz + (size_t)k * n;
      if (visc) {                                 // viscous systems: inverse of the mass part
        k_visc_mass_inv<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, s->N, s->Ng, Kinv, op.mass_coef, op.detJ,
                                                                    s->basis + (size_t)k * n, zk, nullptr);
        ++s->nlaunch;
        e = STDG_OK;
      } else {
        e = k < m0 ? gnn_precond(s, s->basis + (size_t)k * n, zk, 0) : gnn_precond(s, s->basis, zk, 1);
      }
      if (e != STDG_OK) return e;
      e = op_apply(s, op, zk, w);
      if (e != STDG_OK) return e;
      // classical Gram-Schmidt, second pass only when the first cancelled (gate at hd[260])
      k_sumsq<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, w, s->part);
      k_final<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, 1, s->part, hd + 258);
      for (int pass = 0; pass < 2; ++pass) {
        double* hp = hd + pass * 128;
        const double* gate = pass == 0 ? nullptr : hd + 260;
        if (pass == 1) k_reorth_gate<<<1, 32, 0, s->stream>>>(k + 1, hd, hd + 258, hd + 260);
        k_multidot<<<dim3(kRedBlocks, k + 1), kRedThreads, 0, s->stream>>>(n, s->basis, w, s->part, gate);
        k_final<<<k + 1, kRedThreads, 0, s->stream>>>(kRedBlocks, k + 1, s->part, hp, gate);
        k_multiaxpy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, k + 1, s->basis, hp, -1.0, w, gate);
      }
      s->nlaunch += 9;
      ++s->nlaunch;
      k_sumsq<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, w, s->part);
      ++s->nlaunch;
      k_final<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, 1, s->part, hd + 256);
      ++s->nlaunch;
      k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, w, hd + 256, 0, w);
      cudaMemcpyAsync(s->hostbuf, hd, 257 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
      if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("GMRES: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
      for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = s->hostbuf[i] + s->hostbuf[128 + i];
      H[(size_t)(k + 1) * m + k] = std::sqrt(s->hostbuf[256]);
      for (int i = 0; i < k; ++i) {
        double t1 = cs[i] * H[(size_t)i * m + k] + sn[i] * H[(size_t)(i + 1) * m + k];
        H[(size_t)(i + 1) * m + k] = -sn[i] * H[(size_t)i * m + k] + cs[i] * H[(size_t)(i + 1) * m + k];
        H[(size_t)i * m + k] = t1;
      }
      double den = std::hypot(H[(size_t)k * m + k], H[(size_t)(k + 1) * m + k]);
      cs[k] = H[(size_t)k * m + k] / den;
      sn[k] = H[(size_t)(k + 1) * m + k] / den;
      H[(size_t)k * m + k] = den;
      H[(size_t)(k + 1) * m + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      ++it;
      if (!std::isfinite(g[k + 1])) { set_error("GMRES: non-finite residual estimate"); return STDG_ENAN; }
      if (std::fabs(g[k + 1]) <= tol_abs || it >= maxit) { ++k; break; }
    }
    if (k > m) k = m;
    for (int i = k - 1; i >= 0; --i) {
      double sum = g[i];
      for (int jj = i + 1; jj < k; ++jj) sum -= H[(size_t)i * m + jj] * y[jj];
      y[i] = sum / H[(size_t)i * m + i];
    }
    std::memcpy(s->hostbuf, y.data(), k * sizeof(double));
    cudaMemcpyAsync(hd, s->hostbuf, k * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    ++s->nlaunch;
    k_multiaxpy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, k, s->kzz, hd, 1.0, x);
    ++restarts;
  }
  *iters = it; *nrestarts = restarts; *res_abs = beta;
  if (beta > tol_abs) { set_error("FGMRES reached max_iters (%d)", it); return STDG_ENOCONV; }
  return STDG_OK;
}

static stdg_status ensure_lowprec(stdg_solver* s) {
  if (s->fr) return STDG_OK;
  stdg_status e = ensure_block_inverse(s);
  if (e != STDG_OK) return e;
  if (!s->lpB && !s->wB) {
    cudaError_t ce;
    if (s->op_warp) { s->lpkind = s->opt.precision; ce = warp_prepare(s, s->opt.precision); }
    else ce = lp_build_blocks(s, s->opt.precision);
    s->nlaunch += 2;
    if (ce != cudaSuccess) { set_error("low-precision block copies failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  }
  const size_t n = (size_t)s->ne * s->Nst;
  for (float** v : {&s->fr, &s->fp, &s->fq, &s->fz, &s->fx, &s->fb})
    if ((e = dev_alloc(s, (void**)v, n * sizeof(float))) != STDG_OK) return e;
  if ((e = dev_alloc(s, (void**)&s->dmix, kMaxNg * kMaxNg * sizeof(double))) != STDG_OK) return e;
  cudaMemcpyAsync(s->dmix, s->K.data(), s->Ng * s->Ng * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("low-precision setup failed"); return STDG_ECUDA; }
  return STDG_OK;
}

// Mixed precision, inner-outer.  Outer: flexible CG in binary64 on the Kronecker-decoupled system
// S X = B' (S = -A_sp (x) I with the pin, B' = -(I (x) Tp^-1) b), operator applied by the
// binary64-accurate pair kernel; each new direction is S-orthogonalised against the last m
// directions (flexible CG, Notay 2000), and x, r and all scalars are binary64, so the binary32 parts
// change how fast it converges, not the accuracy it reaches.  Preconditioner: a fixed number of
// block-Jacobi CG iterations in binary32 (binary32 or bfloat16 operator, binary32 vectors) started
// from zero on S d = r / ||r||, captured once per solve as a CUDA graph: s->mix_inner of them, or,
// with mg, s->mix_inner_mg with block Jacobi plus the agglomeration coarse correction of mg.cu.
// Stops when ||(I (x) Tp) r|| (the full-system residual) <= tol ||b||.
static stdg_status solve_mixed(stdg_solver* s, const double* b, double* x, double tol, double bn, int* iters,
                               int* outer, double* res_abs, bool mg, bool gnn = false, int* gnn_bad_steps = nullptr) {
  stdg_status e = ensure_lowprec(s);
  if (e == STDG_OK && mg) e = mg_ensure(s);
  if (e != STDG_OK) return e;
  const int nrz = kLpBlocksK + (mg ? mg_partial_blocks() : 0);   // r.z partial rows: block Jacobi, coarse
  const int mgl = mg ? mg_launches(s) : 0;
  const int N = s->N, Ng = s->Ng, m = s->mix_m;
  const int64_t n = s->ne * (int64_t)s->Nst;
  if (!s->fcgP && (e = dev_alloc(s, (void**)&s->fcgP, (size_t)m * n * sizeof(double))) != STDG_OK) return e;
  if (!s->fcgQ && (e = dev_alloc(s, (void**)&s->fcgQ, (size_t)m * n * sizeof(double))) != STDG_OK) return e;
  LpKernels lk = lp_kernels();
  double Tpd[kMaxNg * kMaxNg];
  TpArg Tp{}, Tpinv{};
  const double idt2 = 1.0 / (s->dt * s->dt);
  for (int c = 0; c < Ng * Ng; ++c) { Tpd[c] = Tp.v[c] = s->tm.Tp[c]; Tpinv.v[c] = s->tm.K[c] * idt2; }
  // inner (binary32) scalars
  double* rz = s->scal; double* pq = s->scal + 8; double* alpha = s->scal + 16; double* beta = s->scal + 24;
  double* rrnew = s->scal + 32; double* res = s->scal + 48; double* rznew = s->scal + 56;
  double* flag = s->scal + 96;                            // breakdown of the binary32 recurrence
  // outer (binary64) scalars: m x Ng dots z.Q_j, P_j.Q_j, coefficients; Ng-wide rest
  double* o_rp = s->scal + 400; double* o_al = s->scal + 408; double* o_rr = s->scal + 416;
  double* o_zq = s->scal + 500; double* o_pqs = s->scal + 600; double* o_c = s->scal + 700;   // m * Ng <= 80 each
  double* r = s->kr; double* z = s->kz; double* rhs = s->kb;
  const ApplyArgs S = pressure_op(s, 1, 1, -1.0, 1.0);
  ++s->nlaunch;
  k_timemix<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, Tpinv, -1.0, b, rhs);
  cudaMemsetAsync(x, 0, n * sizeof(double), s->stream);
  cudaMemcpyAsync(r, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
  double rdec = host_norm(s, r, n);                       // ||r|| of the decoupled system
  const int npq = warp_blocks_lp(s);
  if (npq <= 0) { set_error("binary32 operator not prepared"); return STDG_ECUDA; }
  if (!s->opdot && (e = dev_alloc(s, (void**)&s->opdot, (size_t)npq * kMaxNg * sizeof(double))) != STDG_OK) return e;
  auto body = [&](int slot, cudaEvent_t* evs) -> stdg_status {
    (void)slot;
    if (evs) cudaEventRecordWithFlags(evs[0], s->stream, cudaEventRecordExternal);
    // the operator also writes per-block p.q partials, reduced with the step length in one launch
    cudaError_t ce = launch_apply_lp(s, s->fp, s->fq, 1, 1, -1.0f, 1.0f, s->opdot);
    if (evs) cudaEventRecordWithFlags(evs[1], s->stream, cudaEventRecordExternal);
    if (ce != cudaSuccess) { set_error("low-precision operator launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
    k_final_alpha_guard<<<1, kRedThreads, 0, s->stream>>>(npq, Ng, s->opdot, rz, alpha, flag);
    lp_update_bjacobi(s->stream, (int)s->ne, N, Ng, alpha, s->fx, s->fr, s->fp, s->fq, s->lpBinv, s->fz, s->part);
    if (mg) mg_apply_f32(s, s->fr, s->fz, s->part + (size_t)kLpBlocksK * Ng);
    k_final_beta<<<Ng, kRedThreads, 0, s->stream>>>(nrz, Ng, s->part, rz, beta);
    lk.dir(s->stream, n, N, Ng, beta, s->fz, s->fp);
    return STDG_OK;
  };
  const int kin = mg ? s->mix_inner_mg : s->mix_inner;
  GraphLoop inner;
  const bool use_graph = s->opt.graph_batch > 1;
  if (use_graph && (e = graph_capture(s, kin, body, inner)) != STDG_OK) return e;
  int total = 0, it = 0, ring = 0, refresh = 0, harvested = 0;
  int* gnn_flag = reinterpret_cast<int*>(s->scal + 990);   // non-finite network output in this step
  double rfull = bn;
  bool net_step = false;                                   // with gnn: inner-solve and network steps alternate
  while (total < s->opt.max_iters && it < 100000) {
    if (net_step) {
      // ---- the network's direction: z = RMS(r) net(r / RMS(r)), the flexible step along it is the
      // energy-optimal correction in the enlarged search space; skipped (and counted) when the
      // output is not finite or vanishes
      net_step = false;
      cudaMemsetAsync(z, 0, n * sizeof(double), s->stream);
      cudaMemsetAsync(gnn_flag, 0, sizeof(int), s->stream);
      if ((e = gnn_correct(s, r, z, gnn_flag)) != STDG_OK) return e;
      cudaMemcpyAsync(s->hostbuf + 990, gnn_flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
      const double zn = host_norm(s, z, n);               // synchronises the stream
      if (*reinterpret_cast<const int*>(s->hostbuf + 990) != 0 || !(zn > 0.0) || !std::isfinite(zn)) {
        if (gnn_bad_steps) ++*gnn_bad_steps;
        continue;
      }
    } else {
    net_step = gnn;
    // harvested pairs (r_k, x* - x_k) at the start of every inner-solve step after the first
    if (it > 0 && gnn_mg_harvest_room(s, harvested)) { gnn_mg_harvest_snap(s, harvested, r, x, nullptr); ++harvested; }
    // ---- preconditioner: kin binary32 block-Jacobi CG iterations on S d = r / ||r||, d0 = 0
    lk.f32s(s->stream, n, 1.0 / rdec, r, s->fr);
    cudaMemsetAsync(s->fx, 0, n * sizeof(float), s->stream);
    cudaMemsetAsync(flag, 0, sizeof(double), s->stream);
    lk.bjacobi(s->stream, (int)s->ne, N, Ng, s->lpBinv, s->fr, s->fz, s->part);
    if (mg) mg_apply_f32(s, s->fr, s->fz, s->part + (size_t)kLpBlocksK * Ng);
    k_final<<<Ng, kRedThreads, 0, s->stream>>>(nrz, Ng, s->part, rz);
    cudaMemcpyAsync(s->fp, s->fz, n * sizeof(float), cudaMemcpyDeviceToDevice, s->stream);
    s->nlaunch += 3 + mgl;
    if (use_graph) {
      if ((e = graph_launch(s, inner, 5 + mgl, s->lpkind == STDG_PREC_MIXED_BF16 ? 3 : 2)) != STDG_OK) return e;
    } else {
      for (int j = 0; j < kin; ++j) {
        if ((e = body(j, nullptr)) != STDG_OK) return e;
        s->nlaunch += 5 + mgl; ++s->op_launches;
      }
    }
    total += kin;
    // z = ||r|| d in binary64
    cudaMemsetAsync(z, 0, n * sizeof(double), s->stream);
    lk.accum(s->stream, n, rdec, s->fx, z);
    }
    // ---- flexible CG step: p = z - Sum_j (z.Q_j / P_j.Q_j) P_j over the stored directions
    const int slot = ring % m, used = ring < m ? ring : m;
    double* p = s->fcgP + (size_t)slot * n;
    double* q = s->fcgQ + (size_t)slot * n;
    if (used == 0) {
      cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    } else {
      k_fcg_dots<<<dim3(kRedBlocks, used), kRedThreads, 0, s->stream>>>(n, N, Ng, used, s->fcgQ, z, s->part);
      k_final<<<used * Ng, kRedThreads, 0, s->stream>>>(kRedBlocks, used * Ng, s->part, o_zq);
      k_fcg_coef<<<1, 64, 0, s->stream>>>(used * Ng, o_zq, o_pqs, o_c);
      // the slot being overwritten is excluded: when the ring is full its coefficient is set to 0
      if (used == m) cudaMemsetAsync(o_c + slot * Ng, 0, Ng * sizeof(double), s->stream);
      k_fcg_dir<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, used, o_c, s->fcgP, z, s->kp);
      cudaMemcpyAsync(p, s->kp, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
      s->nlaunch += 4;
    }
    e = op_apply(s, S, p, q);
    if (e != STDG_OK) return e;
    k_coldot<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, p, q, s->part);
    k_final<<<Ng, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng, s->part, o_pqs + slot * Ng);
    k_coldot<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, r, p, s->part);
    k_final<<<Ng, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng, s->part, o_rp);
    k_cg_alpha<<<1, 32, 0, s->stream>>>(Ng, o_rp, o_pqs + slot * Ng, o_al);
    k_cg_update<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, o_al, x, r, p, q, Tp, s->part);
    k_final<<<Ng + 1, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng + 1, s->part, o_rr);
    cudaMemcpyAsync(s->hostbuf + 880, o_rr, (Ng + 1) * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    s->nlaunch += 9;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("mixed solve: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
    ++it; ++ring;
    double rr = 0.0;
    for (int a = 0; a < Ng; ++a) rr += s->hostbuf[880 + a];
    rdec = std::sqrt(rr);
    rfull = std::sqrt(s->hostbuf[880 + Ng]);
    if (!std::isfinite(rfull)) { set_error("mixed solve: non-finite residual"); return STDG_ENAN; }
    if (rfull <= tol * bn || rdec == 0.0) {
      // the recurrence says converged: evaluate b - A x with the binary64 kernel (the pair kernel's
      // rounding, ~1e-14 of |A| |x|, can exceed tol |b|); if it misses the tolerance, continue from
      // that residual with a fresh set of directions (at most 3 times)
      if ((e = op_apply(s, pressure_op(s, 1, 0, 1.0, -1.0), x, s->kq, true)) != STDG_OK) return e;
      k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, b, nullptr, 1, s->kq);   // kq = b - A x
      ++s->nlaunch;
      rfull = host_norm(s, s->kq, n);
      if (rfull <= tol * bn || rdec == 0.0 || refresh >= 3) break;
      ++refresh;
      k_timemix<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, Tpinv, -1.0, s->kq, r);   // r = -(I (x) Tp^-1)(b - A x)
      ++s->nlaunch;
      rdec = host_norm(s, r, n);
      ring = 0;
    }
  }
  if (harvested > 0) gnn_mg_harvest_finish(s, harvested, x);
  int herr = 0;
  cudaMemcpy(&herr, s->derr, sizeof(int), cudaMemcpyDeviceToHost);
  if (herr) { set_error("low-precision operator: a bounded wait timed out"); return STDG_ETIMEOUT; }
  *iters = total;
  *outer = it;
  *res_abs = rfull;
  if (rfull > tol * bn) { set_error("mixed solve did not reach the tolerance (%d inner, %d outer iterations)", total, it); return STDG_ENOCONV; }
  return STDG_OK;
}

stdg_status solve_pressure(stdg_solver* s, const double* b, double* x, double tol, int method,
                           stdg_solve_stats* st) {
  stdg_status e = ensure_krylov(s);
  if (e != STDG_OK) return e;
  auto t0 = std::chrono::steady_clock::now();
  if (method == STDG_SOLVER_CG && s->pt != 0) {
    set_error("STDG_SOLVER_CG needs p_t = 0 (the system is nonsymmetric otherwise)");
    return STDG_EINVAL;
  }
  const int64_t n = s->ne * (int64_t)s->Nst;
  const double bn = host_norm(s, b, n);
  if (!std::isfinite(bn)) { set_error("stdg_solve: non-finite right-hand side"); return STDG_ENAN; }
  int it = 0, rs = 0;
  double rabs = 0.0;
  stdg_status r = STDG_OK;
  if (st) st->fallback = 0;
  if (bn == 0.0) {
    cudaMemsetAsync(x, 0, n * sizeof(double), s->stream);
  } else if (method == STDG_SOLVER_GMRES) {
    r = gmres(s, pressure_op(s, 1, 0, 1.0, -1.0), b, x, true, tol * bn, &it, &rs, &rabs);
  } else if (method == STDG_SOLVER_FGMRES_BJ || method == STDG_SOLVER_FGMRES_GNN) {
    r = ensure_block_inverse(s);
    if (r == STDG_OK && !s->gnn) { set_error("FGMRES with block Jacobi / learned preconditioner needs stdg_gnn_init"); r = STDG_EINVAL; }
    if (r == STDG_OK)
      r = fgmres(s, pressure_op(s, 1, 0, 1.0, -1.0), b, x, true, tol * bn, &it, &rs, &rabs,
                 method == STDG_SOLVER_FGMRES_GNN ? 1 : 0);
    if (method == STDG_SOLVER_FGMRES_GNN && (r == STDG_ENOCONV || r == STDG_ENAN)) {
      // the learned preconditioner failed: plain GMRES (the paper's solver) produces the result
      std::string why = last_error();
      int it2 = 0, rs2 = 0;
      r = gmres(s, pressure_op(s, 1, 0, 1.0, -1.0), b, x, true, tol * bn, &it2, &rs2, &rabs);
      if (r != STDG_OK) {
        std::string after = last_error();
        set_error("learned FGMRES failed (%s after %d iterations); plain GMRES fallback: %s", why.c_str(), it,
                  after.c_str());
      }
      it += it2; rs += rs2;
      if (st) st->fallback = 1;
    }
  } else if (method == STDG_SOLVER_KRON_MG_GNN) {
    if (s->opt.precision != STDG_PREC_MIXED_F32 && s->opt.precision != STDG_PREC_MIXED_BF16) {
      set_error("STDG_SOLVER_KRON_MG_GNN needs a mixed precision option"); return STDG_EINVAL;
    }
    if (!s->gnn) { set_error("STDG_SOLVER_KRON_MG_GNN needs stdg_gnn_init"); return STDG_EINVAL; }
    int bad = 0;
    r = solve_mixed(s, b, x, tol, bn, &it, &rs, &rabs, true, true, &bad);
    if (st) st->fallback = bad;
  } else if ((method == STDG_SOLVER_KRON_CG || method == STDG_SOLVER_KRON_PCG || method == STDG_SOLVER_KRON_MG) &&
             (s->opt.precision == STDG_PREC_MIXED_F32 || s->opt.precision == STDG_PREC_MIXED_BF16)) {
    r = solve_mixed(s, b, x, tol, bn, &it, &rs, &rabs, method == STDG_SOLVER_KRON_MG);
  } else if (method == STDG_SOLVER_CG || method == STDG_SOLVER_KRON_CG || method == STDG_SOLVER_KRON_PCG ||
             method == STDG_SOLVER_KRON_MG) {
    // A = A_sp (x) Tp (pinned):  A x = b  <=>  (-A_sp (x) I) x = -(I (x) Tp^-1) b,  Tp^-1 = K / dt^2;
    // the full residual is b - A x = -(I (x) Tp) r for the CG residual r.
    TpArg Tp{}, Tpinv{};
    const double idt2 = 1.0 / (s->dt * s->dt);
    for (int q = 0; q < s->Ng * s->Ng; ++q) { Tp.v[q] = s->tm.Tp[q]; Tpinv.v[q] = s->tm.K[q] * idt2; }
    ++s->nlaunch;
    k_timemix<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, s->N, s->Ng, Tpinv, -1.0, b, s->kb);
    r = cg_block(s, pressure_op(s, 1, 1, -1.0, 1.0), s->kb, x, true, Tp, tol * bn, &it, &rabs,
                 method == STDG_SOLVER_KRON_PCG ? 1 : method == STDG_SOLVER_KRON_MG ? 2 : 0);
  } else {
    set_error("unknown solver method %d", method);
    return STDG_EINVAL;
  }
  if (r != STDG_OK && r != STDG_ENOCONV) return r;
  if (st) {
    // report the residual of the full pinned system for every method, evaluated with the binary64
    // kernel (the mixed solves have just done so for their final x)
    const bool mixed_done = r == STDG_OK && bn > 0.0 &&
        (method == STDG_SOLVER_KRON_MG_GNN || ((method == STDG_SOLVER_KRON_CG || method == STDG_SOLVER_KRON_PCG ||
          method == STDG_SOLVER_KRON_MG) && (s->opt.precision == STDG_PREC_MIXED_F32 || s->opt.precision == STDG_PREC_MIXED_BF16)));
    double rn = rabs;
    if (!mixed_done && bn > 0.0) {
      stdg_status e2 = op_apply(s, pressure_op(s, 1, 0, 1.0, -1.0), x, s->kq, true);
      if (e2 != STDG_OK) return e2;
      ++s->nlaunch;
      k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, b, nullptr, 1, s->kq);
      rn = host_norm(s, s->kq, n);
    }
    st->iterations = it;
    st->restarts = rs;
    st->rel_residual = bn > 0 ? rn / bn : 0.0;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return r;
}

// ---------------------------------------------------------------------------------------------
// Viscous systems decoupled in time.  The operator of Eq. A1_mod is D (x) K + c G (x) I with
// D = diag(|J_i|) (x) I_N, c = nu dt and G the symmetric positive definite spatial viscous operator
// (the orthonormal bases make every mass matrix diagonal).  With K = W R W^-1 (R real block
// diagonal: 2 x 2 blocks [[a, b], [-b, a]] for complex eigenvalue pairs, 1 x 1 for real ones) and
// x = (I (x) W) y the system becomes (D (x) R + c G (x) I) y = (I (x) W^-1) b: independent systems
// per block of R.  A 2 x 2 block is the complex symmetric system ((a - ib) D + c G) y = b~ on
// y_r + i y_i, a 1 x 1 block a symmetric positive definite one.  Both are solved by conjugate-
// orthogonal CG (COCG, van der Vorst & Melissen 1990: CG with the unconjugated bilinear form u^T v,
// which reduces to CG for real data), preconditioned by the exact inverse of every tet's diagonal
// block (viscpc.cu with K replaced by R).  All blocks share each operator launch (the viscous kernel
// with R as its time matrix); the complex scalars of every block are formed on the device from
// column cross products, so a batch of iterations is one CUDA graph with one host check.  The
// residual tested is that of the original system, ||(I (x) W) r_y||.

// all Ng x Ng column cross products C[a][b] = Sum u[a][k] v[b][k]: partials part[blk * Ng^2 + a Ng + b].
// NG at compile time: on sm_103a even predicated-off binary64 instructions cost FP64-pipe time.
template <int NG>
__global__ void __launch_bounds__(kRedThreads) k_crossdot(int ne, int N, const double* __restrict__ u,
                                                         const double* __restrict__ v, double* part) {
  double acc[NG * NG];
#pragma unroll
  for (int c = 0; c < NG * NG; ++c) acc[c] = 0.0;
  const int Nst = N * NG, total = ne * N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / N;
    const size_t o = (size_t)i * Nst + (e - i * N);
    double uu[NG], vv[NG];
#pragma unroll
    for (int a = 0; a < NG; ++a) { uu[a] = u[o + a * N]; vv[a] = v[o + a * N]; }
#pragma unroll
    for (int a = 0; a < NG; ++a)
#pragma unroll
      for (int b = 0; b < NG; ++b) acc[a * NG + b] = fma(uu[a], vv[b], acc[a * NG + b]);
  }
  __shared__ double red[NG * NG][kRedThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NG * NG; ++c) {
    const double t = warp_sum(acc[c]);
    if (lane == 0) red[c][w] = t;
  }
  __syncthreads();
  if (threadIdx.x < NG * NG) {
    double t = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) t += red[threadIdx.x][k];
    part[(size_t)blockIdx.x * NG * NG + threadIdx.x] = t;
  }
}

struct PairArg { int p[kMaxNg]; };

// The complex scalars of every block of R, from the cross products C (Ng x Ng).  The bilinear form of
// a 2 x 2 block (columns a, a+1 = real, imaginary part) is (C_aa - C_a+1,a+1) + i (C_a,a+1 + C_a+1,a);
// of a 1 x 1 block C_aa.  rho[2a], rho[2a+1]: r^T z of the block led by column a.
//  mode 0: alpha = rho / (p^T q)  -> M (Ng x Ng real form of the multiplier), flag on breakdown
//  mode 1: beta = (r^T z)_new / rho, rho <- (r^T z)_new  -> M
//  mode 2: rho <- r^T z
__global__ void k_cocg_scalars(int Ng, PairArg pr, int mode, const double* __restrict__ C, double* rho, double* M,
                               double* flag) {
  if (threadIdx.x != 0) return;
  for (int q = 0; q < Ng * Ng; ++q) M[q] = 0.0;
  for (int a = 0; a < Ng; ++a) {
    const bool two = pr.p[a] == 1;
    double br, bi;
    if (two) { br = C[a * Ng + a] - C[(a + 1) * Ng + a + 1]; bi = C[a * Ng + a + 1] + C[(a + 1) * Ng + a]; }
    else { br = C[a * Ng + a]; bi = 0.0; }
    double zr = 0.0, zi = 0.0;
    if (mode == 2) { rho[2 * a] = br; rho[2 * a + 1] = bi; }
    else {
      // z = num / den (complex)
      const double nr = mode == 0 ? rho[2 * a] : br, ni = mode == 0 ? rho[2 * a + 1] : bi;
      const double dr = mode == 0 ? br : rho[2 * a], di = mode == 0 ? bi : rho[2 * a + 1];
      const double dd = dr * dr + di * di;
      if (dd > 0.0 && isfinite(dd)) { zr = (nr * dr + ni * di) / dd; zi = (ni * dr - nr * di) / dd; }
      else if (nr != 0.0 || ni != 0.0) flag[0] = 1.0;
      if (mode == 1) { rho[2 * a] = br; rho[2 * a + 1] = bi; }
    }
    M[a * Ng + a] = zr;
    if (two) {
      M[a * Ng + a + 1] = -zi; M[(a + 1) * Ng + a] = zi; M[(a + 1) * Ng + a + 1] = zr;
      ++a;
    }
  }
}

// x += M p, r -= M q (M from the device, Ng x Ng); with want, partials of ||(I (x) W) r||^2
template <int NG>
__global__ void __launch_bounds__(kRedThreads) k_cocg_update(int ne, int N, const double* __restrict__ Mdev,
                                                            double* __restrict__ x, double* __restrict__ r,
                                                            const double* __restrict__ p, const double* __restrict__ q,
                                                            TpArg W, double* part, int want) {
  __shared__ double Ms[NG * NG];
  if (threadIdx.x < NG * NG) Ms[threadIdx.x] = Mdev[threadIdx.x];
  __syncthreads();
  const int Nst = N * NG, total = ne * N;
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / N;
    const size_t o = (size_t)i * Nst + (e - i * N);
    double pp[NG], qq[NG], rn[NG];
#pragma unroll
    for (int a = 0; a < NG; ++a) { pp[a] = p[o + a * N]; qq[a] = q[o + a * N]; }
#pragma unroll
    for (int a = 0; a < NG; ++a) {
      double dx = 0.0, dr = 0.0;
#pragma unroll
      for (int b = 0; b < NG; ++b) { dx = fma(Ms[a * NG + b], pp[b], dx); dr = fma(Ms[a * NG + b], qq[b], dr); }
      x[o + a * N] += dx;
      rn[a] = r[o + a * N] - dr;
      r[o + a * N] = rn[a];
    }
    if (want) {
#pragma unroll
      for (int c = 0; c < NG; ++c) {
        double t = 0.0;
#pragma unroll
        for (int a = 0; a < NG; ++a) t = fma(W.v[c * NG + a], rn[a], t);
        acc = fma(t, t, acc);
      }
    }
  }
  if (want) block_reduce_store(&acc, 1, part, 1);
}

// p = z + M p
template <int NG>
__global__ void __launch_bounds__(kRedThreads) k_cocg_dir(int ne, int N, const double* __restrict__ Mdev,
                                                         const double* __restrict__ z, double* __restrict__ p) {
  __shared__ double Ms[NG * NG];
  if (threadIdx.x < NG * NG) Ms[threadIdx.x] = Mdev[threadIdx.x];
  __syncthreads();
  const int Nst = N * NG, total = ne * N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / N;
    const size_t o = (size_t)i * Nst + (e - i * N);
    double pp[NG];
#pragma unroll
    for (int a = 0; a < NG; ++a) pp[a] = p[o + a * N];
#pragma unroll
    for (int a = 0; a < NG; ++a) {
      double v = z[o + a * N];
#pragma unroll
      for (int b = 0; b < NG; ++b) v = fma(Ms[a * NG + b], pp[b], v);
      p[o + a * N] = v;
    }
  }
}

// launches of the three vector kernels above for the solver's Ng
struct CocgLaunch {
  int Ng;
  void cross(cudaStream_t st, int ne, int N, const double* u, const double* v, double* part) const {
    switch (Ng) {
      case 1: k_crossdot<1><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, u, v, part); break;
      case 2: k_crossdot<2><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, u, v, part); break;
      case 3: k_crossdot<3><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, u, v, part); break;
      case 4: k_crossdot<4><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, u, v, part); break;
      default: k_crossdot<5><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, u, v, part); break;
    }
  }
  void update(cudaStream_t st, int ne, int N, const double* M, double* x, double* r, const double* p, const double* q,
              const TpArg& W, double* part, int want) const {
    switch (Ng) {
      case 1: k_cocg_update<1><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, x, r, p, q, W, part, want); break;
      case 2: k_cocg_update<2><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, x, r, p, q, W, part, want); break;
      case 3: k_cocg_update<3><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, x, r, p, q, W, part, want); break;
      case 4: k_cocg_update<4><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, x, r, p, q, W, part, want); break;
      default: k_cocg_update<5><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, x, r, p, q, W, part, want); break;
    }
  }
  void dir(cudaStream_t st, int ne, int N, const double* M, const double* z, double* p) const {
    switch (Ng) {
      case 1: k_cocg_dir<1><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, z, p); break;
      case 2: k_cocg_dir<2><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, z, p); break;
      case 3: k_cocg_dir<3><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, z, p); break;
      case 4: k_cocg_dir<4><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, z, p); break;
      default: k_cocg_dir<5><<<kRedBlocks, kRedThreads, 0, st>>>(ne, N, M, z, p); break;
    }
  }
};

__global__ void k_final_norm(int nparts, const double* __restrict__ part, double* out) {
  __shared__ double red[kRedThreads / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) t += red[q];
    out[0] = sqrt(t);
  }
}

__global__ void k_f64_from_f32(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (double)in[e];
}
__global__ void k_add(int64_t n, const double* __restrict__ d, double* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] += d[e];
}

// COCG on the decoupled viscous systems; x holds the initial guess (zero_x0: x = 0) and receives the
// solution.  lowprec: the operator is applied with binary32 blocks (vectors converted around the
// launch), for the inner solves of the refinement in solve_viscous.  Returns STDG_EUNSUPPORTED when
// K has no usable block-diagonal form (the caller then uses GMRES), STDG_ENOCONV / STDG_ENAN as the
// other solvers.
static stdg_status cocg_viscous(stdg_solver* s, const ApplyArgs& a, double nu, const double* b, double* x,
                                double tol_abs, int* iters, double* res, bool zero_x0 = false,
                                bool lowprec = false) {
  const int Ng = s->Ng, N = s->N;
  const int64_t n = s->ne * (int64_t)s->Nst;
  if (s->vbd < 0) s->vbd = time_blockdiag(s->K.data(), Ng, s->vW, s->vWinv, s->vR, s->vpair) ? 1 : 0;
  if (!s->vbd) return STDG_EUNSUPPORTED;
  stdg_status e = visc_pc_ensure(s);
  if (e == STDG_OK && lowprec) e = ensure_lowprec(s);
  if (e != STDG_OK) return e;
  if (lowprec) {
    cudaError_t ce = warp_prepare_f32_visc(s);
    if (ce != cudaSuccess) { set_error("binary32 viscous blocks: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  }
  TpArg W{}, Wi{};
  PairArg pr{};
  for (int q = 0; q < Ng * Ng; ++q) { W.v[q] = s->vW[q]; Wi.v[q] = s->vWinv[q]; }
  for (int c = 0; c < Ng; ++c) pr.p[c] = s->vpair[c];
  ApplyArgs at = a;                                   // the decoupled operator: time matrix R
  for (int q = 0; q < Ng * Ng; ++q) at.Kmass[q] = s->vR[q];
  double* y = s->kx; double* r = s->kr; double* z = s->kz; double* p = s->kp; double* q = s->kq;
  double* bt = s->kb;
  double* C = s->scal + 300;                          // Ng^2 cross products
  double* rho = s->scal + 330;                        // 2 Ng
  double* Ma = s->scal + 340; double* Mb = s->scal + 370;   // Ng^2 each
  double* flag = s->scal + 398; double* resd = s->scal + 399;
  const int G2 = Ng * Ng;
  const LpKernels lk = lp_kernels();
  auto apply = [&](const double* in, double* out) -> stdg_status {
    if (!lowprec) return op_apply(s, at, in, out);
    lk.f32(s->stream, n, in, s->fp);
    const cudaError_t ce = warp_launch_f32_visc(s, s->fp, s->fq, at.scale, at.mass_coef, at.Kmass);
    if (ce != cudaSuccess) { set_error("binary32 viscous operator: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
    k_f64_from_f32<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, s->fq, out);
    s->nlaunch += 3;
    ++s->op_launches;
    return STDG_OK;
  };
  s->nlaunch += 1;
  k_timemix<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, Wi, 1.0, b, bt);
  if (zero_x0) {
    cudaMemsetAsync(y, 0, n * sizeof(double), s->stream);
    cudaMemcpyAsync(r, bt, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
  } else {
    s->nlaunch += 2;
    k_timemix<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, Wi, 1.0, x, y);
    if ((e = apply(y, r)) != STDG_OK) return e;
    k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, bt, nullptr, 1, r);
  }
  if ((e = visc_pc_apply(s, nu, r, z, 0, s->vR)) != STDG_OK) return e;
  cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
  cudaMemsetAsync(flag, 0, sizeof(double), s->stream);
  s->nlaunch += 3;
  const CocgLaunch cl{Ng};
  const int ne = (int)s->ne;
  cl.cross(s->stream, ne, N, r, z, s->part);
  k_final<<<G2, kRedThreads, 0, s->stream>>>(kRedBlocks, G2, s->part, C);
  k_cocg_scalars<<<1, 32, 0, s->stream>>>(Ng, pr, 2, C, rho, Ma, flag);
  // a few tens of iterations per solve: batches of at most 4 between host checks
  const int B = s->opt.graph_batch > 1 ? std::min(4, s->opt.graph_batch) : 1;
  auto body = [&](int slot, cudaEvent_t* evs) -> stdg_status {
    if (evs) cudaEventRecordWithFlags(evs[0], s->stream, cudaEventRecordExternal);
    stdg_status e2 = apply(p, q);
    if (evs) cudaEventRecordWithFlags(evs[1], s->stream, cudaEventRecordExternal);
    if (e2 != STDG_OK) return e2;
    const int want = slot == B - 1;
    cl.cross(s->stream, ne, N, p, q, s->part);
    k_final<<<G2, kRedThreads, 0, s->stream>>>(kRedBlocks, G2, s->part, C);
    k_cocg_scalars<<<1, 32, 0, s->stream>>>(Ng, pr, 0, C, rho, Ma, flag);
    cl.update(s->stream, ne, N, Ma, y, r, p, q, W, s->part, want);
    if (want) {
      k_final_norm<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, s->part, resd);
      cudaMemcpyAsync(s->hostbuf + slot, resd, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    }
    if ((e2 = visc_pc_apply(s, nu, r, z, 0, s->vR)) != STDG_OK) return e2;
    cl.cross(s->stream, ne, N, r, z, s->part);
    k_final<<<G2, kRedThreads, 0, s->stream>>>(kRedBlocks, G2, s->part, C);
    k_cocg_scalars<<<1, 32, 0, s->stream>>>(Ng, pr, 1, C, rho, Mb, flag);
    cl.dir(s->stream, ne, N, Mb, z, p);
    return STDG_OK;
  };
  int it = 0;
  double rabs = INFINITY;
  const int kind = lowprec ? 2 : df_serves(s, at) ? 1 : 0;
  const int kpi = 11 + (lowprec ? 2 : 0);
  if (B > 1) {
    e = run_batched(s, B, kpi, s->opt.max_iters, tol_abs, body, &it, &rabs, kind, true);
  } else {
    e = STDG_OK;
    while (it < s->opt.max_iters) {
      if ((e = body(0, nullptr)) != STDG_OK) break;
      s->nlaunch += kpi;
      ++it;
      if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("viscous COCG: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
      rabs = s->hostbuf[0];
      if (!std::isfinite(rabs)) { set_error("Krylov: non-finite residual"); e = STDG_ENAN; break; }
      if (rabs <= tol_abs) break;
    }
  }
  double hflag = 0.0;
  cudaMemcpyAsync(&hflag, flag, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  ++s->nlaunch;
  k_timemix<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, W, 1.0, y, x);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("viscous COCG: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
  *iters = it;
  *res = rabs;
  if (e != STDG_OK) return e;
  if (hflag != 0.0) { set_error("viscous COCG: breakdown (p^T A p = 0)"); return STDG_ENOCONV; }
  if (!(rabs <= tol_abs)) { set_error("viscous COCG reached max_iters (%d)", it); return STDG_ENOCONV; }
  return STDG_OK;
}

// Inner solve of the mixed-precision viscous refinement: x += A^-1 b to tol_abs (the decoupled
// residual norm), all vectors binary32 (the solver's binary32 work vectors, free between pressure
// solves), operator from the binary32 viscous blocks, multipliers and cross products restricted to
// the tridiagonal entries the block-diagonal time matrix R can couple (cocg32.cu).  b and x are
// binary64; x is left unchanged unless the solve reaches tol_abs.
static stdg_status cocg_viscous32(stdg_solver* s, const ApplyArgs& a, double nu, const double* b, double* x,
                                  double tol_abs, int* iters, double* res) {
  const int Ng = s->Ng, N = s->N, ne = (int)s->ne;
  const int64_t n = s->ne * (int64_t)s->Nst;
  if (s->vbd < 0) s->vbd = time_blockdiag(s->K.data(), Ng, s->vW, s->vWinv, s->vR, s->vpair) ? 1 : 0;
  if (!s->vbd) return STDG_EUNSUPPORTED;
  stdg_status e = visc_pc_ensure(s);
  if (e == STDG_OK) e = ensure_lowprec(s);
  if (e != STDG_OK) return e;
  cudaError_t ce = warp_prepare_f32_visc(s);
  if (ce != cudaSuccess) { set_error("binary32 viscous blocks: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  Mix32 W{}, Wi{};
  PairArg pr{};
  for (int q = 0; q < Ng * Ng; ++q) { W.v[q] = (float)s->vW[q]; Wi.v[q] = (float)s->vWinv[q]; }
  for (int c = 0; c < Ng; ++c) pr.p[c] = s->vpair[c];
  ApplyArgs at = a;                                   // the decoupled operator: time matrix R
  for (int q = 0; q < Ng * Ng; ++q) at.Kmass[q] = s->vR[q];
  float* y = s->fx; float* r = s->fr; float* z = s->fz; float* p = s->fp; float* q = s->fq;
  double* C = s->scal + 300;                          // Ng^2 cross products
  double* rho = s->scal + 330;                        // 2 Ng
  double* Ma = s->scal + 340; double* Mb = s->scal + 370;   // Ng^2 each
  double* flag = s->scal + 398; double* resd = s->scal + 399;
  const int G2 = Ng * Ng;
  c32_mix_to32(s->stream, ne, N, Ng, Wi, b, r);      // r = (I (x) W^-1) b, y = 0
  cudaMemsetAsync(y, 0, n * sizeof(float), s->stream);
  if ((e = visc_pc_apply32(s, nu, r, z, s->vR)) != STDG_OK) return e;
  cudaMemcpyAsync(p, z, n * sizeof(float), cudaMemcpyDeviceToDevice, s->stream);
  cudaMemsetAsync(flag, 0, sizeof(double), s->stream);
  c32_cross(s->stream, ne, N, Ng, r, z, s->part);
  k_final<<<G2, kRedThreads, 0, s->stream>>>(kRedBlocks, G2, s->part, C);
  k_cocg_scalars<<<1, 32, 0, s->stream>>>(Ng, pr, 2, C, rho, Ma, flag);
  s->nlaunch += 4;
  const int B = s->opt.graph_batch > 1 ? std::min(4, s->opt.graph_batch) : 1;
  auto body = [&](int slot, cudaEvent_t* evs) -> stdg_status {
    if (evs) cudaEventRecordWithFlags(evs[0], s->stream, cudaEventRecordExternal);
    const cudaError_t ae = warp_launch_f32_visc(s, p, q, at.scale, at.mass_coef, at.Kmass);
    if (evs) cudaEventRecordWithFlags(evs[1], s->stream, cudaEventRecordExternal);
    if (ae != cudaSuccess) { set_error("binary32 viscous operator: %s", cudaGetErrorString(ae)); return STDG_ECUDA; }
    const int want = slot == B - 1;
    c32_cross(s->stream, ne, N, Ng, p, q, s->part);
    k_final<<<G2, kRedThreads, 0, s->stream>>>(kRedBlocks, G2, s->part, C);
    k_cocg_scalars<<<1, 32, 0, s->stream>>>(Ng, pr, 0, C, rho, Ma, flag);
    c32_update(s->stream, ne, N, Ng, Ma, y, r, p, q, W, s->part, want);
    if (want) {
      k_final_norm<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, s->part, resd);
      cudaMemcpyAsync(s->hostbuf + slot, resd, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    }
    stdg_status e2 = visc_pc_apply32(s, nu, r, z, s->vR);
    if (e2 != STDG_OK) return e2;
    c32_cross(s->stream, ne, N, Ng, r, z, s->part);
    k_final<<<G2, kRedThreads, 0, s->stream>>>(kRedBlocks, G2, s->part, C);
    k_cocg_scalars<<<1, 32, 0, s->stream>>>(Ng, pr, 1, C, rho, Mb, flag);
    c32_dir(s->stream, ne, N, Ng, Mb, z, p);
    return STDG_OK;
  };
  int it = 0;
  double rabs = INFINITY;
  constexpr int kpi = 10;                             // kernels per iteration (+1 norm per check)
  if (B > 1) {
    e = run_batched(s, B, kpi, s->opt.max_iters, tol_abs, body, &it, &rabs, 2, true);
    s->nlaunch += it / B;
  } else {
    e = STDG_OK;
    while (it < s->opt.max_iters) {
      if ((e = body(0, nullptr)) != STDG_OK) break;
      s->nlaunch += kpi + 1;
      ++s->op_launches;
      ++it;
      if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("viscous COCG: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
      rabs = s->hostbuf[0];
      if (!std::isfinite(rabs)) { set_error("Krylov: non-finite residual"); e = STDG_ENAN; break; }
      if (rabs <= tol_abs) break;
    }
  }
  double hflag = 0.0;
  cudaMemcpyAsync(&hflag, flag, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("viscous COCG: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
  *iters = it;
  *res = rabs;
  if (e != STDG_OK) return e;
  if (hflag != 0.0) { set_error("viscous COCG: breakdown (p^T A p = 0)"); return STDG_ENOCONV; }
  if (!(rabs <= tol_abs)) { set_error("viscous COCG reached max_iters (%d)", it); return STDG_ENOCONV; }
  ++s->nlaunch;
  c32_mix_acc64(s->stream, ne, N, Ng, W, y, x);     // x += (I (x) W) y
  return STDG_OK;
}

stdg_status solve_viscous(stdg_solver* s, const double* b, double* x, double nu, double tol, int* iters,
                          double* res) {
  ApplyArgs a{};
  a.ne = (int)s->ne; a.N = s->N; a.Ng = s->Ng;
  a.t2f = s->dm.t2f; a.t2n = s->dm.t2n; a.left = s->dm.left;
  a.Bdiag = s->Bdiag; a.Aoff = s->Aoff; a.Bextra = s->Bvisc; a.detJ = s->dm.detJ;
  a.extra_coef = -1.0; a.scale = -nu * s->dt; a.mass_coef = 1.0; a.pin_diag = 0.0;
  a.tacc_identity = 1; a.pinned = 0;
  for (int q = 0; q < s->Ng * s->Ng; ++q) a.Kmass[q] = s->K[q];
  const int64_t n = s->ne * (int64_t)s->Nst;
  const double bn = host_norm(s, b, n);
  if (!std::isfinite(bn)) { set_error("viscous solve: non-finite right-hand side"); return STDG_ENAN; }
  if (bn == 0.0) { cudaMemsetAsync(x, 0, n * sizeof(double), s->stream); *iters = 0; *res = 0; return STDG_OK; }
  int rs = 0;
  // Decoupled COCG (above); then GMRES from its result, which only checks the true residual of the
  // original system unless COCG stopped short.  STDG_VISC_SOLVER=gmres in the environment selects the
  // previous solvers: CG (p_t = 0) or GMRES with a short restart, right-preconditioned by the exact
  // inverse of every tet's diagonal block (the system is mass-dominated and well conditioned; the
  // classical Gram-Schmidt passes against up to m basis vectors cost as much as the operator at
  // m ~ 25, so m = 20 bounds that work); STDG_VISC_PC=0 leaves that GMRES unpreconditioned.
  static const bool use_pc = !(std::getenv("STDG_VISC_PC") && std::atoi(std::getenv("STDG_VISC_PC")) == 0);
  static const bool use_cocg = !(std::getenv("STDG_VISC_SOLVER") && std::string(std::getenv("STDG_VISC_SOLVER")) == "gmres");
  if (s->pt == 0 && !use_cocg) {
    TpArg I{};
    I.v[0] = 1.0;
    return cg_block(s, a, b, x, false, I, tol * bn, iters, res);
  }
  int it1 = 0;
  if (use_cocg && s->opt.precision == STDG_PREC_MIXED_F32 && s->vbd != 0) {
    // mixed precision: binary64 refinement around binary32 inner COCG solves.  Each outer step forms
    // the true residual r = b - A x with the binary64-accurate operator and solves A d = r with the
    // binary32 operator to 1e-5 ||r|| (its rounding limits how far an inner solve can go), x += d.
    stdg_status e0 = ensure_basis(s, s->visc_inner64 ? 2 : 1);
    if (e0 != STDG_OK) return e0;
    double* ro = s->basis;
    const int64_t nn = s->ne * (int64_t)s->Nst;
    for (int outer = 0; outer < 8; ++outer) {
      if ((e0 = op_apply(s, a, x, ro)) != STDG_OK) return e0;
      ++s->nlaunch;
      k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(nn, b, nullptr, 1, ro);
      const double nr = host_norm(s, ro, nn);
      if (!std::isfinite(nr)) { set_error("viscous solve: non-finite residual"); return STDG_ENAN; }
      if (nr <= tol * bn) { *iters = it1; *res = nr; return STDG_OK; }
      int itk = 0;
      double rk = 0.0;
      e0 = s->visc_inner64 ? cocg_viscous(s, a, nu, ro, s->basis + nn, std::max(1e-5 * nr, 0.5 * tol * bn), &itk, &rk,
                                          true, true)
                           : cocg_viscous32(s, a, nu, ro, x, std::max(1e-5 * nr, 0.5 * tol * bn), &itk, &rk);
      it1 += itk;
      if (e0 == STDG_EUNSUPPORTED || e0 == STDG_ENOCONV) break;   // binary64 solvers below
      if (e0 != STDG_OK) return e0;
      if (s->visc_inner64) {
        ++s->nlaunch;
        k_add<<<kRedBlocks, kRedThreads, 0, s->stream>>>(nn, s->basis + nn, x);
      }
    }
  }
  if (use_cocg) {
    double r1 = 0.0;
    // half the tolerance: the recursively updated residual may drift from the true one by rounding
    stdg_status e1 = cocg_viscous(s, a, nu, b, x, 0.5 * tol * bn, &it1, &r1);
    if (e1 != STDG_OK && e1 != STDG_EUNSUPPORTED && e1 != STDG_ENOCONV) return e1;
  }
  int it2 = 0;
  stdg_status e2 = gmres(s, a, b, x, false, tol * bn, &it2, &rs, res, std::min(20, s->opt.restart), use_pc ? nu : -1.0);
  *iters = it1 + it2;
  return e2;
}

// ---------------------------------------------------------------------------------------------
// Allocation-free pressure solve.  Same Kronecker-decoupled block CG as stdg_solve(KRON_CG), but
// its work vectors live in one fixed device array compiled into the library instead of memory
// the solver allocates on first use.  The array holds four vectors of up to kNoAllocMaxDofs
// doubles, the reduction partials and a few scalars (8.5 MB on every device that loads the
// library, kept until the process exits).
constexpr int64_t kNoAllocMaxDofs = 262144;
constexpr int64_t kNoAllocPart = (int64_t)kRedBlocks * 8;
constexpr int64_t kNoAllocDoubles = 4 * kNoAllocMaxDofs + kNoAllocPart + 64;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[128] = {nullptr};

// Device address of g_noalloc_scratch on the current device, looked up once per device.
static stdg_status noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) { set_error("allocation-free solve: no usable device"); return STDG_ECUDA; }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("allocation-free solve: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return STDG_ECUDA;
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return STDG_OK;
}

static stdg_status noalloc_fetch(stdg_solver* s, const double* dev_src, double* host_dst) {
  if (cudaMemcpyAsync(host_dst, dev_src, sizeof(double), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess) {
    set_error("allocation-free solve: %s", cudaGetErrorString(cudaGetLastError()));
    return STDG_ECUDA;
  }
  return STDG_OK;
}

static stdg_status noalloc_norm(stdg_solver* s, const double* v, int64_t n, double* part, double* dst, double* out) {
  k_sumsq<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, v, part);
  k_final<<<1, kRedThreads, 0, s->stream>>>(kRedBlocks, 1, part, dst);
  s->nlaunch += 2;
  double h = 0.0;
  stdg_status e = noalloc_fetch(s, dst, &h);
  *out = std::sqrt(h);
  return e;
}

stdg_status solve_pressure_noalloc(stdg_solver* s, const double* b, double* x, double tol, stdg_solve_stats* st) {
  auto t0 = std::chrono::steady_clock::now();
  const int N = s->N, Ng = s->Ng;
  const int64_t n = s->ne * (int64_t)s->Nst;
  if (n > kNoAllocMaxDofs) {
    set_error("stdg_solve_noalloc: %lld pressure unknowns exceed the allocation-free limit of %lld "
              "(use stdg_solve)", (long long)n, (long long)kNoAllocMaxDofs);
    return STDG_EINVAL;
  }
  double* base = nullptr;
  stdg_status e = noalloc_scratch(&base);
  if (e != STDG_OK) return e;
  double* bt = base;
  double* r = base + kNoAllocMaxDofs;
  double* p = base + 2 * kNoAllocMaxDofs;
  double* q = base + 3 * kNoAllocMaxDofs;
  double* part = base + 4 * kNoAllocMaxDofs;
  double* scal = part + kNoAllocPart;
  double* rr = scal; double* pq = scal + 8; double* alpha = scal + 16; double* beta = scal + 24;
  double* rrnew = scal + 32; double* res = scal + 48; double* nrm = scal + 56;
  double bn = 0.0;
  if ((e = noalloc_norm(s, b, n, part, nrm, &bn)) != STDG_OK) return e;
  if (!std::isfinite(bn)) { set_error("stdg_solve_noalloc: non-finite right-hand side"); return STDG_ENAN; }
  // x starts at zero; every other scratch value is written before it is read
  cudaMemsetAsync(x, 0, n * sizeof(double), s->stream);
  int it = 0;
  double rabs = 0.0;
  if (bn > 0.0) {
    TpArg Tp{}, Tpinv{};
    const double idt2 = 1.0 / (s->dt * s->dt);
    for (int c = 0; c < Ng * Ng; ++c) { Tp.v[c] = s->tm.Tp[c]; Tpinv.v[c] = s->tm.K[c] * idt2; }
    const ApplyArgs op = pressure_op(s, 1, 1, -1.0, 1.0);
    k_timemix<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, Tpinv, -1.0, b, bt);
    cudaMemcpyAsync(r, bt, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    cudaMemcpyAsync(p, bt, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    k_coldot<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, r, r, part);
    k_final<<<Ng, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng, part, rr);
    s->nlaunch += 3;
    const double tol_abs = tol * bn;
    rabs = INFINITY;
    while (it < s->opt.max_iters) {
      if ((e = op_apply(s, op, p, q)) != STDG_OK) return e;
      k_coldot<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, p, q, part);
      k_final<<<Ng, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng, part, pq);
      k_cg_alpha<<<1, 32, 0, s->stream>>>(Ng, rr, pq, alpha);
      k_cg_update<<<kRedBlocks, kRedThreads, 0, s->stream>>>(s->ne, N, Ng, alpha, x, r, p, q, Tp, part);
      k_final<<<Ng + 1, kRedThreads, 0, s->stream>>>(kRedBlocks, Ng + 1, part, rrnew);
      k_cg_beta<<<1, 32, 0, s->stream>>>(Ng, rr, rrnew, beta, res);
      k_cg_dir<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, N, Ng, beta, r, p);
      s->nlaunch += 7;
      ++it;
      if ((e = noalloc_fetch(s, res, &rabs)) != STDG_OK) return e;
      if (!std::isfinite(rabs)) { set_error("stdg_solve_noalloc: non-finite residual"); return STDG_ENAN; }
      if (rabs <= tol_abs) break;
    }
  }
  if (st) {
    double rn = 0.0;
    if ((e = op_apply(s, pressure_op(s, 1, 0, 1.0, -1.0), x, q)) != STDG_OK) return e;
    k_scale_copy<<<kRedBlocks, kRedThreads, 0, s->stream>>>(n, b, nullptr, 1, q);
    ++s->nlaunch;
    if ((e = noalloc_norm(s, q, n, part, nrm, &rn)) != STDG_OK) return e;
    st->iterations = it;
    st->restarts = 0;
    st->rel_residual = bn > 0.0 ? rn / bn : 0.0;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (bn > 0.0 && rabs > tol * bn) { set_error("stdg_solve_noalloc reached max_iters (%d)", it); return STDG_ENOCONV; }
  return STDG_OK;
}

}  // namespace stdg

