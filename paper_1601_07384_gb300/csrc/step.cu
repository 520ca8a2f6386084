// Support steps of the Picard pressure-correction algorithm (Sec. 2.5-2.6) and its driver.
// Main-grid velocity is stored component-major, Vbar[c][ne][Ng][N], so that each component is a
// pressure-layout vector for the viscous solves.  With orthonormal bases (M_i = dt |J_i| I,
// M_{i,j} = dt M^sp_ij, Mbar_j = dt I, M_j = I (x) K, Mbar_i = |J_i| I (x) K):
//   average   vbar_i   = |J_i|^-1 Sum_{j in S_i} M^sp_ij v_j                     (Eq. average)
//   prevpress Lambda_i = |J_i|^-1 Sum_{j in S_i} M^sp_ij g_j,
//             g_j = dt (I (x) K^-1) Sum_s Q^sp_sj p_s  (boundary: volume part only)  (Eq. prevpress)
//   convection Upsilon^c_i (Eq. convdg, Rusanov flux, s_max = 2 max(|v+|, |v-|) pointwise)
//   goback    F_j = Sum_s M^sp_sj^T vbar_s                                       (Eq. goback)
//   viscous   |J_i| K-mixing + nu dt (-(A_sp x)_i + Bvisc_i x_i) = rhs          (Eq. A1_mod)
#include <chrono>
#include <cmath>
#include <cstring>

#include "pair.cuh"
#include "solver.h"

namespace stdg {

struct GArg { double v[kMaxNg]; };
struct MArg { double v[kMaxNg * kMaxNg]; };

// |det(B - A, C - A, c - A)| = 6 vol(T_ij) for face vertices fv = (A, B, C) and apex c
__device__ inline double subvol6(const double* fv, const double* c) {
  double e[3][3];
  for (int d = 0; d < 3; ++d) { e[0][d] = fv[3 + d] - fv[d]; e[1][d] = fv[6 + d] - fv[d]; e[2][d] = c[d] - fv[d]; }
  return fabs(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
              e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]));
}

__device__ inline void psi_hat(int N, const MultiIdx& mi, const double* C, const double* x0h, const double* x,
                               double* T, double* out) {
  const double hinv = 1.0 / x0h[3];
  const double y0 = (x[0] - x0h[0]) * hinv, y1 = (x[1] - x0h[1]) * hinv, y2 = (x[2] - x0h[2]) * hinv;
  for (int m = 0; m < N; ++m) {
    double v = 1.0;
    for (int e = 0; e < mi.e[3 * m]; ++e) v *= y0;
    for (int e = 0; e < mi.e[3 * m + 1]; ++e) v *= y1;
    for (int e = 0; e < mi.e[3 * m + 2]; ++e) v *= y2;
    T[m] = v;
  }
  for (int m = 0; m < N; ++m) {
    double s = 0.0;
    for (int n = 0; n <= m; ++n) s = fma(C[m * N + n], T[n], s);
    out[m] = s;
  }
}

// ---- averaging: out[c][i][a][k] = 1/|J_i| Sum_f Sum_l Mij[j][s][k][l] in[j][c][a][l]
__global__ void k_average(int ne, int N, int Ng, const int* __restrict__ t2f, const int* __restrict__ left,
                          const double* __restrict__ detJ, const double* __restrict__ Mij,
                          const double* __restrict__ in, double* __restrict__ out) {
  const int i = blockIdx.x, Nst = N * Ng;
  const size_t NN = (size_t)N * N;
  const double inv = 1.0 / detJ[i];
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    const int c = o / Nst, rem = o % Nst, a = rem / N, k = rem % N;
    double s = 0.0;
    for (int f = 0; f < 4; ++f) {
      const int j = t2f[4 * i + f];
      const int sd = left[j] == i ? 0 : 1;
      const double* M = Mij + ((size_t)j * 2 + sd) * NN + (size_t)k * N;
      const double* v = in + ((size_t)j * 3 + c) * Nst + a * N;
      for (int l = 0; l < N; ++l) s = fma(M[l], v[l], s);
    }
    out[((size_t)c * ne + i) * Nst + rem] = s * inv;
  }
}

// ---- g_j = dt (I (x) K^-1) Sum_s Q_sj p_s  (boundary: Q volume part of the single side)
__global__ void k_face_grad(int N, int Ng, const int* __restrict__ left, const int* __restrict__ right,
                            const double* __restrict__ Q, const double* __restrict__ Pp, double dt, MArg Ki,
                            double* __restrict__ G) {
  extern __shared__ double sm[];
  const int j = blockIdx.x, Nst = N * Ng;
  const size_t NN = (size_t)N * N;
  const int l = left[j], r = right[j];
  double* g = sm;   // 3 x Nst
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    const int c = o / Nst, rem = o % Nst, b = rem / N, m = rem % N;
    double s = 0.0;
    if (r >= 0) {
      for (int sd = 0; sd < 2; ++sd) {
        const double* q = Q + ((size_t)j * 6 + sd * 3 + c) * NN + (size_t)m * N;
        const double* pp = Pp + (size_t)(sd ? r : l) * Nst + b * N;
        for (int ll = 0; ll < N; ++ll) s = fma(q[ll], pp[ll], s);
      }
    } else {
      const double* q = Q + ((size_t)j * 6 + 3 + c) * NN + (size_t)m * N;
      const double* pp = Pp + (size_t)l * Nst + b * N;
      for (int ll = 0; ll < N; ++ll) s = fma(q[ll], pp[ll], s);
    }
    g[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    const int c = o / Nst, rem = o % Nst, a = rem / N, m = rem % N;
    double s = 0.0;
    for (int b = 0; b < Ng; ++b) s = fma(Ki.v[a * Ng + b], g[c * Nst + b * N + m], s);
    G[(size_t)j * 3 * Nst + o] = dt * s;
  }
}

// ---- goback: F[j][c][a][m] = Sum_s Sum_k Mij[j][s][k][m] vbar[c][s][a][k]; boundary: F = Vbc
__global__ void k_goback(int ne, int N, int Ng, const int* __restrict__ left, const int* __restrict__ right,
                         const double* __restrict__ Mij, const double* __restrict__ vbar,
                         const double* __restrict__ Vbc, double* __restrict__ F) {
  const int j = blockIdx.x, Nst = N * Ng;
  const size_t NN = (size_t)N * N;
  const int l = left[j], r = right[j];
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    if (r < 0) { F[(size_t)j * 3 * Nst + o] = Vbc[(size_t)j * 3 * Nst + o]; continue; }
    const int c = o / Nst, rem = o % Nst, a = rem / N, m = rem % N;
    double s = 0.0;
    for (int sd = 0; sd < 2; ++sd) {
      const double* M = Mij + ((size_t)j * 2 + sd) * NN + m;
      const double* v = vbar + ((size_t)c * ne + (sd ? r : l)) * Nst + a * N;
      for (int k = 0; k < N; ++k) s = fma(M[(size_t)k * N], v[k], s);
    }
    F[(size_t)j * 3 * Nst + o] = s;
  }
}

// ---- start of a step: V[j][c][0][m] = Sum_a g1[a] Vn[j][c][a][m], other modes 0; boundary = Vbc
__global__ void k_trace(int nf, int N, int Ng, const int* __restrict__ right, GArg g1, const double* __restrict__ Vn,
                        const double* __restrict__ Vbc, double* __restrict__ V) {
  const int Nst = N * Ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nf * 3 * Nst; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / (3 * Nst);
    const int rem = (int)(e % Nst), a = rem / N, m = rem % N;
    const int64_t base = e - rem;
    if (right[j] < 0) { V[e] = Vbc[e]; continue; }
    if (a != 0) { V[e] = 0.0; continue; }
    double s = 0.0;
    for (int b = 0; b < Ng; ++b) s = fma(g1.v[b], Vn[base + b * N + m], s);
    V[e] = s;
  }
}

// ---- viscous right-hand side (Eq. A1_mod):
// rhs[c][i][a][k] = |J| g0[a] Sum_b g1[b] vbar_n[c][i][b][k] - Ups[c][i][a][k] - |J| Sum_b K[a][b] Lam[c][i][b][k]
//                   - nu Sum_{boundary f} Sum_d Sum_m Q^{bd,d}[m][k] G[j][c][d][a][m]
__global__ void k_visc_rhs(int ne, int N, int Ng, const int* __restrict__ t2f, const int* __restrict__ t2n,
                           const double* __restrict__ detJ, const double* __restrict__ Q, GArg g0, GArg g1, MArg K,
                           double nu, const double* __restrict__ vbar_n, const double* __restrict__ Ups,
                           const double* __restrict__ Lam, const double* __restrict__ Gbc, double* __restrict__ rhs) {
  const int i = blockIdx.x, Nst = N * Ng;
  const size_t NN = (size_t)N * N;
  const double dj = detJ[i];
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    const int c = o / Nst, rem = o % Nst, a = rem / N, k = rem % N;
    const size_t vb = ((size_t)c * ne + i) * Nst;
    double tr = 0.0, kl = 0.0;
    for (int b = 0; b < Ng; ++b) {
      tr = fma(g1.v[b], vbar_n[vb + b * N + k], tr);
      kl = fma(K.v[a * Ng + b], Lam[vb + b * N + k], kl);
    }
    double s = dj * g0.v[a] * tr - Ups[vb + rem] - dj * kl;
    for (int f = 0; f < 4; ++f) {
      if (t2n[4 * i + f] >= 0) continue;
      const int j = t2f[4 * i + f];
      double bsum = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double* q = Q + ((size_t)j * 6 + d) * NN + k;
        const double* gg = Gbc + (((size_t)j * 3 + c) * 3 + d) * Nst + a * N;
        for (int m = 0; m < N; ++m) bsum = fma(q[(size_t)m * N], gg[m], bsum);
      }
      s -= nu * bsum;
    }
    rhs[vb + rem] = s;
  }
}

// ---- boundary data on boundary dual cells T_ij x slab (reading R2 / R25)
// Vbc[j][c][a][m] = Sum_{q,t} w ψ_m γ_a(τ_t) v_c ; Gbc[j][c][d][a][m] = dt Sum_{qf,t} wf ψ_m γ_a v_c n_d
__global__ void __launch_bounds__(128) k_boundary(int N, int Ng, int nq, int nqf, int nt, const int* __restrict__ left,
                                                  const int* __restrict__ right, const int* __restrict__ fl,
                                                  const double* __restrict__ bary, const double* __restrict__ J,
                                                  const double* __restrict__ detJ, const double* __restrict__ fvx,
                                                  const double* __restrict__ normal, const double* __restrict__ area,
                                                  const double* __restrict__ C, const double* __restrict__ x0h,
                                                  const double* __restrict__ sub_xi, const double* __restrict__ sub_w,
                                                  const double* __restrict__ tri_st, const double* __restrict__ tri_w,
                                                  const double* __restrict__ ttau, const double* __restrict__ tw,
                                                  const double* __restrict__ tg, MultiIdx mi, FieldArg fld, double t0,
                                                  double dt, const int* __restrict__ bidx, double* __restrict__ Vbc,
                                                  double* __restrict__ Gbc) {
  const int j = blockIdx.x;
  if (right[j] >= 0) return;
  // data points of this boundary face (host-callback data): nq*nt sub-tetrahedron points, then nqf*nt face points
  const int64_t pid0 = (int64_t)bidx[j] * (nq + nqf) * nt;
  extern __shared__ double sm[];
  const int Nst = N * Ng;
  const int CH = 64;
  double* ps = sm;                 // CH x N  (w * psi)
  double* vv = ps + CH * N;        // CH x 3
  double* tmp = vv + CH * 3;       // CH x N scratch
  __shared__ int tq[64], tt[64];
  const int i = left[j];
  const double* Cj = C + (size_t)j * N * N;
  const double* xh = x0h + 4 * (size_t)j;
  const double* fv = fvx + 9 * (size_t)j;
  const double* nj = normal + 3 * (size_t)j;
  for (int pass = 0; pass < 2; ++pass) {
    const int npts = (pass == 0 ? nq : nqf) * nt;
    for (int base = 0; base < npts; base += CH) {
      const int cnt = min(CH, npts - base);
      for (int u = threadIdx.x; u < cnt; u += blockDim.x) {
        const int pt = base + u, q = pt / nt, ti = pt % nt;
        double x[3], w;
        if (pass == 0) {
          // unit-tet rule laid on (A, B, C, barycentre of T_i): the canonical vertex order of T_ij
          const double* xi = sub_xi + 3 * (size_t)q;
          const double* bc = bary + 3 * (size_t)i;
          for (int d = 0; d < 3; ++d)
            x[d] = fv[d] + xi[0] * (fv[3 + d] - fv[d]) + xi[1] * (fv[6 + d] - fv[d]) + xi[2] * (bc[d] - fv[d]);
          w = subvol6(fv, bc) * sub_w[q] * tw[ti];
        } else {
          const double s = tri_st[2 * q], tt2 = tri_st[2 * q + 1];
          for (int d = 0; d < 3; ++d) x[d] = fv[d] + s * (fv[3 + d] - fv[d]) + tt2 * (fv[6 + d] - fv[d]);
          w = 2.0 * area[j] * tri_w[q] * tw[ti] * dt;
        }
        psi_hat(N, mi, Cj, xh, x, tmp + u * N, ps + u * N);
        for (int m = 0; m < N; ++m) ps[u * N + m] *= w;
        eval_field(fld, x, t0 + ttau[ti] * dt, pid0 + (pass == 0 ? 0 : (int64_t)nq * nt) + pt, ttau[ti], vv + 3 * u);
        tq[u] = q; tt[u] = ti;
      }
      __syncthreads();
      const int nout = pass == 0 ? 3 * Nst : 9 * Nst;
      for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        int c, dd = 0, rem;
        if (pass == 0) { c = o / Nst; rem = o % Nst; } else { c = o / (3 * Nst); dd = (o / Nst) % 3; rem = o % Nst; }
        const int a = rem / N, m = rem % N;
        double s = 0.0;
        for (int u = 0; u < cnt; ++u) s = fma(ps[u * N + m] * tg[tt[u] * Ng + a], vv[3 * u + c], s);
        if (pass == 0) {
          double* dst = Vbc + (size_t)j * 3 * Nst + o;
          *dst = (base == 0 ? 0.0 : *dst) + s;
        } else {
          double* dst = Gbc + (size_t)j * 9 * Nst + o;
          *dst = (base == 0 ? 0.0 : *dst) + s * nj[dd];
        }
      }
      __syncthreads();
    }
  }
}

// ---- initial data: V[j][c][0][m] = Sum_{sides} Sum_q w psi_m v0_c(x_q), other time modes 0
__global__ void __launch_bounds__(128) k_initial(int N, int Ng, int nq, const int* __restrict__ left,
                                                 const int* __restrict__ right, const double* __restrict__ fvx,
                                                 const double* __restrict__ fshift, const double* __restrict__ bary,
                                                 const double* __restrict__ C, const double* __restrict__ x0h,
                                                 const double* __restrict__ sub_xi, const double* __restrict__ sub_w,
                                                 MultiIdx mi, FieldArg fld, double* __restrict__ V) {
  extern __shared__ double sm[];
  const int j = blockIdx.x, Nst = N * Ng;
  const int CH = 64;
  double* ps = sm;
  double* vv = ps + CH * N;
  double* tmp = vv + CH * 3;
  const double* Cj = C + (size_t)j * N * N;
  const double* xh = x0h + 4 * (size_t)j;
  const int nsides = right[j] >= 0 ? 2 : 1;
  const int npts = nq * nsides;
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) V[(size_t)j * 3 * Nst + o] = 0.0;
  __syncthreads();
  for (int base = 0; base < npts; base += CH) {
    const int cnt = min(CH, npts - base);
    for (int u = threadIdx.x; u < cnt; u += blockDim.x) {
      const int pt = base + u, sd = pt / nq, q = pt % nq;
      const int i = sd ? right[j] : left[j];
      const double* xi = sub_xi + 3 * (size_t)q;
      const double* fv = fvx + 9 * (size_t)j;
      // the apex of T_ij in l(j)'s frame (r(j)'s barycentre shifted by fshift on periodic meshes)
      double bc[3];
      for (int d = 0; d < 3; ++d) bc[d] = bary[3 * (size_t)i + d] + (sd ? fshift[3 * (size_t)j + d] : 0.0);
      double x[3];
      for (int d = 0; d < 3; ++d)
        x[d] = fv[d] + xi[0] * (fv[3 + d] - fv[d]) + xi[1] * (fv[6 + d] - fv[d]) + xi[2] * (bc[d] - fv[d]);
      const double w = subvol6(fv, bc) * sub_w[q];
      psi_hat(N, mi, Cj, xh, x, tmp + u * N, ps + u * N);
      for (int m = 0; m < N; ++m) ps[u * N + m] *= w;
      eval_field(fld, x, 0.0, (int64_t)j * 2 * nq + pt, 0.0, vv + 3 * u);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < 3 * N; o += blockDim.x) {
      const int c = o / N, m = o % N;
      double s = 0.0;
      for (int u = 0; u < cnt; ++u) s = fma(ps[u * N + m], vv[3 * u + c], s);
      V[(size_t)j * 3 * Nst + c * Nst + m] += s;
    }
    __syncthreads();
  }
}

// ---- Rusanov space-time DG convection on the main grid (Eq. convdg), per tet.
struct ConvArgs {
  int ne, N, Ng, nq, nqf, nt;
  const int *t2f, *t2n, *t2code, *left, *code_l, *code_r;
  const double *detJ, *Jinv, *normal, *area, *fvx;
  const double *phi, *dphi, *w, *fphi, *tri_st, *tri_w, *ttau, *tw, *tg;
  FieldArg fld;
  double t0, dt;
  const float2 *tgP, *twP;   // the time basis at the time points [nt][Ng] and the time weights, as pairs
  const int* bidx;      // compact boundary index per face (points of host-callback data)
  int bnpt;             // data points per boundary face: (nq + nqf) * nt, face points after nq * nt
  const double* vbar;   // [3][ne][Nst]
  double* ups;          // [3][ne][Nst]
};

// One block per tet.  The space-time quadrature is sum-factorised in time: for every spatial point
// (one thread each) the spatial sums Sum_k phi_k(x_q) V[c][b][k] are formed once, the flux is
// evaluated at the n_t time points from them, and the time test functions are folded in at once,
// G[q][c][e][a] = Sum_t gamma_a(tau_t) H(x_q, tau_t)[c][e]; the spatial test functions are applied
// in a second pass.  Compared with evaluating every space-time point from scratch this divides the
// work by n_t (3 at p_t = 1, 7 at p_t = 4); the sums are the same up to rounding order.
//
// The two dense contractions (basis values x coefficients, and test functions x G) are formed from
// binary32 pairs, a = hi + lo with hi = fl32(a), lo = fl32(a - hi): each product hi_a hi_b is exact by
// an FMA, the cross terms are added to its error, and the sum is kept as an unevaluated binary32
// pair (TwoSum), converted to binary64 at the end of the sum.  That is binary64-accurate (relative
// error ~1e-14 of the sum of |terms|) at 12 FP32 operations per term on a pipe 64 times faster than
// sm_103a's FP64 pipe, which the binary64 kernel kept 86 % busy.  The flux itself (products of the
// velocities, the Rusanov speed) stays binary64.
constexpr int kConvCH = 128;        // spatial points per pass (= threads per block)
constexpr int kMaxTimePts = 8;      // time points of the compile-time kernels (7 at p_t = 4)

// S[c][b] = Sum_k phi_k(x_q) V[c][b][k] at one quadrature point, as normalised pairs: each basis value
// is loaded once and used by the 3 Ng sums (the coefficients V are the same for every point: shared
// memory broadcasts)
__device__ __forceinline__ void contract_point(const float2* __restrict__ ph, const float2* V, int N, int Ng, int Nst,
                                               float2 (&S)[3][kMaxNg]) {
  float ss[3][kMaxNg], cc[3][kMaxNg];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < kMaxNg; ++b) { ss[c][b] = 0.0f; cc[c][b] = 0.0f; }
  for (int k = 0; k < N; ++k) {
    const float2 pk = ph[k];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < kMaxNg; ++b)
        if (b < Ng) pair_fma(pk, V[c * Nst + b * N + k], ss[c][b], cc[c][b]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < kMaxNg; ++b) S[c][b] = pair_norm(ss[c][b], cc[c][b]);
}

__global__ void k_split_pairs(int64_t n, const double* __restrict__ in, float2* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = pair_split(in[e]);
}

__global__ void __launch_bounds__(kConvCH) k_convection(ConvArgs a, const float2* __restrict__ phiP,
                                                        const float2* __restrict__ dphiP,
                                                        const float2* __restrict__ fphiP) {
  extern __shared__ double sm[];
  const int i = blockIdx.x, N = a.N, Ng = a.Ng, Nst = N * Ng, ne = a.ne, nt = a.nt;
  double* acc = sm;                                          // 3 x Nst
  float2* ViP = reinterpret_cast<float2*>(acc + 3 * Nst);    // 3 x Nst (own coefficients, pairs)
  float2* VnP = ViP + 3 * Nst;                               // 3 x Nst (neighbour coefficients, pairs)
  double* G = reinterpret_cast<double*>(VnP + 3 * Nst);      // kConvCH x 9 x Ng (volume) or x 3 x Ng (faces)
  float2* GP = reinterpret_cast<float2*>(G);                 // the same, as pairs (each thread converts its own)
  const double* Ji = a.Jinv + 9 * (size_t)i;
  const double dj = a.detJ[i];
  const int u = threadIdx.x;
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    acc[o] = 0.0;
    const int c = o / Nst, rem = o % Nst;
    ViP[o] = pair_split(a.vbar[((size_t)c * ne + i) * Nst + rem]);
  }
  __syncthreads();
  // volume term: - int grad(phi~_k) . F_c(vbar); the flux and its time folding in binary32 pairs
  // (the FP64 pipe, 1/64 of the FP32 rate on sm_103a, stays free of the per-point work)
  __shared__ float2 JiP[9];
  if (threadIdx.x < 9) JiP[threadIdx.x] = pair_split(Ji[threadIdx.x]);
  __syncthreads();
  for (int base = 0; base < a.nq; base += kConvCH) {
    const int cnt = min(kConvCH, a.nq - base);
    if (u < cnt) {
      const int q = base + u;
      const float2* ph = phiP + (size_t)q * N;
      float2 SP[3][kMaxNg];
      contract_point(ph, ViP, N, Ng, Nst, SP);
      float2* Gu = GP + (size_t)u * 9 * Ng;       // accumulators (s, c) of G[c][e][ta]
      for (int e = 0; e < 9 * Ng; ++e) Gu[e] = make_float2(0.0f, 0.0f);
      const float2 wqP = pair_split(a.dt * dj * a.w[q]);
      for (int ti = 0; ti < nt; ++ti) {
        const float2* g = a.tgP + ti * Ng;
        float2 vP[3], uP[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float ss = 0.0f, cc = 0.0f;
#pragma unroll
          for (int b = 0; b < kMaxNg; ++b)
            if (b < Ng) pair_fma(g[b], SP[c][b], ss, cc);
          vP[c] = pair_norm(ss, cc);
        }
        // u = Jinv v: grad_x phi = Sum_e Jinv[e][d] d_e phi
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          float ss = 0.0f, cc = 0.0f;
          pair_fma(JiP[3 * e], vP[0], ss, cc);
          pair_fma(JiP[3 * e + 1], vP[1], ss, cc);
          pair_fma(JiP[3 * e + 2], vP[2], ss, cc);
          uP[e] = pair_norm(ss, cc);
        }
        const float2 W = pair_mul(wqP, a.twP[ti]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 Wv = pair_mul(W, vP[c]);
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const float2 h = pair_mul(Wv, uP[e]);     // H[c][e] = W v_c u_e
            float2* Gce = Gu + (c * 3 + e) * Ng;
            for (int ta = 0; ta < Ng; ++ta) {
              float2 G = Gce[ta];
              pair_fma(g[ta], h, G.x, G.y);
              Gce[ta] = G;
            }
          }
        }
      }
      for (int e = 0; e < 9 * Ng; ++e) Gu[e] = pair_norm(Gu[e].x, Gu[e].y);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
      const int c = o / Nst, rem = o % Nst, ta = rem / N, k = rem % N;
      float ss = 0.0f, cc = 0.0f;
      for (int v = 0; v < cnt; ++v) {
        const float2* dp = dphiP + (size_t)(base + v) * 3 * N + k;
        const float2* Gv = GP + (size_t)v * 9 * Ng + c * 3 * Ng + ta;
        pair_fma(Gv[0], dp[0], ss, cc);
        pair_fma(Gv[Ng], dp[N], ss, cc);
        pair_fma(Gv[2 * Ng], dp[2 * N], ss, cc);
      }
      acc[o] -= pair_value(ss, cc);
    }
    __syncthreads();
  }
  // face terms: + int_{face} phi~_k F^RS . n_i
  for (int f = 0; f < 4; ++f) {
    const int j = a.t2f[4 * i + f];
    const int nb = a.t2n[4 * i + f];
    const bool me_left = a.left[j] == i;
    const int code = a.t2code[4 * i + f];
    const int codeb = nb >= 0 ? (me_left ? a.code_r[j] : a.code_l[j]) : 0;
    const double sg = me_left ? 1.0 : -1.0;
    const float2 nP[3] = {pair_split(sg * a.normal[3 * j]), pair_split(sg * a.normal[3 * j + 1]),
                          pair_split(sg * a.normal[3 * j + 2])};
    const double* fv = a.fvx + 9 * (size_t)j;
    if (nb >= 0) {
      for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
        const int c = o / Nst, rem = o % Nst;
        VnP[o] = pair_split(a.vbar[((size_t)c * ne + nb) * Nst + rem]);
      }
    }
    __syncthreads();
    for (int base = 0; base < a.nqf; base += kConvCH) {
      const int cnt = min(kConvCH, a.nqf - base);
      if (u < cnt) {
        const int q = base + u;
        const float2* ph = fphiP + ((size_t)code * a.nqf + q) * N;
        float2 SmP[3][kMaxNg], SpP[3][kMaxNg];
        contract_point(ph, ViP, N, Ng, Nst, SmP);
        double x[3] = {0.0, 0.0, 0.0};
        if (nb >= 0) {
          contract_point(fphiP + ((size_t)codeb * a.nqf + q) * N, VnP, N, Ng, Nst, SpP);
        } else {
          const double s = a.tri_st[2 * q], t = a.tri_st[2 * q + 1];
          for (int d = 0; d < 3; ++d) x[d] = fv[d] + s * (fv[3 + d] - fv[d]) + t * (fv[6 + d] - fv[d]);
        }
        float2* Gu = GP + (size_t)u * 3 * Ng;     // accumulators (s, c) of G[c][ta]
        for (int e = 0; e < 3 * Ng; ++e) Gu[e] = make_float2(0.0f, 0.0f);
        const float2 wqP = pair_split(a.dt * 2.0 * a.area[j] * a.tri_w[q]);
        for (int ti = 0; ti < nt; ++ti) {
          const float2* g = a.tgP + ti * Ng;
          float2 vm[3], vp[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float ss = 0.0f, cc = 0.0f;
#pragma unroll
            for (int b = 0; b < kMaxNg; ++b)
              if (b < Ng) pair_fma(g[b], SmP[c][b], ss, cc);
            vm[c] = pair_norm(ss, cc);
          }
          if (nb >= 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              float ss = 0.0f, cc = 0.0f;
#pragma unroll
              for (int b = 0; b < kMaxNg; ++b)
                if (b < Ng) pair_fma(g[b], SpP[c][b], ss, cc);
              vp[c] = pair_norm(ss, cc);
            }
          } else {
            double vb[3];
            eval_field(a.fld, x, a.t0 + a.ttau[ti] * a.dt,
                       (int64_t)a.bidx[j] * a.bnpt + (int64_t)a.nq * nt + (int64_t)q * nt + ti, a.ttau[ti], vb);
            for (int c = 0; c < 3; ++c) vp[c] = pair_split(vb[c]);
          }
          // Rusanov flux, s_max = 2 max(|v+|, |v-|) pointwise (the square roots in binary64)
          float s1 = 0.0f, c1 = 0.0f, s2 = 0.0f, c2 = 0.0f, s3 = 0.0f, c3 = 0.0f, s4 = 0.0f, c4 = 0.0f;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            pair_fma(vm[c], nP[c], s1, c1);
            pair_fma(vp[c], nP[c], s2, c2);
            pair_fma(vm[c], vm[c], s3, c3);
            pair_fma(vp[c], vp[c], s4, c4);
          }
          const float2 unm = pair_norm(s1, c1), unp = pair_norm(s2, c2);
          const double smax = 2.0 * fmax(sqrt(pair_value(s4, c4)), sqrt(pair_value(s3, c3)));
          const float2 W = pair_mul(wqP, a.twP[ti]);
          const float2 hs = pair_mul(W, pair_split(0.5 * smax));
          const float2 Wh = pair_mul(W, make_float2(0.5f, 0.0f));
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            // h = W (0.5 (v+_c un+ + v-_c un-) - 0.5 s_max (v+_c - v-_c))
            const float2 cen = pair_mul(Wh, pair_add(pair_mul(vp[c], unp), pair_mul(vm[c], unm)));
            const float2 h = pair_add(cen, pair_neg(pair_mul(hs, pair_add(vp[c], pair_neg(vm[c])))));
            float2* Gc = Gu + c * Ng;
            for (int ta = 0; ta < Ng; ++ta) {
              float2 G = Gc[ta];
              pair_fma(g[ta], h, G.x, G.y);
              Gc[ta] = G;
            }
          }
        }
        for (int e = 0; e < 3 * Ng; ++e) Gu[e] = pair_norm(Gu[e].x, Gu[e].y);
      }
      __syncthreads();
      for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
        const int c = o / Nst, rem = o % Nst, ta = rem / N, k = rem % N;
        float ss = 0.0f, cc = 0.0f;
        for (int v = 0; v < cnt; ++v)
          pair_fma(fphiP[((size_t)code * a.nqf + base + v) * N + k], GP[(size_t)v * 3 * Ng + c * Ng + ta], ss, cc);
        acc[o] += pair_value(ss, cc);
      }
      __syncthreads();
    }
  }
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    const int c = o / Nst, rem = o % Nst;
    a.ups[((size_t)c * ne + i) * Nst + rem] = acc[o];
  }
}

// ---- The same convection with N and Ng at compile time (the benchmarked degrees), reorganised:
//  * points of all four faces go through shared passes of kConvCH (two passes at p = 4 instead of
//    four passes with 49 of 128 threads busy);
//  * the test-function sums are owned by threads: thread (c, k) keeps the sums of its time columns
//    in registers across all passes, so one coalesced table load serves all of them (the general
//    kernel loads the table once per multiply-add and reads and writes its sums in shared memory);
//  * the per-point sums Sum_k phi_k(x_q) V[.][k] read the basis tables transposed ([k][point]:
//    coalesced over the threads of a pass);
//  * the pair arithmetic of the contractions and of the time folding runs two sums at a time in
//    packed binary32 operations (f32x2).
// The arithmetic per term is that of the general kernel (the same products, error terms and
// error-free sums), so the results agree with it to the rounding of the pair sums.

// S[m] = Sum_k tab[k * stride] V[m * N + k] for the NA coefficient rows of V, as normalised pairs
template <int N, int NA>
__device__ __forceinline__ void conv_contract(const float2* __restrict__ tab, int stride, const float2* V,
                                              float2 (&S)[NA]) {
  constexpr int NA2 = (NA + 1) / 2;
  float2 sm[NA2], cm[NA2];
#pragma unroll
  for (int m = 0; m < NA2; ++m) sm[m] = cm[m] = make_float2(0.0f, 0.0f);
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const float2 pk = tab[(size_t)k * stride];
    const float2 ah2 = make_float2(pk.x, pk.x), nah2 = make_float2(-pk.x, -pk.x), al2 = make_float2(pk.y, pk.y);
#pragma unroll
    for (int m = 0; m < NA2; ++m) {
      const float2 v0 = V[(2 * m) * N + k];
      const float2 v1 = 2 * m + 1 < NA ? V[(2 * m + 1) * N + k] : make_float2(0.0f, 0.0f);
      pair_fma2(ah2, nah2, al2, make_float2(v0.x, v1.x), make_float2(v0.y, v1.y), sm[m], cm[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < NA2; ++m) {
    S[2 * m] = pair_norm(sm[m].x, cm[m].x);
    if (2 * m + 1 < NA) S[2 * m + 1] = pair_norm(sm[m].y, cm[m].y);
  }
}

// G[ta] += h g_ta for the NG time columns of one row of G (NGP pairs, stored (s, c)), packed over
// consecutive columns; g holds NGP pairs, the padding one zero
template <int NGP>
__device__ __forceinline__ void conv_fold(float2* G, float2 h, const float2* g) {
  const float2 hh2 = make_float2(h.x, h.x), nh2 = make_float2(-h.x, -h.x), hl2 = make_float2(h.y, h.y);
#pragma unroll
  for (int m = 0; m < NGP / 2; ++m) {
    float4 G2 = *reinterpret_cast<float4*>(G + 2 * m);
    float2 sv = make_float2(G2.x, G2.z), cv = make_float2(G2.y, G2.w);
    pair_fma2(hh2, nh2, hl2, make_float2(g[2 * m].x, g[2 * m + 1].x), make_float2(g[2 * m].y, g[2 * m + 1].y), sv, cv);
    *reinterpret_cast<float4*>(G + 2 * m) = make_float4(sv.x, cv.x, sv.y, cv.y);
  }
}

template <int N, int NG>
struct ConvT {
  static constexpr int Nst = N * NG, NA = 3 * NG, NGP = (NG + 1) & ~1;
  // owners of the test-function sums: thread -> (split, component c, row k), time columns
  // [split TG, split TG + TG)
  static constexpr int NSPLIT = 3 * N * NG <= kConvCH ? NG : 1;
  static constexpr int TG = NG / NSPLIT, TG2 = (TG + 1) / 2, NOWN = 3 * N * NSPLIT;
  // shared memory (pairs): own coefficients, then the volume fold G[point][c][e][NGP], which the face
  // passes reuse for the neighbour coefficients of the four faces and the face fold G[point][c][NGP]
  // (own coefficients padded to an even count: the folds are read and written as float4)
  static constexpr int kOwn = (NA * N + 1) & ~1;
  static constexpr int kVol = kConvCH * 9 * NGP, kFace = 4 * NA * N + kConvCH * 3 * NGP;
  // then the owners' binary64 sums [NOWN][TG]
  static constexpr size_t kAccOff = ((size_t)kOwn + (kVol > kFace ? kVol : kFace)) * sizeof(float2);
  static constexpr size_t kSmem = kAccOff + (size_t)NOWN * TG * sizeof(double);
};

// the owner's share of Sum_v a_v G_v over the pass: a_v broadcast pair, G rows of the pass
template <int TG, int NGP>
__device__ __forceinline__ void conv_owner_acc(float2 av, const float2* G, float2 (&As)[(TG + 1) / 2],
                                               float2 (&Ac)[(TG + 1) / 2]) {
  const float2 ah2 = make_float2(av.x, av.x), nah2 = make_float2(-av.x, -av.x), al2 = make_float2(av.y, av.y);
  if constexpr (TG == 1) {
    const float2 g = G[0];
    pair_fma2(ah2, nah2, al2, make_float2(g.x, 0.0f), make_float2(g.y, 0.0f), As[0], Ac[0]);
  } else {
#pragma unroll
    for (int m = 0; m < (TG + 1) / 2; ++m) {
      const float4 G2 = *reinterpret_cast<const float4*>(G + 2 * m);
      pair_fma2(ah2, nah2, al2, make_float2(G2.x, G2.z), make_float2(G2.y, G2.w), As[m], Ac[m]);
    }
  }
}

template <int N, int NG>
__global__ void __launch_bounds__(kConvCH, 3) k_convection_t(ConvArgs a, const float2* __restrict__ phiT,
                                                             const float2* __restrict__ dphiP,
                                                             const float2* __restrict__ fphiT,
                                                             const float2* __restrict__ fphiP) {
  using C = ConvT<N, NG>;
  constexpr int Nst = C::Nst, NA = C::NA, NGP = C::NGP, TG = C::TG, TG2 = C::TG2;
  extern __shared__ float2 cvs[];
  float2* ViP = cvs;                              // [c][b][k]: own coefficients as pairs
  float2* Gv = cvs + C::kOwn;                      // volume: [point][c][e][NGP]
  float2* VnP = Gv;                               // faces: [face][c][b][k] neighbour coefficients
  float2* Gf = Gv + 4 * NA * N;                   // faces: [point][c][NGP]
  __shared__ float2 JiP[9];
  __shared__ float2 fnP[4][3];
  __shared__ int fjj[4], fnb[4], fcode[4], fcodeb[4];
  __shared__ float2 gtab[kMaxTimePts * NGP];      // time basis at the time points, padding columns zero
  const int i = blockIdx.x, u = threadIdx.x, ne = a.ne, nt = a.nt;
  for (int o = u; o < nt * NGP; o += kConvCH) {
    const int ti = o / NGP, b = o - ti * NGP;
    gtab[o] = b < NG ? a.tgP[ti * NG + b] : make_float2(0.0f, 0.0f);
  }
  for (int o = u; o < NA * N; o += kConvCH) {
    const int c = o / Nst, rem = o - c * Nst;
    ViP[o] = pair_split(a.vbar[((size_t)c * ne + i) * Nst + rem]);
  }
  if (u < 9) JiP[u] = pair_split(a.Jinv[9 * (size_t)i + u]);
  if (u < 4) {
    const int j = a.t2f[4 * i + u], nb = a.t2n[4 * i + u];
    const bool me_left = a.left[j] == i;
    const double sg = me_left ? 1.0 : -1.0;
    fjj[u] = j; fnb[u] = nb; fcode[u] = a.t2code[4 * i + u];
    fcodeb[u] = nb >= 0 ? (me_left ? a.code_r[j] : a.code_l[j]) : 0;
    for (int d = 0; d < 3; ++d) fnP[u][d] = pair_split(sg * a.normal[3 * j + d]);
  }
  const bool own = u < C::NOWN;
  const int osp = u / (3 * N), orem = u - osp * 3 * N, oc = orem / N, ok = orem - oc * N, ota0 = osp * TG;
  double* accd = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(cvs) + C::kAccOff) + (size_t)u * TG;
  if (own)
#pragma unroll
    for (int t = 0; t < TG; ++t) accd[t] = 0.0;
  auto owner_flush = [&](const float2 (&As)[TG2], const float2 (&Ac)[TG2]) {   // a pass's pair sums, in binary64
#pragma unroll
    for (int m = 0; m < TG2; ++m) {
      accd[2 * m] += pair_value(As[m].x, Ac[m].x);
      if (2 * m + 1 < TG) accd[2 * m + 1] += pair_value(As[m].y, Ac[m].y);
    }
  };
  const double dj = a.detJ[i];
  __syncthreads();

  // volume term: - int grad(phi~_k) . F_c(vbar)
  for (int base = 0; base < a.nq; base += kConvCH) {
    const int cnt = min(kConvCH, a.nq - base);
    if (u < cnt) {
      const int q = base + u;
      float2 S[NA];
      conv_contract<N, NA>(phiT + q, a.nq, ViP, S);
      float2* Gu = Gv + (size_t)u * 9 * NGP;
#pragma unroll
      for (int e = 0; e < 9 * NGP; e += 2) *reinterpret_cast<float4*>(Gu + e) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float2 wqP = pair_split(a.dt * dj * a.w[q]);
      for (int ti = 0; ti < nt; ++ti) {
        const float2* g = gtab + ti * NGP;
        float2 vP[3], uP[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float ss = 0.0f, cc = 0.0f;
#pragma unroll
          for (int b = 0; b < NG; ++b) pair_fma(g[b], S[c * NG + b], ss, cc);
          vP[c] = pair_norm(ss, cc);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          float ss = 0.0f, cc = 0.0f;
          pair_fma(JiP[3 * e], vP[0], ss, cc);
          pair_fma(JiP[3 * e + 1], vP[1], ss, cc);
          pair_fma(JiP[3 * e + 2], vP[2], ss, cc);
          uP[e] = pair_norm(ss, cc);
        }
        const float2 W = pair_mul(wqP, a.twP[ti]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 Wv = pair_mul(W, vP[c]);
#pragma unroll
          for (int e = 0; e < 3; ++e) conv_fold<NGP>(Gu + (c * 3 + e) * NGP, pair_mul(Wv, uP[e]), g);
        }
      }
#pragma unroll 6
      for (int e = 0; e < 9 * NGP; ++e) Gu[e] = pair_norm(Gu[e].x, Gu[e].y);
    }
    __syncthreads();
    if (own) {
      float2 As[TG2], Ac[TG2];
#pragma unroll
      for (int m = 0; m < TG2; ++m) As[m] = Ac[m] = make_float2(0.0f, 0.0f);
#pragma unroll 1
      for (int v = 0; v < cnt; ++v) {
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const float2 dp = dphiP[((size_t)(base + v) * 3 + e) * N + ok];
          conv_owner_acc<TG, NGP>(make_float2(-dp.x, -dp.y), Gv + ((size_t)v * 9 + oc * 3 + e) * NGP + ota0, As, Ac);
        }
      }
      owner_flush(As, Ac);
    }
    __syncthreads();
  }

  // face terms: + int_{face} phi~_k F^RS . n_i, the points of all four faces in shared passes
  for (int f = 0; f < 4; ++f) {
    const int nb = fnb[f];
    if (nb < 0) continue;
    for (int o = u; o < NA * N; o += kConvCH) {
      const int c = o / Nst, rem = o - c * Nst;
      VnP[f * NA * N + o] = pair_split(a.vbar[((size_t)c * ne + nb) * Nst + rem]);
    }
  }
  __syncthreads();
  const int nqf = a.nqf, nfp = 4 * nqf;
  for (int base = 0; base < nfp; base += kConvCH) {
    const int cnt = min(kConvCH, nfp - base);
    if (u < cnt) {
      const int P = base + u, f = P / nqf, q = P - f * nqf;
      const int j = fjj[f], nb = fnb[f];
      float2 SmP[NA], SpP[NA];
      conv_contract<N, NA>(fphiT + (size_t)fcode[f] * N * nqf + q, nqf, ViP, SmP);
      double x[3] = {0.0, 0.0, 0.0};
      if (nb >= 0) {
        conv_contract<N, NA>(fphiT + (size_t)fcodeb[f] * N * nqf + q, nqf, VnP + f * NA * N, SpP);
      } else {
        const double* fv = a.fvx + 9 * (size_t)j;
        const double s0 = a.tri_st[2 * q], t0 = a.tri_st[2 * q + 1];
        for (int d = 0; d < 3; ++d) x[d] = fv[d] + s0 * (fv[3 + d] - fv[d]) + t0 * (fv[6 + d] - fv[d]);
      }
      float2* Gu = Gf + (size_t)u * 3 * NGP;
#pragma unroll
      for (int e = 0; e < 3 * NGP; e += 2) *reinterpret_cast<float4*>(Gu + e) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float2 wqP = pair_split(a.dt * 2.0 * a.area[j] * a.tri_w[q]);
      const float2* nP = fnP[f];
      for (int ti = 0; ti < nt; ++ti) {
        const float2* g = gtab + ti * NGP;
        float2 vm[3], vp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float ss = 0.0f, cc = 0.0f;
#pragma unroll
          for (int b = 0; b < NG; ++b) pair_fma(g[b], SmP[c * NG + b], ss, cc);
          vm[c] = pair_norm(ss, cc);
        }
        if (nb >= 0) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float ss = 0.0f, cc = 0.0f;
#pragma unroll
            for (int b = 0; b < NG; ++b) pair_fma(g[b], SpP[c * NG + b], ss, cc);
            vp[c] = pair_norm(ss, cc);
          }
        } else {
          double vb[3];
          eval_field(a.fld, x, a.t0 + a.ttau[ti] * a.dt,
                     (int64_t)a.bidx[j] * a.bnpt + (int64_t)a.nq * nt + (int64_t)q * nt + ti, a.ttau[ti], vb);
          for (int c = 0; c < 3; ++c) vp[c] = pair_split(vb[c]);
        }
        // Rusanov flux, s_max = 2 max(|v+|, |v-|) pointwise (the square roots in binary64)
        float s1 = 0.0f, c1 = 0.0f, s2 = 0.0f, c2 = 0.0f, s3 = 0.0f, c3 = 0.0f, s4 = 0.0f, c4 = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pair_fma(vm[c], nP[c], s1, c1);
          pair_fma(vp[c], nP[c], s2, c2);
          pair_fma(vm[c], vm[c], s3, c3);
          pair_fma(vp[c], vp[c], s4, c4);
        }
        const float2 unm = pair_norm(s1, c1), unp = pair_norm(s2, c2);
        const double smax = 2.0 * fmax(sqrt(pair_value(s4, c4)), sqrt(pair_value(s3, c3)));
        const float2 W = pair_mul(wqP, a.twP[ti]);
        const float2 hs = pair_mul(W, pair_split(0.5 * smax));
        const float2 Wh = pair_mul(W, make_float2(0.5f, 0.0f));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          // h = W (0.5 (v+_c un+ + v-_c un-) - 0.5 s_max (v+_c - v-_c))
          const float2 cen = pair_mul(Wh, pair_add(pair_mul(vp[c], unp), pair_mul(vm[c], unm)));
          const float2 h = pair_add(cen, pair_neg(pair_mul(hs, pair_add(vp[c], pair_neg(vm[c])))));
          conv_fold<NGP>(Gu + c * NGP, h, g);
        }
      }
#pragma unroll 6
      for (int e = 0; e < 3 * NGP; ++e) Gu[e] = pair_norm(Gu[e].x, Gu[e].y);
    }
    __syncthreads();
    if (own) {
      float2 As[TG2], Ac[TG2];
#pragma unroll
      for (int m = 0; m < TG2; ++m) As[m] = Ac[m] = make_float2(0.0f, 0.0f);
#pragma unroll 1
      for (int v = 0; v < cnt; ++v) {
        const int P = base + v, f = P / nqf, q = P - f * nqf;
        const float2 fp = fphiP[((size_t)fcode[f] * nqf + q) * N + ok];
        conv_owner_acc<TG, NGP>(fp, Gf + ((size_t)v * 3 + oc) * NGP + ota0, As, Ac);
      }
      owner_flush(As, Ac);
    }
    __syncthreads();
  }
  if (own) {
#pragma unroll
    for (int t = 0; t < TG; ++t) a.ups[((size_t)oc * ne + i) * Nst + (ota0 + t) * N + ok] = accd[t];
  }
}

// tables transposed per block: out[b][c][r] = pair(in[b][r][c]) for nb blocks of R x C
__global__ void k_split_pairs_t(int64_t nb, int R, int C, const double* __restrict__ in, float2* __restrict__ out) {
  const int64_t per = (int64_t)R * C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nb * per; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per;
    const int rem = (int)(e - b * per), c = rem / R, r = rem - c * R;
    out[e] = pair_split(in[b * per + (int64_t)r * C + c]);
  }
}

// max |x[e]| over e >= skip
__global__ void k_maxabs(int64_t n, int64_t skip, const double* __restrict__ x, double* part) {
  double m = 0.0;
  for (int64_t e = skip + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, red[k]);
    part[blockIdx.x] = t;
  }
}
// out = a x + b y
__global__ void k_blend(int64_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = a * x[e] + b * y[e];
}
__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}

static FieldArg to_arg(const stdg_field& f, const double* modes = nullptr) {
  FieldArg a{};
  a.kind = f.kind; a.c[0] = f.c[0]; a.c[1] = f.c[1]; a.c[2] = f.c[2]; a.a = f.a; a.d = f.d; a.nu = f.nu;
  a.nmodes = f.kind == STDG_FIELD_CURL_MODES ? f.nmodes : 0;
  a.modes = modes;
  return a;
}

// Checks a stdg_field and, for STDG_FIELD_CURL_MODES, uploads its modes as rows (k, A, phi, 2 pi k x A).
static stdg_status field_prepare(stdg_solver* s, const stdg_field& f, double** modes_dev) {
  *modes_dev = nullptr;
  if (f.kind < STDG_FIELD_ZERO || f.kind > STDG_FIELD_CURL_MODES) { set_error("unknown field kind %d", f.kind); return STDG_EINVAL; }
  if (f.kind != STDG_FIELD_CURL_MODES) return STDG_OK;
  if (!f.modes || f.nmodes < 1 || f.nmodes > 256) { set_error("STDG_FIELD_CURL_MODES needs 1..256 modes"); return STDG_EINVAL; }
  std::vector<double> h((size_t)f.nmodes * 10);
  const double tp = 2.0 * 3.14159265358979323846;
  for (int m = 0; m < f.nmodes; ++m) {
    const double* k = f.modes + 7 * m;
    double* o = h.data() + 10 * m;
    for (int c = 0; c < 7; ++c) o[c] = k[c];
    o[7] = tp * (k[1] * k[5] - k[2] * k[4]);
    o[8] = tp * (k[2] * k[3] - k[0] * k[5]);
    o[9] = tp * (k[0] * k[4] - k[1] * k[3]);
  }
  stdg_status e = dev_alloc(s, (void**)modes_dev, h.size() * sizeof(double));
  if (e != STDG_OK) return e;
  if (cudaMemcpy(*modes_dev, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("field mode upload failed"); return STDG_ECUDA;
  }
  return STDG_OK;
}

// boundary data of the current step: the device field kind, or the host callback's table
static FieldArg bc_arg(const stdg_solver* s) {
  FieldArg a = to_arg(s->bc, s->bc_modes);
  if (s->bc_fn) { a.kind = kFieldTable; a.table = s->bc_table; }
  return a;
}

static MultiIdx make_mi(int p) {
  MultiIdx mi{};
  std::vector<int> ex = multi_indices(p);
  for (size_t k = 0; k < ex.size(); ++k) mi.e[k] = (unsigned char)ex[k];
  return mi;
}

static stdg_status ensure_step(stdg_solver* s) {
  if (s->Vbar) return STDG_OK;
  const size_t nv = (size_t)s->nf * 3 * s->Nst * sizeof(double);
  const size_t nb = (size_t)s->ne * 3 * s->Nst * sizeof(double);
  const size_t np = (size_t)s->ne * s->Nst * sizeof(double);
  stdg_status e;
  for (double** p : {&s->Vbar, &s->Vbar_n, &s->Lam, &s->Ups, &s->rhsv})
    if ((e = dev_alloc(s, (void**)p, nb)) != STDG_OK) return e;
  for (double** p : {&s->F, &s->Vbc, &s->vtmp})
    if ((e = dev_alloc(s, (void**)p, nv)) != STDG_OK) return e;
  if ((e = dev_alloc(s, (void**)&s->Gbc, 3 * nv)) != STDG_OK) return e;
  for (double** p : {&s->bvec, &s->dp, &s->wk1, &s->wk2})
    if ((e = dev_alloc(s, (void**)p, np)) != STDG_OK) return e;
  cudaMemset(s->Vbc, 0, nv);
  cudaMemset(s->Gbc, 0, 3 * nv);
  return ensure_krylov(s);
}

static cudaError_t launch_boundary(stdg_solver* s, double t0, const FieldArg& fld) {
  if (fld.kind == STDG_FIELD_ZERO) {               // no-slip walls: every projection is exactly 0
    const size_t nv = (size_t)s->nf * 3 * s->Nst * sizeof(double);
    cudaMemsetAsync(s->Vbc, 0, nv, s->stream);
    cudaMemsetAsync(s->Gbc, 0, 3 * nv, s->stream);
    return cudaGetLastError();
  }
  const int CH = 64;
  size_t smem = ((size_t)CH * s->N * 2 + CH * 3) * sizeof(double);
  cudaFuncSetAttribute(k_boundary, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  ++s->nlaunch;
  k_boundary<<<(int)s->nf, 128, smem, s->stream>>>(
      s->N, s->Ng, s->nq_nl, s->nqf_nl, s->nt_nl, s->dm.left, s->dm.right, s->dm.fl, s->dm.bary, s->dm.J,
      s->dm.detJ, s->dm.fvx, s->dm.normal, s->dm.area, s->C, s->x0h, s->dr.tet_nl_xi, s->dr.tet_nl_w,
      s->dr.tri_nl_st, s->dr.tri_nl_w, s->d_ttau, s->d_tw, s->d_tg, make_mi(s->p), fld, t0, s->dt, s->bidx,
      s->Vbc, s->Gbc);
  return cudaGetLastError();
}

// Boundary data of the slab [t0, t0 + dt]; with a host callback its values at the collected points are
// evaluated first and uploaded (the previous step ended with a stream synchronisation, so the table
// and the host buffers are free).
static stdg_status boundary_data(stdg_solver* s, double t0) {
  if (s->bc_fn) {
    const size_t n = s->bc_pts.size() / 4;
    for (size_t k = 0; k < n; ++k) {
      for (int c = 0; c < 3; ++c) s->bc_xyzt[4 * k + c] = s->bc_pts[4 * k + c];
      s->bc_xyzt[4 * k + 3] = t0 + s->bc_pts[4 * k + 3] * s->dt;
    }
    s->bc_fn(s->bc_xyzt.data(), (int64_t)n, s->bc_uvw.data(), s->bc_user);
    if (cudaMemcpyAsync(s->bc_table, s->bc_uvw.data(), n * 3 * sizeof(double), cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess || cudaStreamSynchronize(s->stream) != cudaSuccess) {
      set_error("boundary data upload failed"); return STDG_ECUDA;
    }
  }
  if (launch_boundary(s, t0, bc_arg(s)) != cudaSuccess) { set_error("boundary data launch failed"); return STDG_ECUDA; }
  return STDG_OK;
}

static cudaError_t launch_initial(stdg_solver* s, const FieldArg& fld) {
  const int CH = 64;
  size_t smem = ((size_t)CH * s->N * 2 + CH * 3) * sizeof(double);
  cudaFuncSetAttribute(k_initial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  ++s->nlaunch;
  k_initial<<<(int)s->nf, 128, smem, s->stream>>>(s->N, s->Ng, s->nq_nl, s->dm.left, s->dm.right, s->dm.fvx,
                                                  s->dm.fshift, s->dm.bary, s->C, s->x0h, s->dr.tet_nl_xi, s->dr.tet_nl_w,
                                                  make_mi(s->p), fld, s->V);
  return cudaGetLastError();
}

static stdg_status initial_done(stdg_solver* s) {
  cudaMemsetAsync(s->P, 0, (size_t)s->ne * s->Nst * sizeof(double), s->stream);
  s->t = 0.0;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) { set_error("initial projection failed"); return STDG_ECUDA; }
  return STDG_OK;
}

}  // namespace stdg

using namespace stdg;

extern "C" stdg_status stdg_set_initial(stdg_solver* s, const stdg_field* f) {
  if (!s || !f) { set_error("stdg_set_initial: NULL argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  stdg_status e = ensure_step(s);
  if (e != STDG_OK) return e;
  double* modes = nullptr;
  if ((e = field_prepare(s, *f, &modes)) != STDG_OK) return e;
  if (launch_initial(s, to_arg(*f, modes)) != cudaSuccess) { set_error("initial projection launch failed"); return STDG_ECUDA; }
  e = initial_done(s);
  if (modes) dev_free(s, modes);
  return e;
}

extern "C" stdg_status stdg_set_initial_fn(stdg_solver* s, stdg_vel_fn fn, void* user) {
  if (!s || !fn) { set_error("stdg_set_initial_fn: NULL argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  stdg_status e = ensure_step(s);
  if (e != STDG_OK) return e;
  // the points at which k_initial evaluates the data: one pass recording them, the callback on the
  // host, then the projection reading the returned values
  const size_t npts = (size_t)s->nf * 2 * s->nq_nl;
  double *pts = nullptr, *vals = nullptr;
  if ((e = dev_alloc(s, (void**)&pts, npts * 4 * sizeof(double))) != STDG_OK) return e;
  if ((e = dev_alloc(s, (void**)&vals, npts * 3 * sizeof(double))) != STDG_OK) { dev_free(s, pts); return e; }
  FieldArg fa{};
  fa.kind = kFieldCollect; fa.collect = pts;
  cudaMemsetAsync(pts, 0, npts * 4 * sizeof(double), s->stream);
  std::vector<double> hp(npts * 4), hv(npts * 3, 0.0);
  cudaError_t ce = launch_initial(s, fa);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(hp.data(), pts, npts * 4 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce == cudaSuccess) {
    for (size_t k = 0; k < npts; ++k) hp[4 * k + 3] = 0.0;          // t = 0
    fn(hp.data(), (int64_t)npts, hv.data(), user);
    ce = cudaMemcpyAsync(vals, hv.data(), npts * 3 * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  }
  if (ce == cudaSuccess) {
    fa.kind = kFieldTable; fa.table = vals; fa.collect = nullptr;
    ce = launch_initial(s, fa);
  }
  e = ce == cudaSuccess ? initial_done(s) : (set_error("initial projection (callback data) failed: %s",
                                                       cudaGetErrorString(ce)), STDG_ECUDA);
  cudaStreamSynchronize(s->stream);
  dev_free(s, vals);
  dev_free(s, pts);
  return e;
}

extern "C" stdg_status stdg_set_boundary(stdg_solver* s, const stdg_field* f) {
  if (!s || !f) { set_error("stdg_set_boundary: NULL argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  double* modes = nullptr;
  stdg_status e = field_prepare(s, *f, &modes);
  if (e != STDG_OK) return e;
  if (s->bc_modes) { cudaStreamSynchronize(s->stream); dev_free(s, s->bc_modes); }
  s->bc = *f;
  s->bc.modes = nullptr;                         // the caller's host array is not kept
  s->bc_modes = modes;
  s->bc_fn = nullptr; s->bc_user = nullptr;
  return STDG_OK;
}

extern "C" stdg_status stdg_set_boundary_fn(stdg_solver* s, stdg_vel_fn fn, void* user) {
  if (!s || !fn) { set_error("stdg_set_boundary_fn: NULL argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  stdg_status e = ensure_step(s);
  if (e != STDG_OK) return e;
  const size_t npts = (size_t)s->nbd * (s->nq_nl + s->nqf_nl) * s->nt_nl;
  if (!s->bc_table && npts > 0 && (e = dev_alloc(s, (void**)&s->bc_table, npts * 3 * sizeof(double))) != STDG_OK)
    return e;
  double* pts = nullptr;
  if (npts > 0 && (e = dev_alloc(s, (void**)&pts, npts * 4 * sizeof(double))) != STDG_OK) return e;
  s->bc_pts.assign(npts * 4, 0.0);
  if (npts > 0) {
    // record the boundary points with the kernel that consumes their values (the convection reads the
    // face points of the same table); Vbc / Gbc are recomputed by the next step
    FieldArg fa{};
    fa.kind = kFieldCollect; fa.collect = pts;
    cudaError_t ce = launch_boundary(s, 0.0, fa);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(s->bc_pts.data(), pts, npts * 4 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
    dev_free(s, pts);
    if (ce != cudaSuccess) { set_error("boundary point collection failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  }
  s->bc_xyzt.assign(npts * 4, 0.0);
  s->bc_uvw.assign(npts * 3, 0.0);
  if (s->bc_modes) { dev_free(s, s->bc_modes); s->bc_modes = nullptr; }
  s->bc = stdg_field{};
  s->bc.kind = STDG_FIELD_ZERO;
  s->bc_fn = fn; s->bc_user = user;
  return STDG_OK;
}

// Profiling: an event on the solver's stream closing `phase` (-1: the start mark of a step).
static void phase_mark(stdg_solver* s, int phase) {
  if (!s->prof) return;
  if (s->phase_ev.empty()) {
    s->phase_ev.assign(64, nullptr);
    for (auto& e : s->phase_ev)
      if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; }
  }
  const size_t k = s->phase_of.size();
  if (k >= s->phase_ev.size() || !s->phase_ev[k]) return;
  cudaEventRecord(s->phase_ev[k], s->stream);
  s->phase_of.push_back(phase);
}
static void phase_fold(stdg_solver* s) {
  if (s->phase_of.size() < 2) { s->phase_of.clear(); return; }
  cudaEventSynchronize(s->phase_ev[s->phase_of.size() - 1]);
  for (size_t k = 1; k < s->phase_of.size(); ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->phase_ev[k - 1], s->phase_ev[k]) == cudaSuccess && s->phase_of[k] >= 0)
      s->phase_ms[s->phase_of[k]] += ms;
  }
  s->phase_of.clear();
}

extern "C" stdg_status stdg_set_theta(stdg_solver* s, double theta) {
  if (!s || !(theta >= 0.5 && theta <= 1.0)) { set_error("stdg_set_theta: theta must lie in [1/2, 1]"); return STDG_EINVAL; }
  if (theta != 1.0 && s->pt != 0) { set_error("stdg_set_theta: the theta method needs p_t = 0"); return STDG_EINVAL; }
  s->theta = theta;
  return STDG_OK;
}

// Ups = the convective term of Eq. convdg for the velocity averages vbar ([3][ne][Nst]) on the slab
// starting at s->t (boundary data of the current boundary field or callback table); builds the pair
// tables on first use.  Launches on s->stream.
static stdg_status convection(stdg_solver* s, const double* vbar, double* ups) {
  const int N = s->N, Ng = s->Ng, Nst = s->Nst, ne = (int)s->ne;
  cudaStream_t st = s->stream;
  stdg_status e;
  const size_t conv_smem = ((size_t)9 * Nst + (size_t)kConvCH * 9 * Ng) * sizeof(double);
  // compile-time kernels for the benchmarked degrees (p = 3, p_t = 1 and p = p_t = 4)
  const int conv_t = s->conv_generic || s->nt_nl > kMaxTimePts ? 0
                     : (N == 35 && Ng == 5)                    ? 1
                     : (N == 20 && Ng == 2)                    ? 2
                                                               : 0;
  if (conv_t == 1)
    cudaFuncSetAttribute(k_convection_t<35, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ConvT<35, 5>::kSmem);
  else if (conv_t == 2)
    cudaFuncSetAttribute(k_convection_t<20, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ConvT<20, 2>::kSmem);
  else
    cudaFuncSetAttribute(k_convection, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem);
  if (!s->cphiP) {                                  // the convection tables as binary32 pairs, once
    const size_t n1 = (size_t)s->nq_nl * N, n2 = (size_t)s->nq_nl * 3 * N, n3 = (size_t)64 * s->nqf_nl * N;
    const size_t n4 = (size_t)s->nt_nl * Ng, n5 = (size_t)s->nt_nl;
    if ((e = dev_alloc(s, (void**)&s->cphiP, (2 * n1 + n2 + 2 * n3 + n4 + n5) * sizeof(float2))) != STDG_OK) return e;
    s->cdphiP = s->cphiP + n1;
    s->cfphiP = s->cdphiP + n2;
    s->ctgP = s->cfphiP + n3;
    s->ctwP = s->ctgP + n4;
    s->cphiT = s->ctwP + n5;                        // transposed copies: [k][point], [code][k][point]
    s->cfphiT = s->cphiT + n1;
    s->nlaunch += 7;
    k_split_pairs<<<256, 256, 0, st>>>((int64_t)n1, s->dr.tet_nl_phi, s->cphiP);
    k_split_pairs<<<256, 256, 0, st>>>((int64_t)n2, s->dr.tet_nl_dphi, s->cdphiP);
    k_split_pairs<<<256, 256, 0, st>>>((int64_t)n3, s->dr.face_nl_phi, s->cfphiP);
    k_split_pairs<<<1, 64, 0, st>>>((int64_t)n4, s->d_tg, s->ctgP);
    k_split_pairs<<<1, 64, 0, st>>>((int64_t)n5, s->d_tw, s->ctwP);
    k_split_pairs_t<<<256, 256, 0, st>>>(1, s->nq_nl, N, s->dr.tet_nl_phi, s->cphiT);
    k_split_pairs_t<<<256, 256, 0, st>>>(64, s->nqf_nl, N, s->dr.face_nl_phi, s->cfphiT);
  }
  ConvArgs ca{ne, N, Ng, s->nq_nl, s->nqf_nl, s->nt_nl, s->dm.t2f, s->dm.t2n, s->dm.t2code, s->dm.left,
              s->dm.code_l, s->dm.code_r, s->dm.detJ, s->dm.Jinv, s->dm.normal, s->dm.area, s->dm.fvx,
              s->dr.tet_nl_phi, s->dr.tet_nl_dphi, s->dr.tet_nl_w, s->dr.face_nl_phi, s->dr.tri_nl_st,
              s->dr.tri_nl_w, s->d_ttau, s->d_tw, s->d_tg, bc_arg(s), s->t, s->dt, s->ctgP, s->ctwP, s->bidx,
              (s->nq_nl + s->nqf_nl) * s->nt_nl, vbar, ups};
  if (conv_t == 1)
    k_convection_t<35, 5><<<ne, kConvCH, ConvT<35, 5>::kSmem, st>>>(ca, s->cphiT, s->cdphiP, s->cfphiT, s->cfphiP);
  else if (conv_t == 2)
    k_convection_t<20, 2><<<ne, kConvCH, ConvT<20, 2>::kSmem, st>>>(ca, s->cphiT, s->cdphiP, s->cfphiT, s->cfphiP);
  else
    k_convection<<<ne, kConvCH, conv_smem, st>>>(ca, s->cphiP, s->cdphiP, s->cfphiP);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) { set_error("convection launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  return STDG_OK;
}

// averaging and face gradient: the pair-arithmetic kernels (support.cu) at the compile-time degrees,
// the binary64 ones above otherwise (the go back and the pressure right-hand side stay binary64)
static void step_average(stdg_solver* s, const double* in, double* out) {
  const int ne = (int)s->ne, N = s->N, Ng = s->Ng;
  if (!support_fp64() &&
      sup_average(s->stream, ne, N, Ng, s->dm.t2f, s->dm.left, s->dm.detJ, s->Mij, in, out) != cudaErrorNotSupported)
    return;
  k_average<<<ne, 128, 0, s->stream>>>(ne, N, Ng, s->dm.t2f, s->dm.left, s->dm.detJ, s->Mij, in, out);
}
static void step_face_grad(stdg_solver* s, const double* P, MArg Ki, double* G) {
  const int nf = (int)s->nf, N = s->N, Ng = s->Ng, Nst = s->Nst;
  if (!support_fp64() && sup_face_grad(s->stream, nf, N, Ng, s->dm.left, s->dm.right, s->Q, P, s->dt, s->Kinv.data(),
                                       G) != cudaErrorNotSupported)
    return;
  k_face_grad<<<nf, 128, 3 * Nst * sizeof(double), s->stream>>>(N, Ng, s->dm.left, s->dm.right, s->Q, P, s->dt, Ki, G);
}

extern "C" stdg_status stdg_step(stdg_solver* s, double nu, int n_picard, int method, double tol,
                                 stdg_step_stats* stats) {
  if (!s || n_picard < 1 || n_picard > 8 || !(tol > 0.0) || nu < 0.0) { set_error("stdg_step: invalid argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  auto t_start = std::chrono::steady_clock::now();
  stdg_status e = ensure_step(s);
  if (e != STDG_OK) return e;
  const int N = s->N, Ng = s->Ng, Nst = s->Nst;
  const int ne = (int)s->ne, nf = (int)s->nf;
  const int64_t np = (int64_t)ne * Nst;
  cudaStream_t st = s->stream;
  GArg g0{}, g1{};
  MArg K{}, Ki{};
  for (int a = 0; a < Ng; ++a) { g0.v[a] = s->g0[a]; g1.v[a] = s->g1[a]; }
  for (int q = 0; q < Ng * Ng; ++q) { K.v[q] = s->K[q]; Ki.v[q] = s->Kinv[q]; }
  stdg_step_stats local{};
  s->phase_of.clear();
  phase_mark(s, -1);
  // previous slab average and new-slab boundary data
  ++s->nlaunch;
  step_average(s, s->V, s->Vbar_n);
  if ((e = boundary_data(s, s->t)) != STDG_OK) return e;
  // step 0: v^{n+1,0}(x, tau) = v^n(x, 1), p^{n+1,0} = 0
  ++s->nlaunch;
  k_trace<<<1216, 256, 0, st>>>(nf, N, Ng, s->dm.right, g1, s->V, s->Vbc, s->vtmp);
  cudaMemcpyAsync(s->V, s->vtmp, (size_t)nf * 3 * Nst * sizeof(double), cudaMemcpyDeviceToDevice, st);
  const double th = s->theta;
  if (th != 1.0) {                                  // theta method: keep p^n
    if (!s->Pn && (e = dev_alloc(s, (void**)&s->Pn, np * sizeof(double))) != STDG_OK) return e;
    if (!s->Pth && (e = dev_alloc(s, (void**)&s->Pth, np * sizeof(double))) != STDG_OK) return e;
    cudaMemcpyAsync(s->Pn, s->P, np * sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
  cudaMemsetAsync(s->P, 0, np * sizeof(double), st);
  phase_mark(s, 0);
  for (int k = 0; k < n_picard; ++k) {
    // 1. averaging and previous-Picard pressure gradient
    ++s->nlaunch;
    step_average(s, s->V, s->Vbar);
    // Lambda of Eq. prevpress, of p^{n+theta,k} = theta p^{n+1,k} + (1 - theta) p^n (Eq. CS_16_theta)
    const double* Plam = s->P;
    if (th != 1.0) {
      ++s->nlaunch;
      k_blend<<<1216, 256, 0, st>>>(np, th, s->P, 1.0 - th, s->Pn, s->Pth);
      Plam = s->Pth;
    }
    ++s->nlaunch;
    step_face_grad(s, Plam, Ki, s->F);
    ++s->nlaunch;
    step_average(s, s->F, s->Lam);
    phase_mark(s, 1);
    // 2. convection
    ++s->nlaunch;
    if ((e = convection(s, s->Vbar, s->Ups)) != STDG_OK) return e;
    phase_mark(s, 2);
    // 3. viscous systems (Eq. A1_mod), one per component, initial guess vbar^{n+1,k}
    ++s->nlaunch;
    k_visc_rhs<<<ne, 128, 0, st>>>(ne, N, Ng, s->dm.t2f, s->dm.t2n, s->dm.detJ, s->Q, g0, g1, K, nu, s->Vbar_n,
                                   s->Ups, s->Lam, s->Gbc, s->rhsv);
    if (cudaGetLastError() != cudaSuccess) { set_error("step kernels failed to launch"); return STDG_ECUDA; }
    int vits = 0;
    for (int c = 0; c < 3; ++c) {
      int it = 0;
      double res = 0.0;
      e = solve_viscous(s, s->rhsv + (size_t)c * np, s->Vbar + (size_t)c * np, nu, tol, &it, &res);
      if (e != STDG_OK) return e;
      vits += it;
    }
    phase_mark(s, 3);
    // 4. goback
    ++s->nlaunch;
    k_goback<<<nf, 128, 0, st>>>(ne, N, Ng, s->dm.left, s->dm.right, s->Mij, s->Vbar, s->Vbc, s->F);
    // 5. pressure correction (Eq. A2_mod)
    ++s->nlaunch;
    if (launch_rhs(ne, N, Ng, s->dm.t2f, s->dm.left, s->Q, s->F, -s->dt, 1, s->bvec, st) != cudaSuccess) {
      set_error("rhs launch failed"); return STDG_ECUDA;
    }
    if (s->gnn && s->ah_nsnap > 0) {
      int tot = 0;
      e = stdg_gnn_harvest(s, s->bvec, s->ah_nsnap, s->ah_every, s->ah_max, &tot);
      if (e != STDG_OK) return e;
    }
    stdg_solve_stats ss{};
    phase_mark(s, 4);
    e = solve_pressure(s, s->bvec, s->dp, tol, method, &ss);
    if (e != STDG_OK) return e;
    phase_mark(s, 5);
    ++s->nlaunch;
    k_axpy<<<1216, 256, 0, st>>>(np, 1.0 / th, s->dp, s->P);     // dp is the increment of p^{n+theta}
    // 6. velocity update (Eq. A3_mod)
    ++s->nlaunch;
    if (launch_update(nf, N, Ng, s->dm.left, s->dm.right, s->Q, s->F, s->dp, s->dt, s->Kinv.data(), s->V, st) != cudaSuccess) {
      set_error("update launch failed"); return STDG_ECUDA;
    }
    phase_mark(s, 6);
    local.press_iters[k] = ss.iterations;
    local.fallbacks += ss.fallback;
    local.press_residual[k] = ss.rel_residual;
    local.visc_iters[k] = vits;
    local.picard = k + 1;
  }
  // diagnostics: discrete divergence Sum_j D_ij v_j on unpinned tets
  ++s->nlaunch;
  launch_rhs(ne, N, Ng, s->dm.t2f, s->dm.left, s->Q, s->V, -s->dt, 0, s->bvec, st);
  ++s->nlaunch;
  k_maxabs<<<256, 256, 0, st>>>(np, Nst, s->bvec, s->part);
  std::vector<double> part(256);
  cudaMemcpyAsync(s->hostbuf + 512, s->part, 256 * sizeof(double), cudaMemcpyDeviceToHost, st);
  phase_mark(s, 6);
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("step failed: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
  phase_fold(s);
  double mx = 0.0;
  for (int q = 0; q < 256; ++q) mx = std::fmax(mx, s->hostbuf[512 + q]);
  local.max_divergence = mx;
  s->t += s->dt;
  local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (stats) *stats = local;
  return STDG_OK;
}

// The convective term alone (Eq. convdg) for given velocity averages, on the slab that starts at the
// solver's current time.
extern "C" stdg_status stdg_convection(stdg_solver* s, const double* vbar, double* ups) {
  if (!s || !vbar || !ups) { set_error("stdg_convection: NULL argument"); return STDG_EINVAL; }
  if (s->bc_fn) { set_error("stdg_convection: the boundary data come from a host callback (evaluated per step only)"); return STDG_EUNSUPPORTED; }
  cudaSetDevice(s->device);
  stdg_status e = ensure_step(s);
  if (e != STDG_OK) return e;
  ++s->nlaunch;
  if ((e = convection(s, vbar, ups)) != STDG_OK) return e;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
    set_error("stdg_convection: %s", cudaGetErrorString(cudaGetLastError()));
    return STDG_ECUDA;
  }
  return STDG_OK;
}
