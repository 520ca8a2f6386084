// Preprocessing on the device (the paper precomputes and stores every coefficient matrix,
// Sec. 2.8 and Sec. 4): per face j and side i in {l(j), r(j)}
//   psi_hat   Taylor monomials of Eq. bf_2 on the dual cell, Gram-Schmidt orthonormalised
//             (two Cholesky passes of their Gram matrix; the second restores orthonormality
//             lost to the Gram matrix's conditioning).
//   Q^sp_ij   int_{T_ij} psi_m d_c phi_l - sigma_ij n_c int_{Gamma_j} psi_m phi_l   (Eq. MD_6)
//   M^sp_ij   int_{T_ij} phi_k psi_l                                               (Eq. vis3)
// and the assembled spatial five-point blocks of Sum_j D_ij M_j^-1 Q (Eq. CS_19) with
// D = -Q^T and orthonormal psi (M_j^sp = I):
//   A_lr = -Sum_c Q_l^cT Q_r^c,  B_i = -Sum_{j in S_i interior} Sum_c Q_ij^cT Q_ij^c,
//   Bvisc_i = +Sum_{j in S_i boundary} Sum_c Q_ij^cT Q_ij^c (Dirichlet ghost, viscous only).
#include "dev.cuh"

namespace stdg {

struct FaceArgs {
  DevMesh m;
  DevRef r;
  int p, N, nq, nqf;
  MultiIdx mi;
  double *Q, *Mij, *C, *x0h;
};

// In-place Cholesky-inverse of the symmetric positive definite N x N matrix G (row-major,
// shared memory): on exit Cinv = L^-1 (lower triangular), G is overwritten by L.
__device__ void chol_inverse(double* G, double* Cinv, int N) {
  for (int k = 0; k < N; ++k) {
    if (threadIdx.x == 0) G[k * N + k] = sqrt(G[k * N + k]);
    __syncthreads();
    const double d = G[k * N + k];
    for (int i = k + 1 + threadIdx.x; i < N; i += blockDim.x) G[i * N + k] /= d;
    __syncthreads();
    const int rem = N - k - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      int i = k + 1 + idx / rem, jj = k + 1 + idx % rem;
      if (jj <= i) G[i * N + jj] -= G[i * N + k] * G[jj * N + k];
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    for (int i = 0; i < c; ++i) Cinv[i * N + c] = 0.0;
    Cinv[c * N + c] = 1.0 / G[c * N + c];
    for (int i = c + 1; i < N; ++i) {
      double s = 0.0;
      for (int k = c; k < i; ++k) s += G[i * N + k] * Cinv[k * N + c];
      Cinv[i * N + c] = -s / G[i * N + i];
    }
  }
  __syncthreads();
}

// rows[q] <- Lo rows[q] for a lower-triangular Lo (in place, descending m).
__device__ void apply_lower(const double* Lo, double* rows, int nrows, int N) {
  for (int q = threadIdx.x; q < nrows; q += blockDim.x) {
    double* t = rows + (size_t)q * N;
    for (int m = N - 1; m >= 0; --m) {
      double s = 0.0;
      for (int n = 0; n <= m; ++n) s += Lo[m * N + n] * t[n];
      t[m] = s;
    }
  }
  __syncthreads();
}

__device__ void gram(const double* T, const double* w, int nrows, int N, double* G) {
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int a = idx / N, b = idx % N;
    double s = 0.0;
    for (int q = 0; q < nrows; ++q) s += w[q] * T[q * N + a] * T[q * N + b];
    G[idx] = s;
  }
  __syncthreads();
}

__device__ inline double ipow(double x, int e) {
  double r = 1.0;
  for (int k = 0; k < e; ++k) r *= x;
  return r;
}

__global__ void __launch_bounds__(256) k_face_blocks(FaceArgs a) {
  extern __shared__ double sm[];
  __shared__ double geo[4];
  const int j = blockIdx.x;
  const int N = a.N, nq = a.nq, nqf = a.nqf;
  const int l = a.m.left[j], r = a.m.right[j];
  const int nsides = r >= 0 ? 2 : 1;
  const int nqt = nq * nsides;
  double* T = sm;
  double* wq = T + (size_t)nqt * N;
  double* Tf = wq + nqt;
  double* wf = Tf + (size_t)nqf * N;
  double* G = wf + nqf;
  double* C1 = G + N * N;
  double* C2 = C1 + N * N;
  const double* fv = a.m.fvx + 9 * (size_t)j;
  // the dual cell in l(j)'s frame: points of r(j) are shifted by fshift (periodic meshes)
  const double* sh = a.m.fshift + 3 * (size_t)j;
  if (threadIdx.x == 0) {
    double vt = 0.0, cen[3] = {0, 0, 0};
    for (int s = 0; s < nsides; ++s) {
      int t = s ? r : l;
      double v = a.m.detJ[t] / 24.0;
      for (int d = 0; d < 3; ++d)
        cen[d] += v * 0.25 * (fv[d] + fv[3 + d] + fv[6 + d] + a.m.bary[3 * t + d] + (s ? sh[d] : 0.0));
      vt += v;
    }
    for (int d = 0; d < 3; ++d) cen[d] /= vt;
    double h = 0.0;
    for (int k = 0; k < 3 + nsides; ++k) {
      const double* P = k < 3 ? fv + 3 * k : a.m.bary + 3 * (k == 3 ? l : r);
      for (int d = 0; d < 3; ++d) h = fmax(h, fabs(P[d] + (k == 4 ? sh[d] : 0.0) - cen[d]));
    }
    geo[0] = cen[0]; geo[1] = cen[1]; geo[2] = cen[2]; geo[3] = h;
  }
  __syncthreads();
  const double x0 = geo[0], y0 = geo[1], z0 = geo[2], hinv = 1.0 / geo[3];
  // volume quadrature points of T_lj (and T_rj) and the Taylor monomials there
  for (int idx = threadIdx.x; idx < nqt; idx += blockDim.x) {
    int s = idx / nq, q = idx % nq;
    int t = s ? r : l, f = s ? a.m.fr[j] : a.m.fl[j];
    const double* xi = a.r.sub_lin_xi + 3 * ((size_t)f * nq + q);
    const double* Jt = a.m.J + 9 * (size_t)t;
    const double* X0 = a.m.X0 + 3 * (size_t)t;
    double x[3];
    for (int d = 0; d < 3; ++d)
      x[d] = X0[d] + Jt[3 * d] * xi[0] + Jt[3 * d + 1] * xi[1] + Jt[3 * d + 2] * xi[2] + (s ? sh[d] : 0.0);
    wq[idx] = a.m.detJ[t] * a.r.sub_lin_w[f * nq + q];
    double yx = (x[0] - x0) * hinv, yy = (x[1] - y0) * hinv, yz = (x[2] - z0) * hinv;
    for (int mm = 0; mm < N; ++mm)
      T[(size_t)idx * N + mm] = ipow(yx, a.mi.e[3 * mm]) * ipow(yy, a.mi.e[3 * mm + 1]) * ipow(yz, a.mi.e[3 * mm + 2]);
  }
  // canonical face quadrature points
  const double area2 = 2.0 * a.m.area[j];
  for (int q = threadIdx.x; q < nqf; q += blockDim.x) {
    double s = a.r.tri_lin_st[2 * q], t = a.r.tri_lin_st[2 * q + 1], x[3];
    for (int d = 0; d < 3; ++d) x[d] = fv[d] + s * (fv[3 + d] - fv[d]) + t * (fv[6 + d] - fv[d]);
    wf[q] = area2 * a.r.tri_lin_w[q];
    double yx = (x[0] - x0) * hinv, yy = (x[1] - y0) * hinv, yz = (x[2] - z0) * hinv;
    for (int mm = 0; mm < N; ++mm)
      Tf[(size_t)q * N + mm] = ipow(yx, a.mi.e[3 * mm]) * ipow(yy, a.mi.e[3 * mm + 1]) * ipow(yz, a.mi.e[3 * mm + 2]);
  }
  __syncthreads();
  // two Gram-Schmidt (Cholesky) passes
  gram(T, wq, nqt, N, G);
  chol_inverse(G, C1, N);
  apply_lower(C1, T, nqt, N);
  gram(T, wq, nqt, N, G);
  chol_inverse(G, C2, N);
  apply_lower(C2, T, nqt, N);
  // combined coefficients C = C2 C1 (into G), applied to the face points
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int m = idx / N, n = idx % N;
    double s = 0.0;
    for (int k = n; k <= m; ++k) s += C2[m * N + k] * C1[k * N + n];
    G[idx] = (n <= m) ? s : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) a.C[(size_t)j * N * N + idx] = G[idx];
  if (threadIdx.x < 4) a.x0h[4 * (size_t)j + threadIdx.x] = geo[threadIdx.x];
  apply_lower(G, Tf, nqf, N);
  const double* nj = a.m.normal + 3 * (size_t)j;
  const size_t NN = (size_t)N * N;
  for (int s = 0; s < nsides; ++s) {
    const int t = s ? r : l, f = s ? a.m.fr[j] : a.m.fl[j];
    const int code = s ? a.m.code_r[j] : a.m.code_l[j];
    const double sig = s ? -1.0 : 1.0;
    const double* Ji = a.m.Jinv + 9 * (size_t)t;
    const double* Ts = T + (size_t)s * nq * N;
    const double* ws = wq + s * nq;
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int m = idx / N, ll = idx % N;
      double r0 = 0.0, r1 = 0.0, r2 = 0.0, mm = 0.0, fs = 0.0;
      for (int q = 0; q < nq; ++q) {
        const double wpsi = ws[q] * Ts[(size_t)q * N + m];
        const double* dp = a.r.sub_lin_dphi + ((size_t)f * nq + q) * 3 * N;
        r0 += wpsi * dp[ll];
        r1 += wpsi * dp[N + ll];
        r2 += wpsi * dp[2 * N + ll];
        mm += ws[q] * a.r.sub_lin_phi[((size_t)f * nq + q) * N + m] * Ts[(size_t)q * N + ll];
      }
      for (int q = 0; q < nqf; ++q)
        fs += wf[q] * Tf[(size_t)q * N + m] * a.r.face_lin_phi[((size_t)code * nqf + q) * N + ll];
      for (int c = 0; c < 3; ++c) {
        // grad_x phi = J^-T grad_xi phi:  d_c = Sum_d Jinv[d][c] d_d
        const double qv = Ji[c] * r0 + Ji[3 + c] * r1 + Ji[6 + c] * r2;
        const size_t base = ((size_t)j * 2 * 3) * NN;
        if (nsides == 2) {
          a.Q[base + ((size_t)s * 3 + c) * NN + idx] = qv - sig * nj[c] * fs;
        } else {
          a.Q[base + (size_t)c * NN + idx] = qv - nj[c] * fs;        // with the face term
          a.Q[base + (size_t)(3 + c) * NN + idx] = qv;               // volume part alone
        }
      }
      a.Mij[((size_t)j * 2 + s) * NN + idx] = mm;
      if (nsides == 1) a.Mij[((size_t)j * 2 + 1) * NN + idx] = 0.0;
    }
    __syncthreads();
  }
}

cudaError_t launch_face_blocks(const DevMesh& m, const DevRef& r, int p, int N, int nq, int nqf,
                               const MultiIdx& mi, double* Q, double* Mij, double* C, double* x0h,
                               cudaStream_t st) {
  FaceArgs a{m, r, p, N, nq, nqf, mi, Q, Mij, C, x0h};
  size_t smem = ((size_t)2 * nq * N + 2 * nq + (size_t)nqf * N + nqf + 3 * (size_t)N * N) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_face_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (m.nf > 0) k_face_blocks<<<m.nf, 256, smem, st>>>(a);
  return cudaGetLastError();
}

// A_lr[k][l] = -Sum_c Sum_m Q_l^c[m][k] Q_r^c[m][l] for every interior face.
__global__ void k_offdiag(int nf, int N, const int* right, const double* Q, double* Aoff) {
  const int j = blockIdx.x;
  const size_t NN = (size_t)N * N;
  if (right[j] < 0) {
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) Aoff[j * NN + idx] = 0.0;
    return;
  }
  const double* Ql = Q + (size_t)j * 6 * NN;
  const double* Qr = Ql + 3 * NN;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int k = idx / N, ll = idx % N;
    double s = 0.0;
    for (int c = 0; c < 3; ++c)
      for (int m = 0; m < N; ++m) s += Ql[c * NN + m * N + k] * Qr[c * NN + m * N + ll];
    Aoff[j * NN + idx] = -s;
  }
}

// B_i = -Sum_{interior j in S_i} Sum_c Q_ij^cT Q_ij^c;  Bvisc_i = +Sum_{boundary j in S_i} (same, slot 0).
__global__ void k_diag(int ne, int N, const int* t2f, const int* t2n, const int* left,
                       const double* Q, double* Bdiag, double* Bvisc) {
  const int i = blockIdx.x;
  const size_t NN = (size_t)N * N;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int k = idx / N, ll = idx % N;
    double sb = 0.0, sv = 0.0;
    for (int f = 0; f < 4; ++f) {
      int j = t2f[4 * i + f];
      int s = (left[j] == i) ? 0 : 1;
      const double* Qs = Q + ((size_t)j * 6 + 3 * s) * NN;
      double acc = 0.0;
      for (int c = 0; c < 3; ++c)
        for (int m = 0; m < N; ++m) acc += Qs[c * NN + m * N + k] * Qs[c * NN + m * N + ll];
      if (t2n[4 * i + f] >= 0) sb -= acc; else sv += acc;
    }
    Bdiag[i * NN + idx] = sb;
    Bvisc[i * NN + idx] = sv;
  }
}

// Binv_i = S_ii^-1 for the symmetric positive definite diagonal block S_ii = -B_i of the pinned
// operator -A (tet 0: the pinned constant mode becomes an identity row and column).  Cholesky in
// shared memory: S = L L^T, S^-1 = L^-T L^-1.
__global__ void __launch_bounds__(128) k_block_inverse(int N, const double* __restrict__ Bdiag, double* __restrict__ Binv) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  const size_t NN = (size_t)N * N;
  double* G = sm;
  double* Ci = sm + NN;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int r = idx / N, c = idx % N;
    double v = -Bdiag[i * NN + idx];
    if (i == 0 && (r == 0 || c == 0)) v = (r == c) ? 1.0 : 0.0;
    G[idx] = v;
  }
  __syncthreads();
  chol_inverse(G, Ci, N);
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int r = idx / N, c = idx % N;
    double s = 0.0;
    for (int k = (r > c ? r : c); k < N; ++k) s += Ci[k * N + r] * Ci[k * N + c];
    Binv[i * NN + idx] = s;
  }
}

cudaError_t launch_block_inverse(int ne, int N, const double* Bdiag, double* Binv, cudaStream_t st) {
  size_t smem = 2 * (size_t)N * N * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_block_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (ne > 0) k_block_inverse<<<ne, 128, smem, st>>>(N, Bdiag, Binv);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const DevMesh& m, int N, const double* Q, double* Aoff, double* Bdiag,
                            double* Bvisc, cudaStream_t st) {
  if (m.nf > 0) k_offdiag<<<m.nf, 128, 0, st>>>(m.nf, N, m.right, Q, Aoff);
  if (m.ne > 0) k_diag<<<m.ne, 128, 0, st>>>(m.ne, N, m.t2f, m.t2n, m.left, Q, Bdiag, Bvisc);
  return cudaGetLastError();
}

}  // namespace stdg
