// Hot-path kernels of the pressure-correction step (Sec. 2.4, 2.6).
//  k_apply   : five-point block operator, tet-pull (each tet gathers its own row of blocks;
//              no atomics, so results are bitwise reproducible).
//  k_rhs     : right-hand side Sum_j D_ij F_j of Eq. A2_mod.
//  k_update  : velocity update of Eq. A3_mod.
//  k_moments : basis-independent velocity moments int phi~ v_h on each sub-tet (Eq. vis3).
#include "dev.cuh"

namespace stdg {

__global__ void __launch_bounds__(128) k_apply(ApplyArgs a, const double* __restrict__ x,
                                               double* __restrict__ y) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  const int N = a.N, Ng = a.Ng, Nst = N * Ng, Np = N + 1;
  const size_t NN = (size_t)N * N;
  double* blk = sm;                       // 5 x N x Np
  double* z = blk + 5 * N * Np;           // 5 x Nst
  double* acc = z + 5 * Nst;              // Nst
  __shared__ int nbr[5];
  __shared__ int src[5];
  __shared__ int trn[5];
  if (threadIdx.x < 5) {
    int sl = threadIdx.x;
    if (sl == 0) { nbr[0] = i; src[0] = -1; trn[0] = 0; }
    else {
      int f = sl - 1;
      int j = a.t2f[4 * i + f];
      int nb = a.t2n[4 * i + f];
      nbr[sl] = nb;
      src[sl] = j;
      trn[sl] = (a.left[j] == i) ? 0 : 1;   // A_{i,nb} = A_lr if i = l, A_lr^T if i = r
    }
  }
  __syncthreads();
  for (int sl = 0; sl < 5; ++sl) {
    if (nbr[sl] < 0) continue;
    const double* B = sl == 0 ? a.Bdiag + (size_t)i * NN : a.Aoff + (size_t)src[sl] * NN;
    const double* E = (sl == 0 && a.Bextra) ? a.Bextra + (size_t)i * NN : nullptr;
    double* dst = blk + sl * N * Np;
    const int t = trn[sl];
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      double v = B[idx];
      if (E) v += a.extra_coef * E[idx];
      int r = idx / N, c = idx % N;
      if (t) dst[c * Np + r] = v; else dst[r * Np + c] = v;
    }
    const double* xs = x + (size_t)nbr[sl] * Nst;
    for (int idx = threadIdx.x; idx < Nst; idx += blockDim.x) {
      double v = xs[idx];
      if (a.pinned && nbr[sl] == 0 && (idx % N) == 0) v = 0.0;
      z[sl * Nst + idx] = v;
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Nst; o += blockDim.x) {
    const int ta = o / N, k = o % N;
    double s = 0.0;
    for (int sl = 0; sl < 5; ++sl) {
      if (nbr[sl] < 0) continue;
      const double* br = blk + sl * N * Np + k * Np;
      const double* zz = z + sl * Nst + ta * N;
      for (int ll = 0; ll < N; ++ll) s = fma(br[ll], zz[ll], s);
    }
    acc[o] = s;
  }
  __syncthreads();
  const double dj = a.mass_coef != 0.0 ? a.detJ[i] : 0.0;
  for (int o = threadIdx.x; o < Nst; o += blockDim.x) {
    const int ta = o / N, k = o % N;
    double v;
    if (a.tacc_identity) v = acc[o];
    else {
      v = 0.0;
      for (int b = 0; b < Ng; ++b) v = fma(a.Tacc[ta * Ng + b], acc[b * N + k], v);
    }
    v *= a.scale;
    if (a.mass_coef != 0.0) {
      double mterm = 0.0;
      for (int b = 0; b < Ng; ++b) mterm = fma(a.Kmass[ta * Ng + b], z[b * N + k], mterm);
      v = fma(a.mass_coef * dj, mterm, v);
    }
    if (a.pinned && i == 0 && k == 0) v = a.pin_diag * x[o];
    y[(size_t)i * Nst + o] = v;
  }
}

cudaError_t launch_apply(const ApplyArgs& a, const double* x, double* y, cudaStream_t st) {
  const int N = a.N, Nst = a.N * a.Ng;
  size_t smem = ((size_t)5 * N * (N + 1) + 6 * (size_t)Nst) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (a.ne > 0) k_apply<<<a.ne, 128, smem, st>>>(a, x, y);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(128) k_rhs(int N, int Ng, const int* __restrict__ t2f,
                                             const int* __restrict__ left, const double* __restrict__ Q,
                                             const double* __restrict__ F, double coef, int pinned,
                                             double* __restrict__ b) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  const int Nst = N * Ng;
  const size_t NN = (size_t)N * N;
  double* Fs = sm;                        // 4 x 3 x Nst
  __shared__ int fj[4], fs[4];
  if (threadIdx.x < 4) {
    int j = t2f[4 * i + threadIdx.x];
    fj[threadIdx.x] = j;
    fs[threadIdx.x] = (left[j] == i) ? 0 : 1;
  }
  __syncthreads();
  for (int f = 0; f < 4; ++f)
    for (int idx = threadIdx.x; idx < 3 * Nst; idx += blockDim.x)
      Fs[f * 3 * Nst + idx] = F[(size_t)fj[f] * 3 * Nst + idx];
  __syncthreads();
  for (int o = threadIdx.x; o < Nst; o += blockDim.x) {
    const int ta = o / N, l = o % N;
    double s = 0.0;
    for (int f = 0; f < 4; ++f) {
      const double* Qs = Q + ((size_t)fj[f] * 6 + 3 * fs[f]) * NN;
      for (int c = 0; c < 3; ++c) {
        const double* Fc = Fs + (f * 3 + c) * Nst + ta * N;
        const double* Qc = Qs + c * NN + l;
        for (int m = 0; m < N; ++m) s = fma(Qc[(size_t)m * N], Fc[m], s);
      }
    }
    s *= coef;
    if (pinned && i == 0 && l == 0) s = 0.0;
    b[(size_t)i * Nst + o] = s;
  }
}

cudaError_t launch_rhs(int ne, int N, int Ng, const int* t2f, const int* left, const double* Q,
                       const double* F, double coef, int pinned, double* b, cudaStream_t st) {
  size_t smem = (size_t)12 * N * Ng * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_rhs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (ne > 0) k_rhs<<<ne, 128, smem, st>>>(N, Ng, t2f, left, Q, F, coef, pinned, b);
  return cudaGetLastError();
}

struct KinvArg { double v[kMaxNg * kMaxNg]; };

__global__ void __launch_bounds__(128) k_update(int N, int Ng, const int* __restrict__ left,
                                                const int* __restrict__ right, const double* __restrict__ Q,
                                                const double* __restrict__ F, const double* __restrict__ dp,
                                                double dt, KinvArg Ki, double* __restrict__ V) {
  extern __shared__ double sm[];
  const int j = blockIdx.x;
  const int Nst = N * Ng, Np = N + 1;
  const size_t NN = (size_t)N * N;
  const int l = left[j], r = right[j];
  const double* Fj = F + (size_t)j * 3 * Nst;
  double* Vj = V + (size_t)j * 3 * Nst;
  if (r < 0) {
    for (int idx = threadIdx.x; idx < 3 * Nst; idx += blockDim.x) Vj[idx] = Fj[idx];
    return;
  }
  double* Qs = sm;                  // 6 x N x Np
  double* ps = Qs + 6 * N * Np;     // 2 x Nst
  double* g = ps + 2 * Nst;         // 3 x Nst
  for (int idx = threadIdx.x; idx < 6 * N * N; idx += blockDim.x) {
    int blkid = idx / (N * N), rem = idx % (N * N);
    Qs[blkid * N * Np + (rem / N) * Np + rem % N] = Q[(size_t)j * 6 * NN + idx];
  }
  for (int idx = threadIdx.x; idx < Nst; idx += blockDim.x) {
    ps[idx] = dp[(size_t)l * Nst + idx];
    ps[Nst + idx] = dp[(size_t)r * Nst + idx];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    const int c = o / Nst, rem = o % Nst, b = rem / N, m = rem % N;
    double s = 0.0;
    for (int sd = 0; sd < 2; ++sd) {
      const double* qr = Qs + (sd * 3 + c) * N * Np + m * Np;
      const double* pp = ps + sd * Nst + b * N;
      for (int ll = 0; ll < N; ++ll) s = fma(qr[ll], pp[ll], s);
    }
    g[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 3 * Nst; o += blockDim.x) {
    const int c = o / Nst, rem = o % Nst, ta = rem / N, m = rem % N;
    double s = 0.0;
    for (int b = 0; b < Ng; ++b) s = fma(Ki.v[ta * Ng + b], g[c * Nst + b * N + m], s);
    Vj[o] = Fj[o] - dt * s;
  }
}

cudaError_t launch_update(int nf, int N, int Ng, const int* left, const int* right, const double* Q,
                          const double* F, const double* dp, double dt, const double* Kinv,
                          double* V, cudaStream_t st) {
  if (nf > 0 && !support_fp64()) {
    const cudaError_t ep = sup_update(st, nf, N, Ng, left, right, Q, F, dp, dt, Kinv, V);
    if (ep != cudaErrorNotSupported) return ep;
  }
  KinvArg k{};
  for (int q = 0; q < Ng * Ng; ++q) k.v[q] = Kinv[q];
  const int Nst = N * Ng;
  size_t smem = ((size_t)6 * N * (N + 1) + 5 * (size_t)Nst) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (nf > 0) k_update<<<nf, 128, smem, st>>>(N, Ng, left, right, Q, F, dp, dt, k, V);
  return cudaGetLastError();
}

__global__ void k_moments(int N, int Ng, const double* __restrict__ Mij, const double* __restrict__ V,
                          double dt, double* __restrict__ U) {
  const int j = blockIdx.x;
  const int Nst = N * Ng;
  const size_t NN = (size_t)N * N;
  for (int o = threadIdx.x; o < 2 * 3 * Nst; o += blockDim.x) {
    const int s = o / (3 * Nst), rem = o % (3 * Nst), c = rem / Nst, ta = (rem % Nst) / N, k = rem % N;
    const double* M = Mij + ((size_t)j * 2 + s) * NN + (size_t)k * N;
    const double* v = V + (size_t)j * 3 * Nst + c * Nst + ta * N;
    double acc = 0.0;
    for (int ll = 0; ll < N; ++ll) acc = fma(M[ll], v[ll], acc);
    U[(size_t)j * 6 * Nst + o] = dt * acc;
  }
}

cudaError_t launch_moments(int nf, int N, int Ng, const double* Mij, const double* V, double dt,
                           double* U, cudaStream_t st) {
  if (nf > 0) k_moments<<<nf, 128, 0, st>>>(N, Ng, Mij, V, dt, U);
  return cudaGetLastError();
}

}  // namespace stdg
