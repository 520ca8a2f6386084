// Learned right preconditioner: a message-passing network over tet-face adjacency, trained and
// applied on the device with hand-written forward, backward and Adam kernels.
//
//   s = RMS(r);  x_i = [r_i / s, g_i]
//   h0 = relu(We x + be);  m = gather_nbr(h^{l-1});  h^l = relu(Ws^l h^{l-1} + Wm^l m + b^l)
//   M(r) = s (Wd h^L + bd)
//
// Weights: binary32 master copy (Adam state binary32) and a working copy in bfloat16 (or binary32)
// used by the forward pass; all products accumulate in binary32.  The dense layers are
// [ne x K] x [K x O] products with K, O <= 2 * 64 + Nst: tiled 64 x 64 on CUDA cores (each
// layer is ~2 GFLOP at 2e5 tets, a few tens of microseconds).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "solver.h"

namespace stdg {

constexpr int kT = 64;    // tile of rows (tets) and of outputs
constexpr int kK = 32;    // reduction chunk

template <typename TW>
__device__ __forceinline__ float wload(const TW* w, size_t i);
template <>
__device__ __forceinline__ float wload<float>(const float* w, size_t i) { return w[i]; }
template <>
__device__ __forceinline__ float wload<__nv_bfloat16>(const __nv_bfloat16* w, size_t i) { return __bfloat162float(w[i]); }

// Y[i][o] (+)= Sum_k A[i][k] W(o, k) (+ b[o]); W(o,k) = W[o*K + k] (wt == 0) or W[k*O + o] (wt == 1).
// relu: Y = max(.,0) and, if pre != nullptr, the pre-activation is stored there.
template <typename TW>
__global__ void __launch_bounds__(256) k_dense(int ne, int K, int O, const float* __restrict__ A, const TW* __restrict__ W,
                                               int wt, const float* __restrict__ b, int accumulate, int relu,
                                               float* __restrict__ pre, float* __restrict__ Y) {
  __shared__ float As[kT][kK + 1];
  __shared__ float Ws[kT][kK + 1];
  const int i0 = blockIdx.x * kT, o0 = blockIdx.y * kT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 16 x 16 threads, 4 x 4 outputs each
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kK) {
    for (int idx = threadIdx.x; idx < kT * kK; idx += blockDim.x) {
      const int r = idx / kK, c = idx % kK;
      const int i = i0 + r, k = k0 + c, o = o0 + r;
      As[r][c] = (i < ne && k < K) ? A[(size_t)i * K + k] : 0.0f;
      Ws[r][c] = (o < O && k < K) ? (wt ? wload<TW>(W, (size_t)k * O + o) : wload<TW>(W, (size_t)o * K + k)) : 0.0f;
    }
    __syncthreads();
    for (int c = 0; c < kK; ++c) {
      float a[4], w[4];
      for (int q = 0; q < 4; ++q) { a[q] = As[ty * 4 + q][c]; w[q] = Ws[tx * 4 + q][c]; }
      for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], w[q], acc[p][q]);
    }
    __syncthreads();
  }
  for (int p = 0; p < 4; ++p)
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ty * 4 + p, o = o0 + tx * 4 + q;
      if (i >= ne || o >= O) continue;
      float v = acc[p][q] + (b ? b[o] : 0.0f);
      const size_t idx = (size_t)i * O + o;
      if (accumulate) v += Y[idx];
      if (relu) {
        if (pre) pre[idx] = v;
        v = fmaxf(v, 0.0f);
      }
      Y[idx] = v;
    }
}

// m_i = Sum_{f} h_{nbr(i,f)}  (symmetric adjacency: also the adjoint of itself)
__global__ void k_gather(int ne, int H, const int* __restrict__ nbr4, const float* __restrict__ h, float* __restrict__ m) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)ne * H; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / H;
    const int c = (int)(e % H);
    float s = 0.0f;
    for (int f = 0; f < 4; ++f) {
      const int n = nbr4[4 * i + f];
      if (n >= 0) s += h[(size_t)n * H + c];
    }
    m[e] = s;
  }
}

// dpre = dh * (pre > 0)
__global__ void k_relu_back(int64_t n, const float* __restrict__ pre, const float* __restrict__ dh, float* __restrict__ dpre) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dpre[e] = pre[e] > 0.0f ? dh[e] : 0.0f;
}

// Weight gradient partials: part[chunk][o][k] = Sum_{i in chunk} D[i][o] X[i][k]; bias partial
// (k == K slot) = Sum_i D[i][o].  Fixed chunking -> deterministic after k_wgrad_reduce.
constexpr int kChunk = 1024;
__global__ void __launch_bounds__(256) k_wgrad(int ne, int O, int K, const float* __restrict__ D, const float* __restrict__ X,
                                               float* __restrict__ part) {
  __shared__ float Ds[kK][kT + 1];
  __shared__ float Xs[kK][kT + 1];
  const int chunk = blockIdx.x, o0 = blockIdx.y * kT, k0 = blockIdx.z * kT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  float bacc[4] = {0, 0, 0, 0};
  const int ibeg = chunk * kChunk, iend = min(ne, ibeg + kChunk);
  for (int i0 = ibeg; i0 < iend; i0 += kK) {
    for (int idx = threadIdx.x; idx < kK * kT; idx += blockDim.x) {
      const int r = idx / kT, c = idx % kT;
      const int i = i0 + r;
      Ds[r][c] = (i < iend && o0 + c < O) ? D[(size_t)i * O + o0 + c] : 0.0f;
      Xs[r][c] = (i < iend && k0 + c < K) ? X[(size_t)i * K + k0 + c] : 0.0f;
    }
    __syncthreads();
    for (int r = 0; r < kK; ++r) {
      float d[4], x[4];
      for (int q = 0; q < 4; ++q) { d[q] = Ds[r][ty * 4 + q]; x[q] = Xs[r][tx * 4 + q]; }
      for (int p = 0; p < 4; ++p) {
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(d[p], x[q], acc[p][q]);
        if (blockIdx.z == 0 && tx == 0) bacc[p] += d[p];
      }
    }
    __syncthreads();
  }
  const size_t stride = (size_t)O * (K + 1);
  for (int p = 0; p < 4; ++p) {
    const int o = o0 + ty * 4 + p;
    if (o >= O) continue;
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + tx * 4 + q;
      if (k < K) part[chunk * stride + (size_t)o * (K + 1) + k] = acc[p][q];
    }
    if (blockIdx.z == 0 && tx == 0) part[chunk * stride + (size_t)o * (K + 1) + K] = bacc[p];
  }
}
// out_W[o][k] (+)= Sum_chunks part; out_b[o] (+)= Sum_chunks part[..][K]
__global__ void k_wgrad_reduce(int nchunk, int O, int K, const float* __restrict__ part, float scale, float* __restrict__ gW,
                               float* __restrict__ gb) {
  const size_t stride = (size_t)O * (K + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)stride; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < nchunk; ++c) s += part[c * stride + e];
    const int o = (int)(e / (K + 1)), k = (int)(e % (K + 1));
    if (k < K) gW[(size_t)o * K + k] += scale * s;
    else if (gb) gb[o] += scale * s;
  }
}

// Adam on the binary32 master weights; refresh the working copy.
template <typename TW>
__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       TW* __restrict__ wc);
template <>
__global__ void k_adam<float>(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                              float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                              float* __restrict__ wc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    m[e] = b1 * m[e] + (1 - b1) * g[e];
    v[e] = b2 * v[e] + (1 - b2) * g[e] * g[e];
    w[e] -= lr * (m[e] / c1) / (sqrtf(v[e] / c2) + eps);
    wc[e] = w[e];
  }
}
template <>
__global__ void k_adam<__nv_bfloat16>(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                      float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                                      __nv_bfloat16* __restrict__ wc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    m[e] = b1 * m[e] + (1 - b1) * g[e];
    v[e] = b2 * v[e] + (1 - b2) * g[e] * g[e];
    w[e] -= lr * (m[e] / c1) / (sqrtf(v[e] / c2) + eps);
    wc[e] = __float2bfloat16_rn(w[e]);
  }
}

}  // namespace stdg

namespace stdg {

// features: X[i] = [r_i / s, g_i], s = sqrt(mean r^2) (device scalar, written by k_gnn_scale)
__global__ void k_gnn_sumsq(int64_t n, const double* __restrict__ r, double* part) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc = fma(r[e], r[e], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}
__global__ void k_gnn_scale(int nparts, const double* part, int64_t n, double* s_out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < nparts; ++k) t += part[k];
    const double s = sqrt(t / (double)n);
    s_out[0] = s > 0.0 ? s : 1.0;
  }
}
__global__ void k_gnn_features(int ne, int C, int G, const double* __restrict__ r, const float* __restrict__ geom,
                               const double* __restrict__ s, float* __restrict__ X) {
  const int F = C + G;
  const double inv = 1.0 / s[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)ne * F; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / F;
    const int c = (int)(e % F);
    X[e] = c < C ? (float)(r[i * C + c] * inv) : geom[i * G + (c - C)];
  }
}
// z = s * out (+ z_in)
__global__ void k_gnn_output(int64_t n, const float* __restrict__ out, const double* __restrict__ s, int add,
                             double* __restrict__ z) {
  const double sc = s[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    z[e] = (add ? z[e] : 0.0) + sc * (double)out[e];
}
// z += s * out where the network output is finite; a non-finite output leaves z unchanged there and
// sets *bad (the correction is then not used for that entry)
__global__ void k_gnn_correct(int64_t n, const float* __restrict__ out, const double* __restrict__ s,
                              double* __restrict__ z, int* bad) {
  const double sc = s[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = sc * (double)out[e];
    if (isfinite(v)) z[e] += v;
    else *bad = 1;
  }
}
// t = -x (- z): a harvested target before the final solution is added
__global__ void k_neg_sum(int64_t n, const double* __restrict__ x, const double* __restrict__ z, double* __restrict__ t) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    t[e] = -(x[e] + (z ? z[e] : 0.0));
}
__global__ void k_sub2(int64_t n, const double* __restrict__ a, double* __restrict__ b) {   // b = a - b
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) b[e] = a[e] - b[e];
}
__global__ void k_axpy_d(int64_t n, double al, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) y[e] = fma(al, x[e], y[e]);
}
// loss terms of one pair: diff = s out - t; part0 = Sum diff^2, part1 = Sum t^2; dout = diff * s (scaled later)
__global__ void k_gnn_lossdiff(int64_t n, const float* __restrict__ out, const double* __restrict__ s,
                               const double* __restrict__ t, float* __restrict__ dout, double* part) {
  double a = 0.0, b = 0.0;
  const double sc = s[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double d = sc * (double)out[e] - t[e];
    a = fma(d, d, a);
    b = fma(t[e], t[e], b);
    dout[e] = (float)(d * sc);
  }
  for (int o = 16; o > 0; o >>= 1) { a += __shfl_down_sync(0xffffffffu, a, o); b += __shfl_down_sync(0xffffffffu, b, o); }
  __shared__ double ra[8], rb[8];
  if ((threadIdx.x & 31) == 0) { ra[threadIdx.x >> 5] = a; rb[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { ta += ra[k]; tb += rb[k]; }
    part[2 * blockIdx.x] = ta;
    part[2 * blockIdx.x + 1] = tb;
  }
}
__global__ void k_scale_f(int64_t n, const double* __restrict__ part2, int nparts, float* __restrict__ v, double* loss) {
  // v *= 2 / Sum t^2 ; loss += Sum diff^2 / Sum t^2  (one thread finishes the reduction first)
  __shared__ double fac;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nparts; ++k) { a += part2[2 * k]; b += part2[2 * k + 1]; }
    fac = b > 0.0 ? 2.0 / b : 0.0;
    if (blockIdx.x == 0) loss[0] += b > 0.0 ? a / b : 0.0;
  }
  __syncthreads();
  const float f = (float)fac;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) v[e] *= f;
}
__global__ void k_fadd(int64_t n, const float* __restrict__ a, float* __restrict__ b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) b[e] += a[e];
}
__global__ void k_to_bf16(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = __float2bfloat16_rn(a[e]);
}

// Full-operator block Jacobi: z_i = A_ii^-1 r_i = -(Binv_i (x) Tp^-1) r_i; pinned entries z = -r.
__global__ void __launch_bounds__(128) k_bj_full(int N, int Ng, const double* __restrict__ Binv, const double* Tpinv,
                                                 const double* __restrict__ r, double* __restrict__ z) {
  extern __shared__ double rs[];
  const int i = blockIdx.x, Nst = N * Ng;
  const size_t NN = (size_t)N * N;
  double* u = rs + Nst;
  for (int o = threadIdx.x; o < Nst; o += blockDim.x) rs[o] = r[(size_t)i * Nst + o];
  __syncthreads();
  for (int o = threadIdx.x; o < Nst; o += blockDim.x) {
    const int b = o / N, k = o % N;
    const double* B = Binv + (size_t)i * NN + k;
    double s = 0.0;
    for (int l = 0; l < N; ++l) s = fma(B[(size_t)l * N], rs[b * N + l], s);
    u[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Nst; o += blockDim.x) {
    const int a = o / N, k = o % N;
    double s = 0.0;
    for (int b = 0; b < Ng; ++b) s = fma(Tpinv[a * Ng + b], u[b * N + k], s);
    z[(size_t)i * Nst + o] = (i == 0 && k == 0) ? -rs[o] : -s;
  }
}

}  // namespace stdg

namespace stdg {

static cudaStream_t S(stdg_solver* s) { return s->stream; }
static const int kGB = 1216;

template <typename TW>
static void dense(stdg_solver* s, int K, int O, const float* A, const void* W, int wt, const float* b, int acc, int relu,
                  float* pre, float* Y) {
  const int ne = (int)s->ne;
  ++s->nlaunch;
  if constexpr (sizeof(TW) == 2) {
    // bfloat16 weights: the product on the tensor cores (activations rounded to bfloat16, binary32 sums)
    TcGemmArgs a{};
    a.M = ne; a.N = O; a.K = K; a.ksplit = 0;
    a.A = A; a.sAm = K; a.sAk = 1;
    a.B = W; a.b_bf16 = 1;
    if (wt) { a.sBn = 1; a.sBk = O; } else { a.sBn = K; a.sBk = 1; }
    a.D = Y; a.ldd = O; a.dsplit = 0;
    a.bias = b; a.accumulate = acc; a.relu = relu; a.pre = pre; a.err = s->derr;
    launch_tc_gemm(a, S(s));
    return;
  }
  dim3 grid((ne + kT - 1) / kT, (O + kT - 1) / kT);
  k_dense<TW><<<grid, 256, 0, S(s)>>>(ne, K, O, A, static_cast<const TW*>(W), wt, b, acc, relu, pre, Y);
}
static void dense_any(stdg_solver* s, int K, int O, const float* A, int64_t woff, int wt, const float* b, int acc,
                      int relu, float* pre, float* Y) {
  GnnState& n = *s->gnn;
  if (n.bf16) dense<__nv_bfloat16>(s, K, O, A, static_cast<__nv_bfloat16*>(n.wc) + woff, wt, b, acc, relu, pre, Y);
  else dense<float>(s, K, O, A, static_cast<float*>(n.wc) + woff, wt, b, acc, relu, pre, Y);
}
static void wgrad(stdg_solver* s, int O, int K, const float* D, const float* Xin, int64_t goff, int64_t gboff) {
  GnnState& n = *s->gnn;
  const int ne = (int)s->ne;
  const int nchunk = (ne + kChunk - 1) / kChunk;
  if (n.bf16 && K + 1 <= 256) {
    // on the tensor cores: part[chunk][o][k] = Sum_{i in chunk} D[i][o] X[i][k], k = K the bias column
    TcGemmArgs a{};
    a.M = O; a.N = K + 1; a.K = ne; a.ksplit = kChunk;
    a.A = D; a.sAm = 1; a.sAk = O;
    a.B = Xin; a.sBn = 1; a.sBk = K; a.b_bf16 = 0; a.b_ones_last = 1;
    a.D = n.wpart; a.ldd = K + 1; a.dsplit = (int64_t)O * (K + 1);
    a.err = s->derr;
    launch_tc_gemm(a, S(s));
  } else {
    dim3 grid(nchunk, (O + kT - 1) / kT, (K + kT - 1) / kT);
    k_wgrad<<<grid, 256, 0, S(s)>>>(ne, O, K, D, Xin, n.wpart);
  }
  k_wgrad_reduce<<<kGB, 256, 0, S(s)>>>(nchunk, O, K, n.wpart, 1.0f, n.g + goff, gboff >= 0 ? n.g + gboff : nullptr);
  s->nlaunch += 2;
}

// forward pass of the network on r (double, pressure layout); leaves activations in the state
static void gnn_forward(stdg_solver* s, const double* r) {
  GnnState& n = *s->gnn;
  const int64_t nv = s->ne * (int64_t)n.C;
  k_gnn_sumsq<<<256, 256, 0, S(s)>>>(nv, r, n.part);
  k_gnn_scale<<<1, 32, 0, S(s)>>>(256, n.part, nv, n.sdev);
  k_gnn_features<<<kGB, 256, 0, S(s)>>>((int)s->ne, n.C, n.G, r, n.geom, n.sdev, n.X);
  s->nlaunch += 3;
  dense_any(s, n.F, n.H, n.X, n.off[0], 0, n.w + n.off[1], 0, 1, n.pre0, n.h[0]);
  for (int l = 0; l < n.L; ++l) {
    k_gather<<<kGB, 256, 0, S(s)>>>((int)s->ne, n.H, s->gnbr, n.h[l], n.mb[l]);
    ++s->nlaunch;
    const int64_t base = 2 + 3 * (int64_t)l;
    dense_any(s, n.H, n.H, n.h[l], n.off[base], 0, n.w + n.off[base + 2], 0, 0, nullptr, n.h[l + 1]);
    dense_any(s, n.H, n.H, n.mb[l], n.off[base + 1], 0, nullptr, 1, 1, n.pre[l], n.h[l + 1]);
  }
  const int64_t dbase = 2 + 3 * (int64_t)n.L;
  dense_any(s, n.H, n.C, n.h[n.L], n.off[dbase], 0, n.w + n.off[dbase + 1], 0, 0, nullptr, n.out);
}

// loss of one pair and accumulation of its gradients into n.g (loss added into n.loss[0])
static void gnn_backward(stdg_solver* s, const double* t) {
  GnnState& n = *s->gnn;
  const int64_t nv = s->ne * (int64_t)n.C, nh = s->ne * (int64_t)n.H;
  k_gnn_lossdiff<<<256, 256, 0, S(s)>>>(nv, n.out, n.sdev, t, n.dout, n.part);
  k_scale_f<<<kGB, 256, 0, S(s)>>>(nv, n.part, 256, n.dout, n.loss);
  s->nlaunch += 2;
  const int64_t dbase = 2 + 3 * (int64_t)n.L;
  wgrad(s, n.C, n.H, n.dout, n.h[n.L], n.off[dbase], n.off[dbase + 1]);
  dense_any(s, n.C, n.H, n.dout, n.off[dbase], 1, nullptr, 0, 0, nullptr, n.dh);
  for (int l = n.L - 1; l >= 0; --l) {
    const int64_t base = 2 + 3 * (int64_t)l;
    k_relu_back<<<kGB, 256, 0, S(s)>>>(nh, n.pre[l], n.dh, n.dpre);
    ++s->nlaunch;
    wgrad(s, n.H, n.H, n.dpre, n.h[l], n.off[base], n.off[base + 2]);
    wgrad(s, n.H, n.H, n.dpre, n.mb[l], n.off[base + 1], -1);
    dense_any(s, n.H, n.H, n.dpre, n.off[base], 1, nullptr, 0, 0, nullptr, n.t1);
    dense_any(s, n.H, n.H, n.dpre, n.off[base + 1], 1, nullptr, 0, 0, nullptr, n.t2);
    k_gather<<<kGB, 256, 0, S(s)>>>((int)s->ne, n.H, s->gnbr, n.t2, n.dh);
    k_fadd<<<kGB, 256, 0, S(s)>>>(nh, n.t1, n.dh);
    s->nlaunch += 2;
  }
  k_relu_back<<<kGB, 256, 0, S(s)>>>(nh, n.pre0, n.dh, n.dpre);
  ++s->nlaunch;
  wgrad(s, n.H, n.F, n.dpre, n.X, n.off[0], n.off[1]);
}

static void refresh_working_copy(stdg_solver* s) {
  GnnState& n = *s->gnn;
  if (n.bf16) k_to_bf16<<<kGB, 256, 0, S(s)>>>(n.np, n.w, static_cast<__nv_bfloat16*>(n.wc));
  else cudaMemcpyAsync(n.wc, n.w, n.np * sizeof(float), cudaMemcpyDeviceToDevice, S(s));
  ++s->nlaunch;
}

stdg_status gnn_precond(stdg_solver* s, const double* r, double* z, int use_gnn) {
  GnnState* n = s->gnn;
  if (!s->Binv) { set_error("block inverse missing"); return STDG_EINVAL; }
  if (!n || !n->tpinv) { set_error("learned preconditioner not initialised (stdg_gnn_init)"); return STDG_EINVAL; }
  k_bj_full<<<(int)s->ne, 128, 2 * s->Nst * sizeof(double), S(s)>>>(s->N, s->Ng, s->Binv, n->tpinv, r, z);
  ++s->nlaunch;
  if (use_gnn) {
    gnn_forward(s, r);
    k_gnn_output<<<kGB, 256, 0, S(s)>>>(s->ne * (int64_t)n->C, n->out, n->sdev, 1, z);
    ++s->nlaunch;
  }
  return cudaGetLastError() == cudaSuccess ? STDG_OK : (set_error("preconditioner launch failed"), STDG_ECUDA);
}

// The learned correction inside the flexible outer iteration of the coarse-corrected mixed solve:
// z += RMS(r) net(r / RMS(r)), skipping non-finite outputs (counted by the caller through *bad).
stdg_status gnn_correct(stdg_solver* s, const double* r, double* z, int* bad) {
  GnnState* n = s->gnn;
  if (!n || !n->tpinv) { set_error("learned correction not initialised (stdg_gnn_init)"); return STDG_EINVAL; }
  gnn_forward(s, r);
  k_gnn_correct<<<kGB, 256, 0, S(s)>>>(s->ne * (int64_t)n->C, n->out, n->sdev, z, bad);
  ++s->nlaunch;
  return cudaGetLastError() == cudaSuccess ? STDG_OK : (set_error("learned correction launch failed"), STDG_ECUDA);
}

// Harvest from the outer iterations of the mixed solve: pair k gets R = r_k (the residual after k
// inner-solve steps) and, first, T = -x_k (- z_k when z is given); gnn_mg_harvest_finish adds the
// final x to every T, leaving the error x* - x_k that the network's direction should approximate.
bool gnn_mg_harvest_room(stdg_solver* s, int k) {
  GnnState* n = s->gnn;
  return n && s->ah_mg > 0 && n->R && k < s->ah_mg && n->npairs + k < n->cap;
}
void gnn_mg_harvest_snap(stdg_solver* s, int k, const double* r, const double* x, const double* z) {
  GnnState& n = *s->gnn;
  const int64_t nv = s->ne * (int64_t)n.C;
  cudaMemcpyAsync(n.R + (size_t)(n.npairs + k) * nv, r, nv * sizeof(double), cudaMemcpyDeviceToDevice, S(s));
  k_neg_sum<<<kGB, 256, 0, S(s)>>>(nv, x, z, n.T + (size_t)(n.npairs + k) * nv);
  ++s->nlaunch;
}
void gnn_mg_harvest_finish(stdg_solver* s, int got, const double* x) {
  GnnState& n = *s->gnn;
  const int64_t nv = s->ne * (int64_t)n.C;
  for (int k = 0; k < got; ++k) k_axpy_d<<<kGB, 256, 0, S(s)>>>(nv, 1.0, x, n.T + (size_t)(n.npairs + k) * nv);
  s->nlaunch += got;
  n.npairs += got;
}

}  // namespace stdg

using namespace stdg;

static uint64_t g_mix(uint64_t& st) {
  st += 0x9E3779B97F4A7C15ull;
  uint64_t z = st;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" stdg_status stdg_gnn_init(stdg_solver* s, int hidden, int layers, int bf16_weights, uint64_t seed) {
  if (!s || hidden < 8 || hidden > 256 || layers < 1 || layers > 8) { set_error("stdg_gnn_init: invalid argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  if (s->gnn) { set_error("stdg_gnn_init: already initialised"); return STDG_EINVAL; }
  GnnState* n = new (std::nothrow) GnnState;
  if (!n) { set_error("out of host memory"); return STDG_ENOMEM; }
  s->gnn = n;
  n->H = hidden; n->L = layers; n->C = s->Nst; n->F = n->C + n->G; n->bf16 = bf16_weights ? 1 : 0;
  const int H = n->H, F = n->F, C = n->C;
  std::vector<int64_t> sizes = {(int64_t)H * F, H};
  for (int l = 0; l < n->L; ++l) { sizes.push_back((int64_t)H * H); sizes.push_back((int64_t)H * H); sizes.push_back(H); }
  sizes.push_back((int64_t)C * H); sizes.push_back(C);
  int64_t o = 0;
  for (int64_t sz : sizes) { n->off.push_back(o); o += (sz + 3) / 4 * 4; }
  n->np = o;
  // deterministic He-style initialisation from splitmix64(seed)
  std::vector<float> w(n->np, 0.0f);
  uint64_t st = seed;
  auto gauss = [&]() {
    double u1 = ((g_mix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0), u2 = ((g_mix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  auto fill = [&](int64_t off, int64_t cnt, double sd) { for (int64_t k = 0; k < cnt; ++k) w[off + k] = (float)(sd * gauss()); };
  fill(n->off[0], (int64_t)H * F, std::sqrt(2.0 / F));
  for (int l = 0; l < n->L; ++l) {
    fill(n->off[2 + 3 * l], (int64_t)H * H, std::sqrt(1.0 / H));
    fill(n->off[3 + 3 * l], (int64_t)H * H, std::sqrt(0.25 / H));
  }
  fill(n->off[2 + 3 * n->L], (int64_t)C * H, 0.1 * std::sqrt(1.0 / H));
  stdg_status e;
  const size_t ne = (size_t)s->ne;
  for (float** p : {&n->w, &n->g, &n->m, &n->v})
    if ((e = dev_alloc(s, (void**)p, n->np * sizeof(float))) != STDG_OK) return e;
  if ((e = dev_alloc(s, &n->wc, n->np * sizeof(float))) != STDG_OK) return e;
  cudaMemcpy(n->w, w.data(), n->np * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(n->m, 0, n->np * sizeof(float)); cudaMemset(n->v, 0, n->np * sizeof(float)); cudaMemset(n->g, 0, n->np * sizeof(float));
  if ((e = dev_alloc(s, (void**)&n->X, ne * F * sizeof(float))) != STDG_OK) return e;
  for (float** p : {&n->pre0, &n->dh, &n->dpre, &n->t1, &n->t2})
    if ((e = dev_alloc(s, (void**)p, ne * H * sizeof(float))) != STDG_OK) return e;
  for (float** p : {&n->out, &n->dout})
    if ((e = dev_alloc(s, (void**)p, ne * C * sizeof(float))) != STDG_OK) return e;
  n->h.assign(n->L + 1, nullptr); n->mb.assign(n->L, nullptr); n->pre.assign(n->L, nullptr);
  for (auto& p : n->h) if ((e = dev_alloc(s, (void**)&p, ne * H * sizeof(float))) != STDG_OK) return e;
  for (auto& p : n->mb) if ((e = dev_alloc(s, (void**)&p, ne * H * sizeof(float))) != STDG_OK) return e;
  for (auto& p : n->pre) if ((e = dev_alloc(s, (void**)&p, ne * H * sizeof(float))) != STDG_OK) return e;
  const int nchunk = (int)((ne + kChunk - 1) / kChunk);
  const int64_t wmax = std::max<int64_t>({(int64_t)H * (F + 1), (int64_t)C * (H + 1), (int64_t)H * (H + 1)});
  if ((e = dev_alloc(s, (void**)&n->wpart, (size_t)nchunk * wmax * sizeof(float))) != STDG_OK) return e;
  if ((e = dev_alloc(s, (void**)&n->sdev, 8 * sizeof(double))) != STDG_OK) return e;
  if ((e = dev_alloc(s, (void**)&n->loss, 8 * sizeof(double))) != STDG_OK) return e;
  if ((e = dev_alloc(s, (void**)&n->part, 512 * sizeof(double))) != STDG_OK) return e;
  if ((e = dev_alloc(s, (void**)&n->tpinv, kMaxNg * kMaxNg * sizeof(double))) != STDG_OK) return e;
  std::vector<double> tpinv(s->Ng * s->Ng);
  for (int q = 0; q < s->Ng * s->Ng; ++q) tpinv[q] = s->K[q] / (s->dt * s->dt);
  cudaMemcpy(n->tpinv, tpinv.data(), tpinv.size() * sizeof(double), cudaMemcpyHostToDevice);
  // geometry features: (|J_i| / mean |J|)^(1/3) and (boundary faces of i) / 4
  std::vector<double> dj(ne);
  std::vector<int> gn(4 * ne);
  cudaMemcpy(dj.data(), s->dm.detJ, ne * sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(gn.data(), s->gnbr, 4 * ne * sizeof(int), cudaMemcpyDeviceToHost);
  double mean = 0.0;
  for (double d : dj) mean += d;
  mean /= (double)ne;
  std::vector<float> geom(2 * ne);
  for (size_t i = 0; i < ne; ++i) {
    int nb = 0;
    for (int f = 0; f < 4; ++f) nb += gn[4 * i + f] < 0;
    geom[2 * i] = (float)std::cbrt(dj[i] / mean);
    geom[2 * i + 1] = 0.25f * nb;
  }
  if ((e = dev_alloc(s, (void**)&n->geom, 2 * ne * sizeof(float))) != STDG_OK) return e;
  cudaMemcpy(n->geom, geom.data(), geom.size() * sizeof(float), cudaMemcpyHostToDevice);
  refresh_working_copy(s);
  if (cudaStreamSynchronize(S(s)) != cudaSuccess) { set_error("stdg_gnn_init: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
  return STDG_OK;
}

extern "C" stdg_status stdg_gnn_params(stdg_solver* s, float* w_out, const float* w_in, int64_t* nparams) {
  if (!s || !s->gnn) { set_error("stdg_gnn_params: network not initialised"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  GnnState& n = *s->gnn;
  if (nparams) *nparams = n.np;
  cudaStreamSynchronize(S(s));
  if (w_out) STDG_CUDA(cudaMemcpy(w_out, n.w, n.np * sizeof(float), cudaMemcpyDeviceToHost));
  if (w_in) {
    STDG_CUDA(cudaMemcpy(n.w, w_in, n.np * sizeof(float), cudaMemcpyHostToDevice));
    refresh_working_copy(s);
    cudaMemset(n.m, 0, n.np * sizeof(float)); cudaMemset(n.v, 0, n.np * sizeof(float));
    n.adam_t = 0;
  }
  return STDG_OK;
}

extern "C" stdg_status stdg_gnn_layout(stdg_solver* s, int64_t* offsets, int* hidden, int* layers, int* nfeat) {
  if (!s || !s->gnn) { set_error("network not initialised"); return STDG_EINVAL; }
  GnnState& n = *s->gnn;
  if (offsets) for (size_t k = 0; k < n.off.size(); ++k) offsets[k] = n.off[k];
  if (hidden) *hidden = n.H;
  if (layers) *layers = n.L;
  if (nfeat) *nfeat = n.F;
  return STDG_OK;
}

extern "C" stdg_status stdg_gnn_apply(stdg_solver* s, const double* r, double* z) {
  if (!s || !s->gnn || !r || !z) { set_error("stdg_gnn_apply: invalid argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  gnn_forward(s, r);
  k_gnn_output<<<kGB, 256, 0, S(s)>>>(s->ne * (int64_t)s->gnn->C, s->gnn->out, s->gnn->sdev, 0, z);
  ++s->nlaunch;
  return cudaGetLastError() == cudaSuccess ? STDG_OK : (set_error("gnn apply failed"), STDG_ECUDA);
}

extern "C" stdg_status stdg_gnn_loss_grad(stdg_solver* s, const double* R, const double* T, int npairs, double* loss,
                                          float* grad_host) {
  if (!s || !s->gnn || !R || !T || npairs < 1) { set_error("stdg_gnn_loss_grad: invalid argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  GnnState& n = *s->gnn;
  const int64_t nv = s->ne * (int64_t)n.C;
  cudaMemsetAsync(n.g, 0, n.np * sizeof(float), S(s));
  cudaMemsetAsync(n.loss, 0, sizeof(double), S(s));
  for (int k = 0; k < npairs; ++k) {
    gnn_forward(s, R + k * nv);
    gnn_backward(s, T + k * nv);
  }
  double l = 0.0;
  STDG_CUDA(cudaMemcpyAsync(&l, n.loss, sizeof(double), cudaMemcpyDeviceToHost, S(s)));
  STDG_CUDA(cudaStreamSynchronize(S(s)));
  if (loss) *loss = l / npairs;
  if (grad_host) {
    std::vector<float> gh(n.np);
    STDG_CUDA(cudaMemcpy(gh.data(), n.g, n.np * sizeof(float), cudaMemcpyDeviceToHost));
    for (int64_t q = 0; q < n.np; ++q) grad_host[q] = gh[q] / npairs;
  }
  return STDG_OK;
}

extern "C" stdg_status stdg_gnn_train(stdg_solver* s, int epochs, double lr, int batch, double* first_loss,
                                      double* last_loss) {
  if (!s || !s->gnn || epochs < 1 || batch < 1 || !(lr > 0.0)) { set_error("stdg_gnn_train: invalid argument"); return STDG_EINVAL; }
  GnnState& n = *s->gnn;
  if (n.npairs < 1) { set_error("stdg_gnn_train: no harvested pairs (stdg_gnn_harvest)"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  const int64_t nv = s->ne * (int64_t)n.C;
  for (int ep = 0; ep < epochs; ++ep) {
    cudaMemsetAsync(n.loss, 0, sizeof(double), S(s));
    for (int k0 = 0; k0 < n.npairs; k0 += batch) {
      cudaMemsetAsync(n.g, 0, n.np * sizeof(float), S(s));
      for (int k = k0; k < std::min(n.npairs, k0 + batch); ++k) {
        gnn_forward(s, n.R + k * nv);
        gnn_backward(s, n.T + k * nv);
      }
      ++n.adam_t;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.0f - std::pow(b1, (float)n.adam_t), c2 = 1.0f - std::pow(b2, (float)n.adam_t);
      if (n.bf16)
        k_adam<__nv_bfloat16><<<kGB, 256, 0, S(s)>>>(n.np, n.w, n.g, n.m, n.v, (float)lr, b1, b2, 1e-8f, c1, c2,
                                                     static_cast<__nv_bfloat16*>(n.wc));
      else
        k_adam<float><<<kGB, 256, 0, S(s)>>>(n.np, n.w, n.g, n.m, n.v, (float)lr, b1, b2, 1e-8f, c1, c2,
                                             static_cast<float*>(n.wc));
      ++s->nlaunch;
    }
    double l = 0.0;
    STDG_CUDA(cudaMemcpyAsync(&l, n.loss, sizeof(double), cudaMemcpyDeviceToHost, S(s)));
    STDG_CUDA(cudaStreamSynchronize(S(s)));
    l /= n.npairs;
    if (!std::isfinite(l)) { set_error("stdg_gnn_train: non-finite loss"); return STDG_ENAN; }
    if (ep == 0 && first_loss) *first_loss = l;
    if (last_loss) *last_loss = l;
  }
  return STDG_OK;
}


extern "C" stdg_status stdg_gnn_harvest(stdg_solver* s, const double* b, int nsnap, int every, int max_pairs,
                                        int* total_pairs) {
  if (!s || !s->gnn || !b || nsnap < 1 || every < 1 || max_pairs < 1) { set_error("stdg_gnn_harvest: invalid argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  GnnState& n = *s->gnn;
  const int64_t nv = s->ne * (int64_t)n.C;
  stdg_status e;
  if (!n.R) {
    n.cap = max_pairs;
    if ((e = dev_alloc(s, (void**)&n.R, (size_t)n.cap * nv * sizeof(double))) != STDG_OK) return e;
    if ((e = dev_alloc(s, (void**)&n.T, (size_t)n.cap * nv * sizeof(double))) != STDG_OK) return e;
  }
  const int room = std::min(nsnap, n.cap - n.npairs);
  if (room <= 0) { if (total_pairs) *total_pairs = n.npairs; return STDG_OK; }
  double* x = nullptr;
  if ((e = dev_alloc(s, (void**)&x, nv * sizeof(double))) != STDG_OK) return e;
  // snapshots of the CG iterates go straight into the target slots
  const int gb = s->opt.graph_batch;
  s->opt.graph_batch = 1;
  s->snaps = n.T + (size_t)n.npairs * nv;
  s->snap_every = every; s->snap_cap = room; s->nsnap = 0;
  stdg_solve_stats st{};
  e = solve_pressure(s, b, x, 1e-12, STDG_SOLVER_KRON_PCG, &st);
  s->opt.graph_batch = gb;
  s->snap_every = 0;
  if (e != STDG_OK && e != STDG_ENOCONV) return e;
  const int got = s->nsnap;
  for (int k = 0; k < got; ++k) {
    double* xk = n.T + (size_t)(n.npairs + k) * nv;     // holds x_k
    double* rk = n.R + (size_t)(n.npairs + k) * nv;
    if ((e = apply_pressure(s, xk, rk, 1, 0, 1.0, -1.0)) != STDG_OK) return e;   // A x_k
    k_sub2<<<kGB, 256, 0, S(s)>>>(nv, b, rk);                                      // r_k = b - A x_k
    k_sub2<<<kGB, 256, 0, S(s)>>>(nv, x, xk);                                      // e_k = x* - x_k
    if ((e = gnn_precond(s, rk, s->kq, 0)) != STDG_OK) return e;                   // BJ(r_k)
    k_axpy_d<<<kGB, 256, 0, S(s)>>>(nv, -1.0, s->kq, xk);                          // t_k = e_k - BJ(r_k)
    s->nlaunch += 3;
  }
  n.npairs += got;
  if (total_pairs) *total_pairs = n.npairs;
  if (cudaStreamSynchronize(S(s)) != cudaSuccess) { set_error("stdg_gnn_harvest: %s", cudaGetErrorString(cudaGetLastError())); return STDG_ECUDA; }
  return STDG_OK;
}

extern "C" stdg_status stdg_gnn_autoharvest_mg(stdg_solver* s, int nsnap, int max_pairs) {
  if (!s || !s->gnn || nsnap < 0 || (nsnap > 0 && max_pairs < 1)) { set_error("stdg_gnn_autoharvest_mg: invalid argument"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  GnnState& n = *s->gnn;
  if (nsnap > 0 && !n.R) {
    const int64_t nv = s->ne * (int64_t)n.C;
    n.cap = max_pairs;
    stdg_status e;
    if ((e = dev_alloc(s, (void**)&n.R, (size_t)n.cap * nv * sizeof(double))) != STDG_OK) return e;
    if ((e = dev_alloc(s, (void**)&n.T, (size_t)n.cap * nv * sizeof(double))) != STDG_OK) return e;
  }
  s->ah_mg = nsnap;
  return STDG_OK;
}

extern "C" stdg_status stdg_gnn_autoharvest(stdg_solver* s, int nsnap, int every, int max_pairs) {
  if (!s || !s->gnn || nsnap < 0 || (nsnap > 0 && (every < 1 || max_pairs < 1))) { set_error("stdg_gnn_autoharvest: invalid argument"); return STDG_EINVAL; }
  s->ah_nsnap = nsnap; s->ah_every = every; s->ah_max = max_pairs;
  return STDG_OK;
}
