// Agglomeration coarse correction for the Kronecker-decoupled pressure systems.
//
// Each decoupled system is S x_q = b_q with S = -A_sp pinned (Sec. 2.7: A_sp is symmetric negative
// semidefinite, one pinned constant per time column).  Block Jacobi (the exact inverse of each tet's
// N x N diagonal block) removes the high-frequency error inside a tet but leaves the smooth error
// between tets; CG with block Jacobi alone needs O(1/h) iterations.  The correction added here works
// on the constant mode of every tet.  With the orthonormal Dubiner basis that mode is basis function
// 0, so the Galerkin restriction of S to piecewise constants is the (0,0) entry of each assembled
// five-point block: a symmetric positive definite matrix with the mesh's face graph as its pattern.
// That matrix is solved approximately by a V-cycle over nested agglomerates: tets are binned by
// centroid into cubes of the mean hexahedron size (6 Kuhn tets per cube on the benchmark meshes),
// then into cubes twice as large at each level, until at most kCoarseMax cells remain; the coarse
// matrices are Galerkin products with piecewise-constant prolongation, smoothed by one damped Jacobi
// sweep before and after the coarse correction, and the coarsest level is solved with its exact
// (dense) inverse.  The preconditioner is additive and symmetric positive definite:
//     z = Binv r + R^T V (R r),
// R = constant-mode coefficients (the pinned coefficient excluded), V = the V-cycle, which is
// symmetric (same Jacobi sweep before and after).  Every column shares the hierarchy.
//
// This is a solver choice; the paper uses unpreconditioned GMRES.  It changes how fast the iteration
// converges, not the system or its stopping test.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "solver.h"

namespace stdg {

constexpr int kCoarseMax = 512;       // the coarsest level is solved with a dense inverse
constexpr int kMgThreads = 256;
constexpr int kMgUp0Blocks = 304;     // 2 x 152 SMs: the blocks that write r.z partials
constexpr int kMgMaxLevels = 16;

struct MgLevel {
  int n = 0;                          // cells on this level
  int *rp = nullptr, *ci = nullptr;   // CSR of the Galerkin matrix (level >= 1)
  float *va = nullptr, *dl = nullptr; // its values; omega / diagonal
  int* par = nullptr;                 // cell -> cell of the next level (not on the coarsest)
  int *cptr = nullptr, *cidx = nullptr;  // children (cells of the previous level) of every cell
  float *r = nullptr, *x = nullptr;   // restricted residual and correction, n x Ng
};

struct MgState {
  int L = 0;                          // index of the coarsest level (levels 1..L are agglomerates)
  float *a0 = nullptr, *d0 = nullptr; // tets: 5 coefficients (diagonal, 4 faces), omega / diagonal
  int* par0 = nullptr;                // tet -> level-1 cell
  MgLevel lv[kMgMaxLevels + 1];
  float* cinv = nullptr;              // dense inverse of the coarsest matrix (symmetric)
  std::vector<int> sizes;             // cells per level, level 0 = tets
};

namespace {

__device__ inline void mg_block_store(double* v, int cnt, double* part) {
  __shared__ double red[kMaxNg][kMgThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < cnt; ++c) {
    double t = v[c];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[c][w] = t;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
    part[(size_t)blockIdx.x * cnt + threadIdx.x] = t;
  }
}

__device__ inline float mg_warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fine residual's constant modes -> level 1: for every level-1 cell, the sum over its tets of the
// residual after one damped Jacobi sweep from zero, s_i = r_i - Sum_j S0_ij (omega / S0_jj) r_j.
// The pinned coefficient (tet 0) is read as 0.
template <typename T>
__global__ void __launch_bounds__(kMgThreads) k_mg_down0(int nc, int Ng, int N, int Nst, const int* __restrict__ cptr,
                                                         const int* __restrict__ cidx, const int* __restrict__ t2n,
                                                         const float* __restrict__ a0, const float* __restrict__ d0,
                                                         const T* __restrict__ r, float* __restrict__ rc) {
  // one warp per level-1 cell; lane t handles term t % 5 (diagonal or face t % 5 - 1) of child t / 5
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nc; c += gridDim.x * wpb) {
    float acc[kMaxNg] = {0, 0, 0, 0, 0};
    const int k0 = cptr[c], nk = cptr[c + 1] - k0;
    for (int t = lane; t < 5 * nk; t += 32) {
      const int i = cidx[k0 + t / 5], f = t % 5;
      if (i == 0) continue;                        // pinned: contributes nothing
      const float* a = a0 + (size_t)i * 5;
      if (f == 0) {
        const float wi = a[0] * d0[i];
#pragma unroll
        for (int q = 0; q < kMaxNg; ++q)
          if (q < Ng) {
            const float ri = (float)r[(size_t)i * Nst + q * N];
            acc[q] += ri - wi * ri;
          }
      } else {
        const int nb = t2n[4 * i + f - 1];
        if (nb <= 0) continue;                     // boundary, or the pinned tet (coefficient 0)
        const float w = a[f] * d0[nb];
#pragma unroll
        for (int q = 0; q < kMaxNg; ++q)
          if (q < Ng) acc[q] -= w * (float)r[(size_t)nb * Nst + q * N];
      }
    }
#pragma unroll
    for (int q = 0; q < kMaxNg; ++q)
      if (q < Ng) {
        const float v = mg_warp_sum(acc[q]);
        if (lane == 0) rc[(size_t)c * Ng + q] = v;
      }
  }
}

// Level l -> l+1: the same on a CSR level; one warp per coarse cell, lane (child slot t / 4, every
// fourth entry of that child's row from t % 4).
__global__ void __launch_bounds__(kMgThreads) k_mg_down(int nc, int Ng, const int* __restrict__ cptr,
                                                        const int* __restrict__ cidx, const int* __restrict__ rp,
                                                        const int* __restrict__ ci, const float* __restrict__ va,
                                                        const float* __restrict__ dl, const float* __restrict__ r,
                                                        float* __restrict__ rc) {
  const int lane = threadIdx.x & 31, slot = lane >> 2, sub = lane & 3;
  const int wpb = blockDim.x >> 5;
  for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nc; c += gridDim.x * wpb) {
    float acc[kMaxNg] = {0, 0, 0, 0, 0};
    for (int k = cptr[c] + slot; k < cptr[c + 1]; k += 8) {
      const int i = cidx[k];
      if (sub == 0)
#pragma unroll
        for (int q = 0; q < kMaxNg; ++q)
          if (q < Ng) acc[q] += r[(size_t)i * Ng + q];
      for (int e = rp[i] + sub; e < rp[i + 1]; e += 4) {
        const int j = ci[e];
        const float w = va[e] * dl[j];
#pragma unroll
        for (int q = 0; q < kMaxNg; ++q)
          if (q < Ng) acc[q] -= w * r[(size_t)j * Ng + q];
      }
    }
#pragma unroll
    for (int q = 0; q < kMaxNg; ++q)
      if (q < Ng) {
        const float v = mg_warp_sum(acc[q]);
        if (lane == 0) rc[(size_t)c * Ng + q] = v;
      }
  }
}

// Coarsest level: x = C^-1 r with the dense symmetric inverse, one warp per row (row i of the
// inverse read contiguously), r staged in shared memory by every block.
__global__ void __launch_bounds__(kMgThreads) k_mg_coarse(int n, int Ng, const float* __restrict__ cinv,
                                                          const float* __restrict__ r, float* __restrict__ x) {
  __shared__ float rs[kCoarseMax * kMaxNg];
  for (int k = threadIdx.x; k < n * Ng; k += blockDim.x) rs[k] = r[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {
    float acc[kMaxNg] = {0, 0, 0, 0, 0};
    for (int j = lane; j < n; j += 32) {
      const float c = cinv[(size_t)i * n + j];
#pragma unroll
      for (int q = 0; q < kMaxNg; ++q)
        if (q < Ng) acc[q] = fmaf(c, rs[j * Ng + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kMaxNg; ++q)
      if (q < Ng) {
        const float v = mg_warp_sum(acc[q]);
        if (lane == 0) x[(size_t)i * Ng + q] = v;
      }
  }
}

// Level l <- l+1: e = omega D^-1 r + P x_c (pre-smoothing from zero plus the coarse correction), then
// x = e + omega D^-1 (r - S e) (post-smoothing); e of the neighbours is formed on the fly.
__global__ void __launch_bounds__(kMgThreads) k_mg_up(int n, int Ng, const int* __restrict__ rp,
                                                      const int* __restrict__ ci, const float* __restrict__ va,
                                                      const float* __restrict__ dl, const int* __restrict__ par,
                                                      const float* __restrict__ r, const float* __restrict__ xc,
                                                      float* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float s[kMaxNg], ei[kMaxNg];
    const float di = dl[i];
    const int pi = par[i];
#pragma unroll
    for (int q = 0; q < kMaxNg; ++q)
      if (q < Ng) {
        s[q] = r[(size_t)i * Ng + q];
        ei[q] = di * s[q] + xc[(size_t)pi * Ng + q];
      }
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int j = ci[e];
      const float w = va[e], dj = dl[j];
      const int pj = par[j];
#pragma unroll
      for (int q = 0; q < kMaxNg; ++q)
        if (q < Ng) s[q] -= w * (dj * r[(size_t)j * Ng + q] + xc[(size_t)pj * Ng + q]);
    }
#pragma unroll
    for (int q = 0; q < kMaxNg; ++q)
      if (q < Ng) x[(size_t)i * Ng + q] = ei[q] + di * s[q];
  }
}

// Tets <- level 1, added to the preconditioned residual's constant modes: z_i0 += x_i, with the
// partials of r.(R^T x) per column (the coarse part of r.z).  The pinned coefficient is left alone.
template <typename T>
__global__ void __launch_bounds__(kMgThreads) k_mg_up0(int ne, int Ng, int N, int Nst, const int* __restrict__ t2n,
                                                       const float* __restrict__ a0, const float* __restrict__ d0,
                                                       const int* __restrict__ par0, const T* __restrict__ r,
                                                       const float* __restrict__ x1, T* __restrict__ z,
                                                       double* __restrict__ part) {
  double dot[kMaxNg] = {0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
    if (i == 0) continue;
    const float* a = a0 + (size_t)i * 5;
    const float di = d0[i];
    const int pi = par0[i];
    T ri[kMaxNg];
    float s[kMaxNg], ei[kMaxNg];
#pragma unroll
    for (int q = 0; q < kMaxNg; ++q)
      if (q < Ng) {
        ri[q] = r[(size_t)i * Nst + q * N];
        ei[q] = di * (float)ri[q] + x1[(size_t)pi * Ng + q];
        s[q] = (float)ri[q] - a[0] * ei[q];
      }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int nb = t2n[4 * i + f];
      if (nb <= 0) continue;
      const float w = a[1 + f], dj = d0[nb];
      const int pj = par0[nb];
#pragma unroll
      for (int q = 0; q < kMaxNg; ++q)
        if (q < Ng) s[q] -= w * (dj * (float)r[(size_t)nb * Nst + q * N] + x1[(size_t)pj * Ng + q]);
    }
#pragma unroll
    for (int q = 0; q < kMaxNg; ++q)
      if (q < Ng) {
        const float xi = ei[q] + di * s[q];
        const size_t o = (size_t)i * Nst + q * N;
        z[o] = z[o] + (T)xi;
        dot[q] += (double)ri[q] * (double)xi;
      }
  }
  mg_block_store(dot, Ng, part);
}

inline int mg_grid(int n) { return std::max(1, std::min((n + kMgThreads - 1) / kMgThreads, 1216)); }
// grid for one warp per item
inline int mg_wgrid(int n) { return std::max(1, std::min((n + kMgThreads / 32 - 1) / (kMgThreads / 32), 4864)); }

// Galerkin product of a CSR level with piecewise-constant prolongation (cell c of the finer level
// -> agg[c]), summed in binary64.
void galerkin(int nfine, const std::vector<int>& rp, const std::vector<int>& ci, const std::vector<double>& va,
              const std::vector<int>& agg, int ncoarse, std::vector<int>& orp, std::vector<int>& oci,
              std::vector<double>& ova) {
  std::vector<std::pair<int64_t, double>> t;
  t.reserve(va.size());
  for (int i = 0; i < nfine; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      t.push_back({(int64_t)agg[i] * ncoarse + agg[ci[e]], va[e]});
  // a cell without any coupling (it holds only the pinned tet) gets a unit diagonal
  std::vector<char> has(ncoarse, 0);
  for (const auto& x : t) has[x.first / ncoarse] = 1;
  for (int c = 0; c < ncoarse; ++c)
    if (!has[c]) t.push_back({(int64_t)c * ncoarse + c, 1.0});
  std::sort(t.begin(), t.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  orp.assign(ncoarse + 1, 0);
  oci.clear(); ova.clear();
  for (size_t k = 0; k < t.size();) {
    size_t m = k;
    double v = 0.0;
    while (m < t.size() && t[m].first == t[k].first) v += t[m++].second;
    const int row = (int)(t[k].first / ncoarse);
    oci.push_back((int)(t[k].first % ncoarse));
    ova.push_back(v);
    orp[row + 1]++;
    k = m;
  }
  for (int i = 0; i < ncoarse; ++i) orp[i + 1] += orp[i];
}

template <typename V>
stdg_status upload(stdg_solver* s, V** d, const std::vector<V>& h) {
  stdg_status e = dev_alloc(s, (void**)d, h.size() * sizeof(V));
  if (e != STDG_OK) return e;
  if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("coarse-level upload failed");
    return STDG_ECUDA;
  }
  return STDG_OK;
}

std::vector<float> to_f32(const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); }

}  // namespace

// Nested agglomerates: tet centroids binned into cubes of edge h1 anchored at lo, then of edge 2 h1,
// 4 h1, ... (a size that merges no bins is skipped), until at most coarse_max cells remain or
// max_levels levels exist.  cell[l][i] = cell of tet i on level l + 1, numbered in bin-key order.
// Returns false if the last level still has more than coarse_max cells.
bool agglomerate_levels(int ne, const double* bary, const double lo[3], double h1, int coarse_max, int max_levels,
                        std::vector<std::vector<int>>& cell, std::vector<int>& sizes) {
  cell.clear();
  sizes.assign(1, ne);
  std::vector<int64_t> ic(3 * (size_t)ne);
  for (int i = 0; i < ne; ++i)
    for (int c = 0; c < 3; ++c)
      ic[3 * (size_t)i + c] = std::max<int64_t>(0, (int64_t)std::floor((bary[3 * (size_t)i + c] - lo[c]) / h1));
  for (int shift = 0; shift < 40 && (int)cell.size() < max_levels; ++shift) {
    std::vector<std::pair<int64_t, int>> key(ne);
    for (int i = 0; i < ne; ++i) {
      const int64_t x = ic[3 * (size_t)i] >> shift, y = ic[3 * (size_t)i + 1] >> shift, z = ic[3 * (size_t)i + 2] >> shift;
      key[i] = {(x << 42) | (y << 21) | z, i};
    }
    std::sort(key.begin(), key.end());
    std::vector<int> id(ne);
    int n = 0;
    for (int k = 0; k < ne; ++k) {
      if (k > 0 && key[k].first != key[k - 1].first) ++n;
      id[key[k].second] = n;
    }
    ++n;
    if (n == sizes.back() && !cell.empty()) continue;   // no agglomeration at this size: grow the cube
    cell.push_back(std::move(id));
    sizes.push_back(n);
    if (n <= coarse_max) break;
  }
  return !cell.empty() && sizes.back() <= coarse_max;
}

double mg_omega() {
  const char* env = std::getenv("STDG_MG_OMEGA");
  const double w = env ? std::atof(env) : 0.8;
  return (w > 0.0 && w < 2.0) ? w : 0.8;
}

stdg_status mg_ensure(stdg_solver* s) {
  if (s->mg) return STDG_OK;
  const int ne = (int)s->ne, nf = (int)s->nf, N = s->N, Ng = s->Ng;
  const size_t NN = (size_t)N * N;
  std::vector<double> bd(ne), ao(nf), X0(3 * (size_t)ne), J(9 * (size_t)ne), bary(3 * (size_t)ne), detJ(ne);
  std::vector<int> t2n(4 * (size_t)ne), t2f(4 * (size_t)ne);
  cudaStream_t st = s->stream;
  // the (0,0) entry of every diagonal block and of every face block
  STDG_CUDA(cudaMemcpy2DAsync(bd.data(), sizeof(double), s->Bdiag, NN * sizeof(double), sizeof(double), ne,
                              cudaMemcpyDeviceToHost, st));
  STDG_CUDA(cudaMemcpy2DAsync(ao.data(), sizeof(double), s->Aoff, NN * sizeof(double), sizeof(double), nf,
                              cudaMemcpyDeviceToHost, st));
  STDG_CUDA(cudaMemcpyAsync(t2n.data(), s->dm.t2n, t2n.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  STDG_CUDA(cudaMemcpyAsync(t2f.data(), s->dm.t2f, t2f.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  STDG_CUDA(cudaMemcpyAsync(X0.data(), s->dm.X0, X0.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  STDG_CUDA(cudaMemcpyAsync(J.data(), s->dm.J, J.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  STDG_CUDA(cudaMemcpyAsync(bary.data(), s->dm.bary, bary.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  STDG_CUDA(cudaMemcpyAsync(detJ.data(), s->dm.detJ, detJ.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  STDG_CUDA(cudaStreamSynchronize(st));
  const double omega = mg_omega();

  // level 0: constant-mode coefficients of the pinned S = -A_sp (tet 0 pinned: unit diagonal, no coupling)
  std::vector<double> a0(5 * (size_t)ne, 0.0);
  for (int i = 0; i < ne; ++i) {
    a0[5 * (size_t)i] = i == 0 ? 1.0 : -bd[i];
    for (int f = 0; f < 4; ++f) {
      const int nb = t2n[4 * (size_t)i + f];
      if (i != 0 && nb > 0) a0[5 * (size_t)i + 1 + f] = -ao[t2f[4 * (size_t)i + f]];
    }
    if (!(a0[5 * (size_t)i] > 0.0)) { set_error("coarse correction: non-positive constant-mode diagonal"); return STDG_EINVAL; }
  }

  // agglomerates: centroids binned into cubes of the mean hexahedron size (6 mean tet volumes), then
  // cubes twice as large per level; the bins nest, so each level's cells partition the previous
  double lo[3] = {INFINITY, INFINITY, INFINITY}, vsum = 0.0;
  for (int i = 0; i < ne; ++i) {
    for (int c = 0; c < 3; ++c) {
      double v = X0[3 * (size_t)i + c];
      lo[c] = std::min(lo[c], v);
      for (int k = 0; k < 3; ++k) lo[c] = std::min(lo[c], v + J[9 * (size_t)i + 3 * c + k]);
    }
    vsum += std::fabs(detJ[i]);
  }
  const double h1 = std::cbrt(vsum / ne);       // |det J| = 6 x volume
  std::vector<std::vector<int>> cell;             // cell[l-1][tet], levels 1..L
  std::vector<int> sizes;
  if (!agglomerate_levels(ne, bary.data(), lo, h1, kCoarseMax, kMgMaxLevels, cell, sizes)) {
    set_error("coarse correction: agglomeration left %d cells", sizes.back());
    return STDG_EINVAL;
  }
  const int L = (int)cell.size();
  MgState* mg = new MgState();
  mg->L = L;
  mg->sizes = sizes;
  s->mg = mg;

  // level 1 = Galerkin product of level 0 restricted to the unpinned constant modes (CSR built from
  // the tet coefficients; the pinned tet has no row)
  std::vector<int> rp0(ne + 1, 0), ci0;
  std::vector<double> va0;
  for (int i = 0; i < ne; ++i) {
    if (i == 0) { rp0[1] = 0; continue; }
    ci0.push_back(i); va0.push_back(a0[5 * (size_t)i]);
    for (int f = 0; f < 4; ++f)
      if (a0[5 * (size_t)i + 1 + f] != 0.0) { ci0.push_back(t2n[4 * (size_t)i + f]); va0.push_back(a0[5 * (size_t)i + 1 + f]); }
    rp0[i + 1] = (int)ci0.size();
  }
  std::vector<int> rp, ci;
  std::vector<double> va;
  galerkin(ne, rp0, ci0, va0, cell[0], sizes[1], rp, ci, va);
  stdg_status e;
  std::vector<float> d0(ne);
  for (int i = 0; i < ne; ++i) d0[i] = (float)(omega / a0[5 * (size_t)i]);
  if ((e = upload(s, &mg->a0, to_f32(a0))) != STDG_OK) return e;
  if ((e = upload(s, &mg->d0, d0)) != STDG_OK) return e;
  if ((e = upload(s, &mg->par0, cell[0])) != STDG_OK) return e;
  for (int l = 1; l <= L; ++l) {
    MgLevel& lv = mg->lv[l];
    lv.n = sizes[l];
    // children: the cells of level l-1 (tets for l = 1) in each cell of level l
    std::vector<int> par_prev(sizes[l - 1]);
    if (l == 1) par_prev = cell[0];
    else
      for (int i = 0; i < ne; ++i) par_prev[cell[l - 2][i]] = cell[l - 1][i];
    std::vector<int> cptr(lv.n + 1, 0), cidx(sizes[l - 1]);
    for (int c : par_prev) cptr[c + 1]++;
    for (int c = 0; c < lv.n; ++c) cptr[c + 1] += cptr[c];
    std::vector<int> fill(cptr.begin(), cptr.end() - 1);
    for (int k = 0; k < sizes[l - 1]; ++k) cidx[fill[par_prev[k]]++] = k;
    if ((e = upload(s, &lv.cptr, cptr)) != STDG_OK) return e;
    if ((e = upload(s, &lv.cidx, cidx)) != STDG_OK) return e;
    if ((e = dev_alloc(s, (void**)&lv.r, (size_t)lv.n * Ng * sizeof(float))) != STDG_OK) return e;
    if ((e = dev_alloc(s, (void**)&lv.x, (size_t)lv.n * Ng * sizeof(float))) != STDG_OK) return e;
    std::vector<double> diag(lv.n, 0.0);
    for (int i = 0; i < lv.n; ++i)
      for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == i) diag[i] = va[k];
    if (l < L) {
      std::vector<int> par(lv.n);
      for (int i = 0; i < ne; ++i) par[cell[l - 1][i]] = cell[l][i];
      std::vector<float> dl(lv.n);
      for (int i = 0; i < lv.n; ++i) {
        if (!(diag[i] > 0.0)) { set_error("coarse correction: non-positive diagonal on level %d", l); return STDG_EINVAL; }
        dl[i] = (float)(omega / diag[i]);
      }
      if ((e = upload(s, &lv.rp, rp)) != STDG_OK) return e;
      if ((e = upload(s, &lv.ci, ci)) != STDG_OK) return e;
      if ((e = upload(s, &lv.va, to_f32(va))) != STDG_OK) return e;
      if ((e = upload(s, &lv.dl, dl)) != STDG_OK) return e;
      if ((e = upload(s, &lv.par, par)) != STDG_OK) return e;
      std::vector<int> nrp, nci;
      std::vector<double> nva;
      galerkin(lv.n, rp, ci, va, par, sizes[l + 1], nrp, nci, nva);
      rp.swap(nrp); ci.swap(nci); va.swap(nva);
    } else {
      // coarsest: dense Cholesky in binary64, then the explicit inverse
      const int n = lv.n;
      std::vector<double> A((size_t)n * n, 0.0);
      for (int i = 0; i < n; ++i)
        for (int k = rp[i]; k < rp[i + 1]; ++k) A[(size_t)i * n + ci[k]] = va[k];
      for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) { set_error("coarse correction: coarsest matrix not positive definite"); return STDG_EINVAL; }
        d = std::sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
          double v = A[(size_t)i * n + j];
          for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
          A[(size_t)i * n + j] = v / d;
        }
      }
      std::vector<double> inv((size_t)n * n, 0.0), col(n);
      for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {                 // L y = e_c
          double v = i == c ? 1.0 : 0.0;
          for (int k = 0; k < i; ++k) v -= A[(size_t)i * n + k] * col[k];
          col[i] = v / A[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {            // L^T x = y
          double v = col[i];
          for (int k = i + 1; k < n; ++k) v -= A[(size_t)k * n + i] * col[k];
          col[i] = v / A[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[(size_t)c * n + i] = col[i];
      }
      if ((e = upload(s, &mg->cinv, to_f32(inv))) != STDG_OK) return e;
    }
  }
  return STDG_OK;
}

int mg_launches(const stdg_solver* s) { return s->mg ? 2 * s->mg->L + 1 : 0; }
int mg_partial_blocks() { return kMgUp0Blocks; }
int mg_levels(const stdg_solver* s, int* sizes, int cap) {
  if (!s->mg) return 0;
  const int n = (int)s->mg->sizes.size();
  for (int l = 0; l < n && l < cap; ++l) sizes[l] = s->mg->sizes[l];
  return n;
}

template <typename T>
static void mg_apply_t(stdg_solver* s, const T* r, T* z, double* part) {
  MgState* mg = s->mg;
  const int Ng = s->Ng, N = s->N, Nst = s->Nst, L = mg->L, ne = (int)s->ne;
  cudaStream_t st = s->stream;
  MgLevel* lv = mg->lv;
  k_mg_down0<T><<<mg_wgrid(lv[1].n), kMgThreads, 0, st>>>(lv[1].n, Ng, N, Nst, lv[1].cptr, lv[1].cidx, s->dm.t2n,
                                                          mg->a0, mg->d0, r, lv[1].r);
  for (int l = 1; l < L; ++l)
    k_mg_down<<<mg_wgrid(lv[l + 1].n), kMgThreads, 0, st>>>(lv[l + 1].n, Ng, lv[l + 1].cptr, lv[l + 1].cidx, lv[l].rp,
                                                           lv[l].ci, lv[l].va, lv[l].dl, lv[l].r, lv[l + 1].r);
  k_mg_coarse<<<mg_wgrid(lv[L].n), kMgThreads, 0, st>>>(lv[L].n, Ng, mg->cinv, lv[L].r, lv[L].x);
  for (int l = L - 1; l >= 1; --l)
    k_mg_up<<<mg_grid(lv[l].n), kMgThreads, 0, st>>>(lv[l].n, Ng, lv[l].rp, lv[l].ci, lv[l].va, lv[l].dl, lv[l].par,
                                                     lv[l].r, lv[l + 1].x, lv[l].x);
  k_mg_up0<T><<<kMgUp0Blocks, kMgThreads, 0, st>>>(ne, Ng, N, Nst, s->dm.t2n, mg->a0, mg->d0, mg->par0, r, lv[1].x, z,
                                                   part);
}

void mg_apply_f32(stdg_solver* s, const float* r, float* z, double* part) { mg_apply_t<float>(s, r, z, part); }
void mg_apply_f64(stdg_solver* s, const double* r, double* z, double* part) { mg_apply_t<double>(s, r, z, part); }

void mg_free(stdg_solver* s) {
  delete s->mg;                                   // device arrays are in s->allocs
  s->mg = nullptr;
}

}  // namespace stdg

extern "C" stdg_status stdg_mesh_agglomerate(const stdg_mesh* m, int coarse_max, int max_levels, int32_t* cell,
                                             int64_t* sizes, int* levels) {
  if (!m || !cell || !sizes || !levels || max_levels < 1 || coarse_max < 1) {
    stdg::set_error("stdg_mesh_agglomerate: NULL argument or non-positive limit");
    return STDG_EINVAL;
  }
  const int ne = (int)m->ne;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, vsum = 0.0;
  for (int64_t v = 0; v < m->nv; ++v)
    for (int c = 0; c < 3; ++c) lo[c] = std::min(lo[c], m->X[3 * v + c]);
  for (int i = 0; i < ne; ++i) vsum += std::fabs(m->detJ[i]);
  std::vector<std::vector<int>> cl;
  std::vector<int> sz;
  const bool ok = stdg::agglomerate_levels(ne, m->bary.data(), lo, std::cbrt(vsum / ne), coarse_max, max_levels, cl, sz);
  *levels = (int)cl.size();
  for (size_t l = 0; l < cl.size(); ++l) {
    sizes[l] = sz[l + 1];
    for (int i = 0; i < ne; ++i) cell[l * (size_t)ne + i] = cl[l][i];
  }
  if (!ok) {
    stdg::set_error("stdg_mesh_agglomerate: %d levels leave more than %d cells", max_levels, coarse_max);
    return STDG_EUNSUPPORTED;
  }
  return STDG_OK;
}
