// Low-precision operator path (binary32 / bfloat16 blocks inside the mixed-precision solves).
//
// k_apply_lp<TB>: the five-point block operator with blocks stored in TB (binary32 or bfloat16)
// and vectors / accumulation in binary32.  Per application it streams every block once
// (HBM-bound: arithmetic intensity Ng*2/sizeof(TB) flop/B is far below the FP32 pipe's balance),
// so the kernel is built around moving blocks fast:
//   * persistent CTAs, each owning a stream of tets; per stage a CTA processes TPB tets;
//   * the 5 blocks of each tet (diagonal + up to 4 face blocks, contiguous, 16-byte padded) are
//     staged into shared memory by 1-D TMA bulk copies (cp.async.bulk ... complete_tx) that
//     complete on one mbarrier per stage; two stages double-buffer the stream;
//   * thread (tet, slot, row k) forms Ng partial sums over the row; rows are walked with a
//     k-dependent skew so that the 32 threads of a warp hit distinct shared-memory banks;
//   * the 5 slot partials are summed in a fixed order (bitwise reproducible results).
// Every mbarrier wait is bounded; on timeout the kernel records an error word and returns.
#include <cuda_bf16.h>

#include "lp_ptx.cuh"
#include "solver.h"

namespace stdg {

constexpr int kStages = 2;

// ---- arithmetic policies -----------------------------------------------------------------
// PolF32 / PolBF16: blocks binary32 / bfloat16, vectors and accumulation binary32.
// PolDF: FP64-accurate products from binary32 pairs ("double-float").  A block entry A is stored
// as (hi, lo) = (fl32(A), fl32(A - hi)); x is split the same way with integer operations (so no
// binary64 instruction is needed per element); a product (ah + al)(zh + zl) is formed exactly in
// its leading part (fma error term) plus the cross terms, and sums use the error-free TwoSum.
struct PolF32 {
  using TB = float; using TZ = float; using XIn = float; using YOut = float; using Real = float;
  struct Acc { float v; };
  static constexpr int kBlockAlign = 4;     // elements per 16 bytes
  __device__ static void zero(Acc& a) { a.v = 0.0f; }
  __device__ static TZ load_x(XIn v) { return v; }
  __device__ static TZ zero_z() { return 0.0f; }
  __device__ static void fma(Acc& a, TB b, TZ z) { a.v = fmaf(b, z, a.v); }
  __device__ static void add(Acc& a, const Acc& b) { a.v += b.v; }
  __device__ static Real value(const Acc& a) { return a.v; }
};
struct PolBF16 {
  using TB = __nv_bfloat16; using TZ = float; using XIn = float; using YOut = float; using Real = float;
  struct Acc { float v; };
  static constexpr int kBlockAlign = 8;
  __device__ static void zero(Acc& a) { a.v = 0.0f; }
  __device__ static TZ load_x(XIn v) { return v; }
  __device__ static TZ zero_z() { return 0.0f; }
  __device__ static void fma(Acc& a, TB b, TZ z) { a.v = fmaf(__bfloat162float(b), z, a.v); }
  __device__ static void add(Acc& a, const Acc& b) { a.v += b.v; }
  __device__ static Real value(const Acc& a) { return a.v; }
};
struct PolDF {
  using TB = float2; using TZ = float2; using XIn = double; using YOut = double; using Real = double;
  struct Acc { float h, l; };
  static constexpr int kBlockAlign = 2;
  __device__ static void zero(Acc& a) { a.h = 0.0f; a.l = 0.0f; }
  __device__ static TZ zero_z() { return make_float2(0.0f, 0.0f); }
  __device__ static TZ load_x(XIn x) { return df_split(x); }
  __device__ static void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
  }
  __device__ static void fma(Acc& a, TB b, TZ z) {
    const float p = __fmul_rn(b.x, z.x);          // never fused into the sum below (error-free TwoSum)
    float e = fmaf(b.x, z.x, -p);
    e = fmaf(b.x, z.y, e);
    e = fmaf(b.y, z.x, e);
    e = fmaf(b.y, z.y, e);
    float s, t;
    two_sum(a.h, p, s, t);
    a.h = s;
    a.l += t + e;
  }
  __device__ static void add(Acc& a, const Acc& b) {
    float s, t;
    two_sum(a.h, b.h, s, t);
    a.h = s;
    a.l += t + b.l;
  }
  __device__ static Real value(const Acc& a) { return (double)a.h + (double)a.l; }
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename Pol>
struct TmaArgs {
  int ne, N, Ng, SB, TPB;        // SB: padded block stride (elements)
  const int *t2f, *t2n, *left;
  const int4 *gface, *gnbr;      // per tet: face block (j << 1 | transposed) or -1; neighbour tet or -1
  const typename Pol::TB *Bd, *Ao;
  typename Pol::Real scale, pin_diag;
  int tacc_identity, pinned;
  typename Pol::Real Tacc[kMaxNg * kMaxNg];
  int* err;                      // error word (bounded waits)
};

// Warp-specialised pipeline.  Warp 0 produces: for each group of TPB tets it reads the per-tet
// gather table, issues the 1-D TMA copies of the 5 blocks of every tet and cp.async copies of the
// x rows of the tets and their neighbours, all completing on the stage's "full" mbarrier.  The
// consumer warps convert x, form the slot partial sums, release the stage on its "empty"
// mbarrier and write y.  Consumers synchronise among themselves with a named barrier only.
constexpr int kWsStages = 2;
constexpr long kSpin = 20000;                    // bound on every mbarrier wait (x <= 1 ms suspend each)

template <typename Pol, int NG>
__global__ void __launch_bounds__(416) k_apply_tma(TmaArgs<Pol> a, const typename Pol::XIn* __restrict__ x,
                                                   typename Pol::YOut* __restrict__ y) {
  using TB = typename Pol::TB;
  using TZ = typename Pol::TZ;
  using XIn = typename Pol::XIn;
  using Acc = typename Pol::Acc;
  using Real = typename Pol::Real;
  constexpr int S = kWsStages;
  constexpr int Ng = NG;                        // time functions: compile-time, accumulators stay in registers
  extern __shared__ __align__(128) unsigned char smraw[];
  const int N = a.N, Nst = N * Ng, SB = a.SB, TPB = a.TPB;
  const int rows = TPB * 5;                     // (tet, slot) rows per group
  const int xlen = rows * Nst;
  const size_t blk_bytes = (size_t)SB * sizeof(TB);
  const size_t stage_blk = (size_t)rows * blk_bytes;
  const size_t off_xraw = S * stage_blk;
  const size_t off_xs = off_xraw + align16((size_t)S * xlen * sizeof(XIn));
  const size_t off_part = off_xs + align16((size_t)xlen * sizeof(TZ));
  const size_t off_tab = off_part + align16((size_t)xlen * sizeof(Acc));
  const size_t off_bars = off_tab + align16((size_t)S * rows * sizeof(int2));
  TB* blkbuf = reinterpret_cast<TB*>(smraw);
  XIn* xraw = reinterpret_cast<XIn*>(smraw + off_xraw);
  TZ* xs = reinterpret_cast<TZ*>(smraw + off_xs);
  Acc* part = reinterpret_cast<Acc*>(smraw + off_part);
  int2* tab = reinterpret_cast<int2*>(smraw + off_tab);        // (neighbour tet or -1, transposed)
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + off_bars);
  uint64_t* empty = full + S;
  __shared__ int s_abort;
  const int ngroups = (a.ne + TPB - 1) / TPB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncw = (blockDim.x >> 5) - 1;        // consumer warps
  const int nct = ncw * 32;
  if (tid == 0) {
    for (int q = 0; q < S; ++q) { mbar_init(&full[q], 1 + 32); mbar_init(&empty[q], ncw); }
    s_abort = 0;
    fence_async_smem();
  }
  __syncthreads();
  if (warp == 0) {
    // ------------------------------------------------------------------ producer
    int it = 0;
    for (int g = blockIdx.x; g < ngroups; g += gridDim.x, ++it) {
      const int st = it % S;
      if (it >= S) {
        long spins = 0;
        while (!mbar_wait_hint(&empty[st], (uint32_t)(((it / S) - 1) & 1))) {
          if (++spins > kSpin || s_abort) { s_abort = 1; break; }
        }
        if (s_abort) break;
      }
      int2* tb = tab + (size_t)st * rows;
      int nbv[5] = {-1, -1, -1, -1, -1}, jv[5] = {-1, -1, -1, -1, -1};
      uint32_t bytes = 0;
      const int i = g * TPB + lane;
      if (lane < TPB) {
        if (i < a.ne) {
          const int4 gf = a.gface[i], gn = a.gnbr[i];
          const int fj[4] = {gf.x, gf.y, gf.z, gf.w}, nn[4] = {gn.x, gn.y, gn.z, gn.w};
          nbv[0] = i; jv[0] = i;
          tb[lane * 5] = make_int2(i, 0);
          for (int f = 0; f < 4; ++f) {
            if (fj[f] >= 0) { nbv[f + 1] = nn[f]; jv[f + 1] = fj[f] >> 1; }
            tb[lane * 5 + f + 1] = make_int2(fj[f] >= 0 ? nn[f] : -1, fj[f] >= 0 ? (fj[f] & 1) : 0);
          }
        } else {
          for (int sl = 0; sl < 5; ++sl) tb[lane * 5 + sl] = make_int2(-1, 0);
        }
        for (int sl = 0; sl < 5; ++sl) if (nbv[sl] >= 0) bytes += (uint32_t)blk_bytes;
      }
      for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
      if (lane == 0) mbar_expect_tx(&full[st], bytes);         // the one explicit arrival
      __syncwarp();
      if (lane < TPB) {
        for (int sl = 0; sl < 5; ++sl) {
          if (nbv[sl] < 0) continue;
          const TB* src = sl == 0 ? a.Bd + (size_t)i * SB : a.Ao + (size_t)jv[sl] * SB;
          tma_load_1d(reinterpret_cast<unsigned char*>(blkbuf) + st * stage_blk + ((size_t)lane * 5 + sl) * blk_bytes,
                      src, (uint32_t)blk_bytes, &full[st]);
        }
      }
      __syncwarp();
      XIn* xr = xraw + (size_t)st * xlen;
      for (int r = 0; r < rows; ++r) {
        const int nb = tb[r].x;
        if (nb < 0) continue;
        const XIn* src = x + (size_t)nb * Nst;
        for (int o = lane; o < Nst; o += 32) cp_async<sizeof(XIn)>(xr + (size_t)r * Nst + o, src + o);
      }
      cp_async_mbar_arrive_noinc(&full[st]);                   // 32 arrivals once this lane's copies land
    }
    cp_async_wait_all();
    return;
  }
  // -------------------------------------------------------------------- consumers
  const int ct = tid - 32, cw = warp - 1;
  const int my_tl = ct / (5 * N), my_sl = (ct / N) % 5, my_k = ct % N;
  const bool computes = ct < rows * N;
  int it = 0;
  for (int g = blockIdx.x; g < ngroups; g += gridDim.x, ++it) {
    const int st = it % S;
    {
      long spins = 0;
      while (!mbar_wait_hint(&full[st], (uint32_t)((it / S) & 1))) {
        if (++spins > kSpin || s_abort) { s_abort = 1; break; }
      }
    }
    named_bar_sync(1, nct);
    if (s_abort) { if (ct == 0) atomicExch(a.err, 1); break; }
    const int2* tb = tab + (size_t)st * rows;
    const XIn* xr = xraw + (size_t)st * xlen;
    for (int r = cw; r < rows; r += ncw) {                     // convert x (pinned entries read as 0)
      const int nb = tb[r].x;
      for (int o = lane; o < Nst; o += 32) {
        TZ v = Pol::zero_z();
        if (nb >= 0 && !(a.pinned && nb == 0 && (o % N) == 0)) v = Pol::load_x(xr[(size_t)r * Nst + o]);
        xs[(size_t)r * Nst + o] = v;
      }
    }
    named_bar_sync(1, nct);
    if (computes) {
      const int r = my_tl * 5 + my_sl, k = my_k;
      Acc acc[NG], acc2[NG];                    // two independent chains per column (even / odd terms)
#pragma unroll
      for (int q = 0; q < Ng; ++q) { Pol::zero(acc[q]); Pol::zero(acc2[q]); }
      const int2 t2 = tb[r];
      if (t2.x >= 0) {
        const TB* B = blkbuf + (size_t)st * rows * SB + (size_t)r * SB;
        const TZ* z = xs + (size_t)r * Nst;
        if (my_sl != 0 && t2.y) {
          int l = 0;
          for (; l + 1 < N; l += 2) {              // A_lr^T row k = column k of A_lr
            const TB b0 = B[(size_t)l * N + k], b1 = B[(size_t)(l + 1) * N + k];
#pragma unroll
            for (int q = 0; q < Ng; ++q) { Pol::fma(acc[q], b0, z[q * N + l]); Pol::fma(acc2[q], b1, z[q * N + l + 1]); }
          }
          if (l < N) {
            const TB b0 = B[(size_t)l * N + k];
#pragma unroll
            for (int q = 0; q < Ng; ++q) Pol::fma(acc[q], b0, z[q * N + l]);
          }
        } else {
          const TB* Bk = B + (size_t)k * N;
          int l = k;                               // row k walked from l = k (bank-conflict-free skew)
          int ll = 0;
          for (; ll + 1 < N; ll += 2) {
            const int l1 = (l + 1 == N) ? 0 : l + 1;
            const TB b0 = Bk[l], b1 = Bk[l1];
#pragma unroll
            for (int q = 0; q < Ng; ++q) { Pol::fma(acc[q], b0, z[q * N + l]); Pol::fma(acc2[q], b1, z[q * N + l1]); }
            l = (l1 + 1 == N) ? 0 : l1 + 1;
          }
          if (ll < N) {
            const TB b0 = Bk[l];
#pragma unroll
            for (int q = 0; q < Ng; ++q) Pol::fma(acc[q], b0, z[q * N + l]);
          }
        }
#pragma unroll
        for (int q = 0; q < Ng; ++q) Pol::add(acc[q], acc2[q]);
      }
#pragma unroll
      for (int q = 0; q < Ng; ++q) part[((size_t)r * Ng + q) * N + k] = acc[q];
    }
    named_bar_sync(1, nct);
    if (lane == 0) mbar_arrive(&empty[st]);                   // blocks and raw x of this stage are free
    for (int idx = ct; idx < TPB * Nst; idx += nct) {
      const int tl = idx / Nst, o = idx - tl * Nst, q = o / N, k = o - q * N;
      const int i = g * TPB + tl;
      if (i >= a.ne) continue;
      Real v;
      if (a.tacc_identity) {
        Acc t = part[((size_t)(tl * 5) * Ng + q) * N + k];
        for (int sl = 1; sl < 5; ++sl) Pol::add(t, part[((size_t)(tl * 5 + sl) * Ng + q) * N + k]);
        v = Pol::value(t);
      } else {
        v = 0;
        for (int b = 0; b < Ng; ++b) {
          Acc t = part[((size_t)(tl * 5) * Ng + b) * N + k];
          for (int sl = 1; sl < 5; ++sl) Pol::add(t, part[((size_t)(tl * 5 + sl) * Ng + b) * N + k]);
          v += a.Tacc[q * Ng + b] * Pol::value(t);
        }
      }
      v *= a.scale;
      if (a.pinned && i == 0 && k == 0) v = a.pin_diag * (Real)x[o];
      y[(size_t)i * Nst + o] = (typename Pol::YOut)v;
    }
  }
  if (s_abort && ct == 0) {
    // bounded wait for any stage the producer may still be filling
    for (int q = 0; q < S; ++q) {
      long spins = 0;
      while (!mbar_wait_hint(&full[q], (uint32_t)(((it + q) / S) & 1)) && ++spins < kSpin) {
      }
    }
  }
}

// ------------------------------------------------------------------ block copies and vectors
template <typename TB>
__global__ void k_to_lp(int64_t nblk, int NN, int SB, const double* __restrict__ src, TB* __restrict__ dst);
template <>
__global__ void k_to_lp<float>(int64_t nblk, int NN, int SB, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nblk * SB; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / SB;
    const int o = (int)(e % SB);
    dst[e] = o < NN ? (float)src[b * NN + o] : 0.0f;
  }
}
template <>
__global__ void k_to_lp<__nv_bfloat16>(int64_t nblk, int NN, int SB, const double* __restrict__ src,
                                       __nv_bfloat16* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nblk * SB; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / SB;
    const int o = (int)(e % SB);
    dst[e] = __float2bfloat16_rn(o < NN ? (float)src[b * NN + o] : 0.0f);
  }
}

template <typename TB>
static cudaError_t build_lp(stdg_solver* s, int64_t ne, int64_t nf, int N, const double* Bdiag, const double* Aoff,
                            void** Bd, void** Ao, int* SB, cudaStream_t st) {
  const int align = 16 / (int)sizeof(TB);
  const int sb = ((N * N + align - 1) / align) * align;
  cudaError_t e = dev_alloc_cuda(s, Bd, (size_t)ne * sb * sizeof(TB));
  if (e != cudaSuccess) return e;
  e = dev_alloc_cuda(s, Ao, (size_t)nf * sb * sizeof(TB));
  if (e != cudaSuccess) return e;
  k_to_lp<TB><<<1216, 256, 0, st>>>(ne, N * N, sb, Bdiag, static_cast<TB*>(*Bd));
  k_to_lp<TB><<<1216, 256, 0, st>>>(nf, N * N, sb, Aoff, static_cast<TB*>(*Ao));
  *SB = sb;
  return cudaGetLastError();
}

cudaError_t lp_build_blocks(stdg_solver* s, int kind) {
  cudaError_t e;
  if (kind == STDG_PREC_MIXED_BF16)
    e = build_lp<__nv_bfloat16>(s, s->ne, s->nf, s->N, s->Bdiag, s->Aoff, &s->lpB, &s->lpA, &s->lpSB, s->stream);
  else
    e = build_lp<float>(s, s->ne, s->nf, s->N, s->Bdiag, s->Aoff, &s->lpB, &s->lpA, &s->lpSB, s->stream);
  if (e == cudaSuccess) s->lpkind = kind;
  return e;
}

// (hi, lo) binary32 pairs of the FP64 blocks, stride padded to a multiple of 2 pairs (16 bytes)
__global__ void k_to_df(int64_t nblk, int NN, int SB, const double* __restrict__ src, float2* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nblk * SB; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / SB;
    const int o = (int)(e % SB);
    const double v = o < NN ? src[b * NN + o] : 0.0;
    const float hi = (float)v;
    dst[e] = make_float2(hi, (float)(v - (double)hi));
  }
}

cudaError_t df_build_blocks(stdg_solver* s) {
  const int sb = ((s->N * s->N + 1) / 2) * 2;
  cudaError_t e = dev_alloc_cuda(s, &s->dfB, (size_t)s->ne * sb * sizeof(float2));
  if (e != cudaSuccess) return e;
  e = dev_alloc_cuda(s, &s->dfA, (size_t)s->nf * sb * sizeof(float2));
  if (e != cudaSuccess) return e;
  k_to_df<<<1216, 256, 0, s->stream>>>(s->ne, s->N * s->N, sb, s->Bdiag, static_cast<float2*>(s->dfB));
  k_to_df<<<1216, 256, 0, s->stream>>>(s->nf, s->N * s->N, sb, s->Aoff, static_cast<float2*>(s->dfA));
  s->dfSB = sb;
  return cudaGetLastError();
}

// tets per stage: at most 384 consumer threads, and at most ~24 KB of blocks per stage (so that
// several CTAs share an SM)
int lp_tets_per_block(int N, size_t block_bytes) {
  int t = 384 / (5 * N);
  const int tb = (int)(24576 / (5 * block_bytes));
  if (tb < t) t = tb;
  if (t < 1) t = 1;
  if (t > 16) t = 16;
  return t;
}

template <typename Pol>
static size_t tma_smem_bytes(int N, int Ng, int SB, int TPB) {
  const size_t rows = (size_t)TPB * 5, xlen = rows * N * Ng;
  const size_t stage_blk = rows * SB * sizeof(typename Pol::TB);
  return kWsStages * stage_blk + align16((size_t)kWsStages * xlen * sizeof(typename Pol::XIn)) +
         align16(xlen * sizeof(typename Pol::TZ)) + align16(xlen * sizeof(typename Pol::Acc)) +
         align16((size_t)kWsStages * rows * sizeof(int2)) + align16(2 * kWsStages * 8);
}

template <typename Pol, int NG>
static cudaError_t launch_tma_ng(stdg_solver* s, const TmaArgs<Pol>& a, const typename Pol::XIn* x,
                                 typename Pol::YOut* y, size_t smem, int threads) {
  cudaError_t e = cudaFuncSetAttribute(k_apply_tma<Pol, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int key = (int)sizeof(typename Pol::TB);
  if (s->tma_grid[key] == 0) {
    int per = 0, nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_tma<Pol, NG>, threads, smem);
    s->tma_grid[key] = nsm * (per > 0 ? per : 1);
  }
  k_apply_tma<Pol, NG><<<s->tma_grid[key], threads, smem, s->stream>>>(a, x, y);
  return cudaGetLastError();
}

template <typename Pol>
static cudaError_t launch_tma(stdg_solver* s, const typename Pol::TB* Bd, const typename Pol::TB* Ao, int SB,
                              const typename Pol::XIn* x, typename Pol::YOut* y, int pinned, int kron, double scale,
                              double pin_diag) {
  TmaArgs<Pol> a{};
  a.ne = (int)s->ne; a.N = s->N; a.Ng = s->Ng; a.SB = SB;
  a.TPB = lp_tets_per_block(s->N, (size_t)SB * sizeof(typename Pol::TB));
  a.t2f = s->dm.t2f; a.t2n = s->dm.t2n; a.left = s->dm.left;
  a.gface = reinterpret_cast<const int4*>(s->gface); a.gnbr = reinterpret_cast<const int4*>(s->gnbr);
  a.Bd = Bd; a.Ao = Ao;
  a.scale = (typename Pol::Real)scale; a.pin_diag = (typename Pol::Real)pin_diag;
  a.tacc_identity = kron; a.pinned = pinned;
  for (int q = 0; q < s->Ng * s->Ng; ++q) a.Tacc[q] = (typename Pol::Real)s->tm.Tp[q];
  a.err = s->derr;
  const size_t smem = tma_smem_bytes<Pol>(s->N, s->Ng, SB, a.TPB);
  const int threads = 32 + ((a.TPB * 5 * s->N + 31) / 32) * 32;   // producer warp + consumers
  switch (s->Ng) {
    case 1: return launch_tma_ng<Pol, 1>(s, a, x, y, smem, threads);
    case 2: return launch_tma_ng<Pol, 2>(s, a, x, y, smem, threads);
    case 3: return launch_tma_ng<Pol, 3>(s, a, x, y, smem, threads);
    case 4: return launch_tma_ng<Pol, 4>(s, a, x, y, smem, threads);
    default: return launch_tma_ng<Pol, 5>(s, a, x, y, smem, threads);
  }
}

cudaError_t launch_apply_lp(stdg_solver* s, const float* x, float* y, int pinned, int kron, float scale, float pin_diag,
                            double* dotpart) {
  if (s->op_warp) return launch_apply_warp_lp(s, x, y, pinned, kron, scale, pin_diag, dotpart);
  if (dotpart) return cudaErrorNotSupported;      // the block-staged kernels write no dot partials
  if (s->lpkind == STDG_PREC_MIXED_BF16)
    return launch_tma<PolBF16>(s, static_cast<const __nv_bfloat16*>(s->lpB), static_cast<const __nv_bfloat16*>(s->lpA),
                               s->lpSB, x, y, pinned, kron, scale, pin_diag);
  return launch_tma<PolF32>(s, static_cast<const float*>(s->lpB), static_cast<const float*>(s->lpA), s->lpSB, x, y,
                            pinned, kron, scale, pin_diag);
}

cudaError_t launch_apply_df(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale,
                            double pin_diag) {
  if (s->op_warp) return launch_apply_warp_df(s, x, y, pinned, kron, scale, pin_diag);
  return launch_tma<PolDF>(s, static_cast<const float2*>(s->dfB), static_cast<const float2*>(s->dfA), s->dfSB, x, y,
                           pinned, kron, scale, pin_diag);
}

// ------------------------------------------------------------------ binary32 Krylov vectors
constexpr int kLpBlocks = 1216;
__device__ inline double lp_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// Block-reduce `cnt` binary32 per-thread partials (cnt <= 8) into part[blockIdx.x * stride + c]: binary32
// within a warp (five shuffle-adds; binary64 ones would cost 5 cnt FP64-pipe operations per thread, tens
// of microseconds per launch on sm_103a), binary64 across the warps, in a fixed order.
template <int MAXC>
__device__ inline void lp_block_store(const float (&v)[MAXC], int cnt, double* part, int stride) {
  __shared__ double red[8][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    if (c >= cnt) break;
    float t = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) red[c][w] = (double)t;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
    part[blockIdx.x * stride + threadIdx.x] = t;
  }
}
// Column dots of binary32 vectors: one thread per (tet, row) pair covering all Ng columns, binary32
// sums per thread (about ten pairs each), binary64 across threads (the binary64 pipe is 1/64 of
// the binary32 rate on sm_103a, so no per-element binary64 work)
__global__ void __launch_bounds__(256) k_lp_coldot(int64_t ne, int N, int Ng, const float* __restrict__ x,
                                                  const float* __restrict__ y, double* part) {
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int Nst = N * Ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int64_t o = i * Nst + (e - i * N);
    for (int a = 0; a < Ng; ++a) acc[a] = fmaf(x[o + a * N], y[o + a * N], acc[a]);
  }
  lp_block_store(acc, Ng, part, Ng);
}
struct LpTp { float v[kMaxNg * kMaxNg]; };
// x += alpha_a p; r -= alpha_a q; with want, partials of r.r per column and of ||(I (x) Tp) r||^2
__global__ void __launch_bounds__(256) k_lp_cg_update(int64_t ne, int N, int Ng, const double* __restrict__ alpha,
                                                     float* __restrict__ x, float* __restrict__ r,
                                                     const float* __restrict__ p, const float* __restrict__ q,
                                                     LpTp Tp, double* part, int want) {
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float al[kMaxNg];
  for (int a = 0; a < Ng; ++a) al[a] = (float)alpha[a];
  const int Nst = N * Ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int64_t o0 = i * Nst + (e - i * N);
    float rv[kMaxNg];
    for (int a = 0; a < Ng; ++a) {
      const int64_t o = o0 + a * N;
      x[o] = fmaf(al[a], p[o], x[o]);
      const float rn = fmaf(-al[a], q[o], r[o]);
      r[o] = rn;
      rv[a] = rn;
      if (want) acc[a] = fmaf(rn, rn, acc[a]);
    }
    if (want)
      for (int a = 0; a < Ng; ++a) {
        float w = 0.0f;
        for (int b = 0; b < Ng; ++b) w = fmaf(Tp.v[a * Ng + b], rv[b], w);
        acc[Ng] = fmaf(w, w, acc[Ng]);
      }
  }
  if (!want) return;
  lp_block_store(acc, Ng + 1, part, Ng + 1);
}
__global__ void k_lp_cg_dir(int64_t ne, int N, int Ng, const double* __restrict__ beta, const float* __restrict__ z,
                            float* __restrict__ p) {
  float be[kMaxNg];
  for (int a = 0; a < Ng; ++a) be[a] = (float)beta[a];
  const int Nst = N * Ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int64_t o = i * Nst + (e - i * N);
    for (int a = 0; a < Ng; ++a) p[o + a * N] = fmaf(be[a], p[o + a * N], z[o + a * N]);
  }
}
// z_i = Binv_i r_i per time column: thread per (tet, row k) covering all Ng columns, so each entry of
// the (symmetric) binary32 inverse is read once; several tets per block pass; partials of r.z per
// column.  NC: N at compile time (0: runtime).
template <int NC>
__global__ void __launch_bounds__(256) k_lp_bjacobi(int ne, int Nrt, int Ng, const float* __restrict__ Binv,
                                                    const float* __restrict__ r, float* __restrict__ z, double* part) {
  extern __shared__ float rs[];
  const int N = NC ? NC : Nrt;
  const int Nst = N * Ng;
  const int TB = blockDim.x / N;                    // tets per pass
  const size_t NN = (size_t)N * N;
  float acc[kMaxNg] = {0, 0, 0, 0, 0};
  const int tl = threadIdx.x / N, k = threadIdx.x - tl * N;
  for (int i0 = blockIdx.x * TB; i0 < ne; i0 += gridDim.x * TB) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < TB * Nst; idx += blockDim.x) {
      const int i = i0 + idx / Nst;
      rs[idx] = i < ne ? r[(size_t)i0 * Nst + idx] : 0.0f;
    }
    __syncthreads();
    const int i = i0 + tl;
    if (tl < TB && i < ne) {
      const float* B = Binv + (size_t)i * NN + k;   // symmetric: column k, coalesced over k
      const float* rr = rs + tl * Nst;
      float sa[kMaxNg] = {0, 0, 0, 0, 0};
#pragma unroll 4
      for (int l = 0; l < N; ++l) {
        const float b = B[(size_t)l * N];
#pragma unroll
        for (int a = 0; a < kMaxNg; ++a)
          if (a < Ng) sa[a] = fmaf(b, rr[a * N + l], sa[a]);
      }
#pragma unroll
      for (int a = 0; a < kMaxNg; ++a)
        if (a < Ng) {
          z[(size_t)i * Nst + a * N + k] = sa[a];
          acc[a] = fmaf(sa[a], rr[a * N + k], acc[a]);
        }
    }
  }
  __syncthreads();
  lp_block_store(acc, Ng, part, Ng);
}
// The update and the preconditioner of one binary32 CG iteration in one pass: x += alpha_a p,
// r -= alpha_a q (alpha from the device), then z = Binv r from the updated rows kept in shared
// memory (thread per (tet, row), all columns), and partials of r.z per column.  With N and Ng at
// compile time (NC, NGC != 0) a thread's N column loads of Binv are all issued before its first
// multiply-add, so each warp keeps N loads in flight.
template <int NC, int NGC>
__global__ void __launch_bounds__(256) k_lp_update_bj(int ne, int Nrt, int Ngrt, const double* __restrict__ alpha,
                                                     float* __restrict__ x, float* __restrict__ r,
                                                     const float* __restrict__ p, const float* __restrict__ q,
                                                     const float* __restrict__ Binv, float* __restrict__ z,
                                                     double* part) {
  constexpr int NGM = NGC ? NGC : kMaxNg;
  extern __shared__ float rs[];
  __shared__ float s_al[kMaxNg];
  const int Ng = NGC ? NGC : Ngrt;
  if (threadIdx.x < Ng) s_al[threadIdx.x] = (float)alpha[threadIdx.x];
  const int N = NC ? NC : Nrt;
  const int Nst = N * Ng;
  const int TB = blockDim.x / N;
  const size_t NN = (size_t)N * N;
  float acc[NGM];
#pragma unroll
  for (int a = 0; a < NGM; ++a) acc[a] = 0.0f;
  const int tl = threadIdx.x / N, k = threadIdx.x - tl * N;
  for (int i0 = blockIdx.x * TB; i0 < ne; i0 += gridDim.x * TB) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < TB * Nst; idx += blockDim.x) {
      if (i0 + idx / Nst >= ne) continue;
      const size_t g = (size_t)i0 * Nst + idx;
      const float al = s_al[(idx % Nst) / N];
      x[g] = fmaf(al, p[g], x[g]);
      const float rn = fmaf(-al, q[g], r[g]);
      r[g] = rn;
      rs[idx] = rn;
    }
    __syncthreads();
    const int i = i0 + tl;
    if (tl < TB && i < ne) {
      const float* B = Binv + (size_t)i * NN + k;
      const float* rr = rs + tl * Nst;
      float sa[NGM];
#pragma unroll
      for (int a = 0; a < NGM; ++a) sa[a] = 0.0f;
      if constexpr (NC > 0) {
        float bv[NC];
#pragma unroll
        for (int l2 = 0; l2 < NC; ++l2) bv[l2] = __ldg(B + (size_t)l2 * NC);
#pragma unroll
        for (int l2 = 0; l2 < NC; ++l2)
#pragma unroll
          for (int a = 0; a < NGM; ++a)
            if (NGC || a < Ng) sa[a] = fmaf(bv[l2], rr[a * NC + l2], sa[a]);
      } else {
#pragma unroll 4
        for (int l2 = 0; l2 < N; ++l2) {
          const float b = B[(size_t)l2 * N];
#pragma unroll
          for (int a = 0; a < NGM; ++a)
            if (a < Ng) sa[a] = fmaf(b, rr[a * N + l2], sa[a]);
        }
      }
#pragma unroll
      for (int a = 0; a < NGM; ++a)
        if (NGC || a < Ng) {
          z[(size_t)i * Nst + a * N + k] = sa[a];
          acc[a] = fmaf(sa[a], rr[a * N + k], acc[a]);
        }
    }
  }
  __syncthreads();
  lp_block_store(acc, Ng, part, Ng);
}

void lp_update_bjacobi(cudaStream_t st, int ne, int N, int Ng, const double* alpha, float* x, float* r, const float* p,
                       const float* q, const float* Binv, float* z, double* part) {
  const int TB = 256 / N;
  const size_t smem = (size_t)TB * N * Ng * sizeof(float);
  if (N == 35 && Ng == 5) k_lp_update_bj<35, 5><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, alpha, x, r, p, q, Binv, z, part);
  else if (N == 20 && Ng == 2) k_lp_update_bj<20, 2><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, alpha, x, r, p, q, Binv, z, part);
  else if (N == 35) k_lp_update_bj<35, 0><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, alpha, x, r, p, q, Binv, z, part);
  else if (N == 20) k_lp_update_bj<20, 0><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, alpha, x, r, p, q, Binv, z, part);
  else if (N == 10) k_lp_update_bj<10, 0><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, alpha, x, r, p, q, Binv, z, part);
  else k_lp_update_bj<0, 0><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, alpha, x, r, p, q, Binv, z, part);
}

// out = float(coef * Sum_b M[a][b] in[b])   (time mixing + conversion)
__global__ void k_lp_from64(int64_t ne, int N, int Ng, const double* __restrict__ M, double coef,
                            const double* __restrict__ in, float* __restrict__ out) {
  const int Nst = N * Ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int k = (int)(e % N);
    for (int a = 0; a < Ng; ++a) {
      double s = 0.0;
      for (int b = 0; b < Ng; ++b) s = fma(M[a * Ng + b], in[i * Nst + b * N + k], s);
      out[i * Nst + a * N + k] = (float)(coef * s);
    }
  }
}
__global__ void k_lp_accum(int64_t n, double scale, const float* __restrict__ d, double* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = fma(scale, (double)d[e], x[e]);
}
__global__ void k_lp_scale(int64_t n, float s, float* __restrict__ p) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    p[e] *= s;
}
__global__ void k_lp_f32s(int64_t n, double sc, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)(sc * in[e]);
}
__global__ void k_lp_f32(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

LpKernels lp_kernels() {
  LpKernels k;
  k.coldot = [](cudaStream_t st, int64_t n, int N, int Ng, const float* x, const float* y, double* part) {
    k_lp_coldot<<<kLpBlocks, 256, 0, st>>>(n / ((int64_t)N * Ng), N, Ng, x, y, part);
  };
  k.update = [](cudaStream_t st, int64_t ne, int N, int Ng, const double* alpha, float* x, float* r, const float* p,
                const float* q, const double* Tp, double* part, int want) {
    LpTp t{};
    for (int c = 0; c < Ng * Ng; ++c) t.v[c] = (float)Tp[c];
    k_lp_cg_update<<<kLpBlocks, 256, 0, st>>>(ne, N, Ng, alpha, x, r, p, q, t, part, want);
  };
  k.dir = [](cudaStream_t st, int64_t n, int N, int Ng, const double* beta, const float* z, float* p) {
    k_lp_cg_dir<<<kLpBlocks, 256, 0, st>>>(n / ((int64_t)N * Ng), N, Ng, beta, z, p);
  };
  k.bjacobi = [](cudaStream_t st, int ne, int N, int Ng, const float* Binv, const float* r, float* z, double* part) {
    const int TB = 256 / N;                         // one thread per (tet, row)
    const size_t smem = (size_t)TB * N * Ng * sizeof(float);
    switch (N) {
      case 20: k_lp_bjacobi<20><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, Binv, r, z, part); break;
      case 35: k_lp_bjacobi<35><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, Binv, r, z, part); break;
      case 10: k_lp_bjacobi<10><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, Binv, r, z, part); break;
      default: k_lp_bjacobi<0><<<kLpBlocks, 256, smem, st>>>(ne, N, Ng, Binv, r, z, part); break;
    }
  };
  k.from64 = [](cudaStream_t st, int64_t ne, int N, int Ng, const double* Mdev, double coef, const double* in, float* out) {
    k_lp_from64<<<kLpBlocks, 256, 0, st>>>(ne, N, Ng, Mdev, coef, in, out);
  };
  k.accum = [](cudaStream_t st, int64_t n, double scale, const float* d, double* x) {
    k_lp_accum<<<kLpBlocks, 256, 0, st>>>(n, scale, d, x);
  };
  k.f32 = [](cudaStream_t st, int64_t n, const double* in, float* out) { k_lp_f32<<<kLpBlocks, 256, 0, st>>>(n, in, out); };
  k.scale = [](cudaStream_t st, int64_t n, float s, float* p) { k_lp_scale<<<kLpBlocks, 256, 0, st>>>(n, s, p); };
  k.f32s = [](cudaStream_t st, int64_t n, double sc, const double* in, float* out) {
    k_lp_f32s<<<kLpBlocks, 256, 0, st>>>(n, sc, in, out);
  };
  return k;
}

}  // namespace stdg

