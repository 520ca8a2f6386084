// Warp-per-tet five-point operator kernel template (shared by the per-policy translation units).
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

#include "lp_ptx.cuh"
#include "solver.h"

namespace stdg {

constexpr long kWarpSpin = 20000;   // x <= 1 ms suspend per try_wait

struct WF32 { using TB = float; using XIn = float; using YOut = float; using Real = float; static constexpr int kPlanes = 1; };
struct WBF16 { using TB = __nv_bfloat16; using XIn = float; using YOut = float; using Real = float; static constexpr int kPlanes = 1; };
struct WDF { using TB = float; using XIn = double; using YOut = double; using Real = double; static constexpr int kPlanes = 2; };

struct WarpArgs {
  int ne, N, NR, NP, Nst, S, pinned, kron;
  const int4* gface;            // per tet: (face << 1 | tet is r) or -1, 4 faces
  const int4* gnbr;             // per tet: neighbour tet or -1
  const void* Bd;               // diagonal blocks, padded layout
  const void* Ao;               // face blocks A_lr, padded layout
  uint32_t blk_bytes;           // one padded block (all planes)
  uint32_t plane_elems;         // NR * NP
  uint32_t xraw_off, stage_bytes, z_off, bar_off, warp_bytes;
  uint32_t red_off;             // CTA kernels: partial sums [warp][NR][Ng] of the output rows
  double scale, pin_diag;
  double Tacc[kMaxNg * kMaxNg];
  // viscous operator (Eq. A1_mod): + mass_coef |J_i| (K (x) I) x_i, exact in the input precision
  const double* detJ;
  double mass_coef;
  double Kmass[kMaxNg * kMaxNg];
  double* dotpart;              // optional: per block and column, Sum of x_i . y_i over its tets
  int* err;
};

// four consecutive entries of a row (element index idx, a multiple of 4)
__device__ __forceinline__ void load_row4(const float* B, int idx, float (&b)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(B + idx);
  b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
}
__device__ __forceinline__ void load_row4(const __nv_bfloat16* B, int idx, float (&b)[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(B + idx);
  b[0] = __uint_as_float(v.x << 16); b[1] = __uint_as_float(v.x & 0xFFFF0000u);
  b[2] = __uint_as_float(v.y << 16); b[3] = __uint_as_float(v.y & 0xFFFF0000u);
}
__device__ __forceinline__ float load_one(const float* B, int idx) { return B[idx]; }
__device__ __forceinline__ float load_one(const __nv_bfloat16* B, int idx) { return __bfloat162float(B[idx]); }

__host__ __device__ constexpr int warp_np_c(int N) { return N % 8 == 4 ? N : warp_np_c(N + 1); }
__host__ __device__ constexpr int warp_nr_c(int N) { return (N + 3) / 4 * 4; }

// Binary64-accurate multiply-add from binary32 pairs, (h, l) += (bh + bl)(zh + zl) with the bl zl
// term (relative size 2^-48) left out: the product bh zh split exactly by a fused multiply-add, its
// high part added to h by an error-free sum.  Two independent accumulators at once (the halves of
// the float2 values), in packed binary32 operations (f32x2, sm_100 and later).  nbh = -bh, formed
// once per chunk: pn = nbh zh is the rounded product negated exactly, so no negation per product.
__device__ __forceinline__ void df_fma2(float2& h, float2& l, float2 bh, float2 nbh, float2 bl, float2 zh, float2 zl) {
  const float2 pn = __fmul2_rn(nbh, zh);
  float2 e = __ffma2_rn(bh, zh, pn);              // bh zh - p, exact
  e = __ffma2_rn(bh, zl, e);
  e = __ffma2_rn(bl, zh, e);
  float2 s, t;
  df_two_diff2(h, pn, s, t);                      // h + p = h - pn, error-free
  h = s;
  l = __fadd2_rn(l, __fadd2_rn(t, e));
}

// pair policy: four entries of a block row (stride 1: vector loads of the hi and lo planes) or
// column (stride NP) times the matching z entries; entries (0, 1) and (2, 3) through the two halves
// of (h, l), one accumulator pair per time column
template <int NG, typename TB>
__device__ __forceinline__ void warp_chunk_df2(const TB* B, int stride, uint32_t plane, const float* z, int NR,
                                               int zplane, float2 (&h)[NG], float2 (&l)[NG]) {
  float bh[4], bl[4];
  if (stride == 1) {
    load_row4(B, 0, bh);
    load_row4(B + plane, 0, bl);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      bh[u] = load_one(B, u * stride);
      bl[u] = load_one(B + plane, u * stride);
    }
  }
  const float2 bh01 = make_float2(bh[0], bh[1]), bh23 = make_float2(bh[2], bh[3]);
  const float2 nb01 = make_float2(-bh[0], -bh[1]), nb23 = make_float2(-bh[2], -bh[3]);
  const float2 bl01 = make_float2(bl[0], bl[1]), bl23 = make_float2(bl[2], bl[3]);
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    const float4 zh = *reinterpret_cast<const float4*>(z + q * NR);
    const float4 zl = *reinterpret_cast<const float4*>(z + zplane + q * NR);
    df_fma2(h[q], l[q], bh01, nb01, bl01, make_float2(zh.x, zh.y), make_float2(zl.x, zl.y));
    df_fma2(h[q], l[q], bh23, nb23, bl23, make_float2(zh.z, zh.w), make_float2(zl.z, zl.w));
  }
}

// binary32 policies: the same four-entry chunk with packed multiply-adds, entries (0, 1) and (2, 3)
// in the two halves of one float2 accumulator per time column (fma.rn.f32x2: half the issue slots of
// four scalar multiply-adds, the same binary32 rounding)
template <int NG, typename TB>
__device__ __forceinline__ void warp_chunk2(const TB* B, int stride, const float* z, int NR, float2 (&acc)[NG]) {
  float b[4];
  if (stride == 1) {
    load_row4(B, 0, b);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = load_one(B, u * stride);
  }
  const float2 b01 = make_float2(b[0], b[1]), b23 = make_float2(b[2], b[3]);
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    const float4 zv = *reinterpret_cast<const float4*>(z + q * NR);
    acc[q] = __ffma2_rn(b01, make_float2(zv.x, zv.y), acc[q]);
    acc[q] = __ffma2_rn(b23, make_float2(zv.z, zv.w), acc[q]);
  }
}

// One warp per tet, persistent over a strided stream of tets.  Lane 0 stages the tet's five blocks
// (its diagonal block and the face blocks of its interior faces) by 1-D TMA bulk copies; all lanes
// stage the x rows of the tet and its neighbours by cp.async.  binary32 x goes straight into rows of
// NR entries ([slot][time column][NR], the padding entries zeroed once and never written), the layout
// the products read; binary64 x (pair policy) is split into (hi, lo) planes of the same layout.
// Rows 0..31 of the output: lane k owns row k over all five blocks and all time columns.  Rows
// 32..N-1 (N = 35 at p = 4): one group of 8 lanes per row, each lane summing its share of the four-
// entry chunks, the group reduced by shuffles at the end.  No block-wide barrier anywhere.
template <typename W, int NG, int NC>
__global__ void __launch_bounds__(128, 1) k_apply_warp(WarpArgs a, const typename W::XIn* __restrict__ x,
                                                    typename W::YOut* __restrict__ y) {
  using TB = typename W::TB;
  using XIn = typename W::XIn;
  using Real = typename W::Real;
  constexpr bool kDF = W::kPlanes == 2;
  constexpr bool kRoll = kDF && (NC == 0 || NC > 20);   // large pair kernels: rolled loops
  constexpr bool kPrefetch = kRoll;                     // there: the blocks two tets ahead go to L2 (measured
                                                        // slower for the binary32 kernel)
  extern __shared__ __align__(128) unsigned char wsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  unsigned char* base = wsm + (size_t)warp * a.warp_bytes;
  float* zs = reinterpret_cast<float*>(base + a.z_off);        // pair policy: (hi, lo) planes of z
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + a.bar_off);
  // NC != 0: N known at compile time (row loops fully unrolled, shared-memory offsets immediate)
  const int N = NC ? NC : a.N, NR = NC ? warp_nr_c(NC) : a.NR, NP = NC ? warp_np_c(NC) : a.NP;
  const int Nst = NC ? NC * NG : a.Nst, S = a.S;
  // kernel parameters in the arithmetic type, converted once (a binary64 conversion or compare per
  // output row would go through the 1/64-rate binary64 pipe)
  const Real scale = (Real)a.scale;
  const bool has_mass = a.mass_coef != 0.0, kron = a.kron != 0, pinned = a.pinned != 0;
  Real tacc[NG * NG];
#pragma unroll
  for (int c = 0; c < NG * NG; ++c) tacc[c] = (Real)a.Tacc[c];
  const int zplane = 5 * NG * NR;
  if constexpr (kDF) {
    for (int e = lane; e < 2 * zplane; e += 32) zs[e] = 0.0f;            // padding entries stay 0
  } else {
    for (int st = 0; st < S; ++st) {
      float* xz = reinterpret_cast<float*>(base + (size_t)st * a.stage_bytes + a.xraw_off);
      for (int e = lane; e < zplane; e += 32) xz[e] = 0.0f;
    }
  }
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 33);   // lane 0's expect_tx + 32 cp.async arrivals
    fence_async_smem();
  }
  __syncwarp();

  auto issue = [&](int i, int st, const int4& gf, const int4& gn) {
    unsigned char* sb = base + (size_t)st * a.stage_bytes;
    XIn* xr = reinterpret_cast<XIn*>(sb + a.xraw_off);
    const int fj[4] = {gf.x, gf.y, gf.z, gf.w};
    const int nn[4] = {gn.x, gn.y, gn.z, gn.w};
    if (lane == 0) {
      uint32_t bytes = a.blk_bytes;
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (fj[f] >= 0) bytes += a.blk_bytes;
      fence_async_smem();                         // earlier generic reads of this stage before the copies
      mbar_expect_tx(&bar[st], bytes);
      tma_load_1d(sb, static_cast<const unsigned char*>(a.Bd) + (size_t)i * a.blk_bytes, a.blk_bytes, &bar[st]);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (fj[f] >= 0)
          tma_load_1d(sb + (size_t)(f + 1) * a.blk_bytes,
                      static_cast<const unsigned char*>(a.Ao) + (size_t)(fj[f] >> 1) * a.blk_bytes, a.blk_bytes,
                      &bar[st]);
    }
#pragma unroll
    for (int sl = 0; sl < 5; ++sl) {
      const int nb = sl == 0 ? i : (fj[sl - 1] >= 0 ? nn[sl - 1] : -1);
      if (nb < 0) continue;
      const XIn* src = x + (size_t)nb * Nst;
      if constexpr (kDF) {
        for (int o = lane; o < Nst; o += 32) cp_async<sizeof(XIn)>(xr + sl * Nst + o, src + o);
      } else {
#pragma unroll
        for (int q = 0; q < NG; ++q)
          for (int l = lane; l < N; l += 32) cp_async<sizeof(XIn)>(xr + (sl * NG + q) * NR + l, src + q * N + l);
      }
    }
    cp_async_mbar_arrive_noinc(&bar[st]);
  };

  const int nw = gridDim.x * wpc;
  float dacc[NG];                                 // x_i . y_i of this lane's rows (dotpart)
#pragma unroll
  for (int q = 0; q < NG; ++q) dacc[q] = 0.0f;
  int i = blockIdx.x * wpc + warp;
  const int4 none = make_int4(-1, -1, -1, -1);
  int4 gf_c = none, gn_c = none, gf_n = none, gn_n = none;
  // iteration it uses stage it % S in its use number it / S (mbarrier phase parity (it / S) & 1)
  bool abort = false, next_issued = false;
  int it = 0;
  if (i < a.ne) {
    gf_c = a.gface[i]; gn_c = a.gnbr[i];
    issue(i, 0, gf_c, gn_c);
    if (S == 2 && i + nw < a.ne) { gf_n = a.gface[i + nw]; gn_n = a.gnbr[i + nw]; }
  }
  for (; i < a.ne; i += nw, ++it) {
    const int st = S == 2 ? (it & 1) : 0;
    const int inx = i + nw;
    const int4 gf = gf_c, gn = gn_c;
    next_issued = false;
    if (S == 2 && inx < a.ne) {                   // next tet's copies run while this one computes
      issue(inx, st ^ 1, gf_n, gn_n);
      next_issued = true;
      gf_c = gf_n; gn_c = gn_n;
      if (inx + nw < a.ne) { gf_n = a.gface[inx + nw]; gn_n = a.gnbr[inx + nw]; }
    }
    {
      long spins = 0;
      const uint32_t par = (uint32_t)((it / S) & 1);
      while (!mbar_wait_hint(&bar[st], par))
        if (++spins > kWarpSpin) { abort = true; break; }
    }
    if (__any_sync(0xffffffffu, abort)) { abort = true; break; }
    __syncwarp();
    if (kPrefetch && lane == 0 && i + S * nw < a.ne) {   // the blocks after the next staged tet: towards L2
      const int ip = i + S * nw;
      const int4 gp = a.gface[ip];
      const int fp[4] = {gp.x, gp.y, gp.z, gp.w};
      bulk_prefetch_l2(static_cast<const unsigned char*>(a.Bd) + (size_t)ip * a.blk_bytes, a.blk_bytes);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (fp[f] >= 0)
          bulk_prefetch_l2(static_cast<const unsigned char*>(a.Ao) + (size_t)(fp[f] >> 1) * a.blk_bytes, a.blk_bytes);
    }
    unsigned char* sb = base + (size_t)st * a.stage_bytes;
    XIn* xr = reinterpret_cast<XIn*>(sb + a.xraw_off);
    const int fj[4] = {gf.x, gf.y, gf.z, gf.w};
    const int nn[4] = {gn.x, gn.y, gn.z, gn.w};
    // pinned entries (constant mode of tet 0, every time column) read as 0
    if constexpr (kDF) {
#pragma unroll
      for (int sl = 0; sl < 5; ++sl) {
        const int nb = sl == 0 ? i : (fj[sl - 1] >= 0 ? nn[sl - 1] : -1);
        if (nb < 0) continue;
#pragma unroll
        for (int q = 0; q < NG; ++q)
          for (int l = lane; l < N; l += 32) {
            XIn v = xr[sl * Nst + q * N + l];
            if (pinned && nb == 0 && l == 0) v = (XIn)0;
            const float2 hl = df_split(v);
            float* zq = zs + (sl * NG + q) * NR + l;
            zq[0] = hl.x;
            zq[zplane] = hl.y;
          }
      }
    } else if (pinned) {
#pragma unroll
      for (int sl = 0; sl < 5; ++sl) {
        const int nb = sl == 0 ? i : (fj[sl - 1] >= 0 ? nn[sl - 1] : -1);
        if (nb == 0 && lane < NG) xr[(sl * NG + lane) * NR] = (XIn)0;
      }
    }
    __syncwarp();
    const float* zb = kDF ? zs : reinterpret_cast<const float*>(xr);   // z rows [slot][q][NR]
    const TB* blk = reinterpret_cast<const TB*>(sb);
    const int blk_elems = (int)(a.blk_bytes / sizeof(TB));
    int pres = 1, trm = 0;                        // per slot: block present / read transposed
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      pres |= (fj[f] >= 0 ? 1 : 0) << (f + 1);
      trm |= (fj[f] >= 0 && (fj[f] & 1) ? 1 : 0) << (f + 1);
    }
    // output row k of tet i from its sums v over the five blocks: time mixing, scale, mass term,
    // pin, store, x.y partials
    auto finish = [&](int k, const Real (&v)[NG]) {
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        Real o = v[q];
        if (!kron) {
          o = 0;
#pragma unroll
          for (int b = 0; b < NG; ++b) o += tacc[q * NG + b] * v[b];
        }
        o *= scale;
        if (has_mass) {                           // x_i as staged (binary64 for the pair policy)
          Real m = 0;
#pragma unroll
          for (int b = 0; b < NG; ++b)
            m += (Real)a.Kmass[q * NG + b] * (Real)(kDF ? xr[b * N + k] : xr[b * NR + k]);
          o += (Real)(a.mass_coef * a.detJ[i]) * m;
        }
        if (pinned && i == 0 && k == 0) o = (Real)a.pin_diag * (Real)x[q * N];
        y[(size_t)i * Nst + q * N + k] = (typename W::YOut)o;
        if (a.dotpart) dacc[q] += (float)((Real)x[(size_t)i * Nst + q * N + k] * o);
      }
    };
    const int nmain = N < 32 ? N : 32;
    if (lane < nmain) {
      const int k = lane;
      float2 dh[NG], dl[NG];                      // pair policy: packed (hi, lo) accumulators per column
      float2 c0[NG], c1[NG];                      // binary32 policies: two packed accumulators per column
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        dh[q] = dl[q] = make_float2(0.0f, 0.0f);
        c0[q] = c1[q] = make_float2(0.0f, 0.0f);
      }
      // pair policy at N > 20 (about 200 instructions per chunk): the block and chunk loops stay rolled,
      // as fully unrolled code outgrows the instruction cache
      auto block_main = [&](int sl) {
        if (!((pres >> sl) & 1)) return;
        const TB* B = blk + sl * blk_elems;
        const float* z = zb + sl * NG * NR;
        if (!((trm >> sl) & 1)) {                 // row k of the block, 4 entries per vector load
          const TB* Br = B + k * NP;
#pragma unroll (kRoll ? 1 : 8)
          for (int l = 0; l < NR; l += 8) {
            if constexpr (kDF) {
              warp_chunk_df2<NG>(Br + l, 1, a.plane_elems, z + l, NR, zplane, dh, dl);
              if (l + 4 < NR) warp_chunk_df2<NG>(Br + l + 4, 1, a.plane_elems, z + l + 4, NR, zplane, dh, dl);
            } else {
              warp_chunk2<NG>(Br + l, 1, z + l, NR, c0);
              if (l + 4 < NR) warp_chunk2<NG>(Br + l + 4, 1, z + l + 4, NR, c1);
            }
          }
        } else {                                  // column k: A_rl = A_lr^T, one word per lane
          const TB* Bc = B + k;
#pragma unroll (kRoll ? 1 : 8)
          for (int l = 0; l < NR; l += 8) {
            if constexpr (kDF) {
              warp_chunk_df2<NG>(Bc + l * NP, NP, a.plane_elems, z + l, NR, zplane, dh, dl);
              if (l + 4 < NR) warp_chunk_df2<NG>(Bc + (l + 4) * NP, NP, a.plane_elems, z + l + 4, NR, zplane, dh, dl);
            } else {
              warp_chunk2<NG>(Bc + l * NP, NP, z + l, NR, c0);
              if (l + 4 < NR) warp_chunk2<NG>(Bc + (l + 4) * NP, NP, z + l + 4, NR, c1);
            }
          }
        }
      };
      if constexpr (kRoll) {
#pragma unroll 1
        for (int sl = 0; sl < 5; ++sl) block_main(sl);
      } else {
        for (int sl = 0; sl < 5; ++sl) block_main(sl);
      }
      Real v[NG];
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        if constexpr (kDF) {
          float s, t;
          df_two_sum(dh[q].x, dh[q].y, s, t);
          v[q] = (double)s + (double)(t + (dl[q].x + dl[q].y));   // the error terms are ~2^-24 of s
        } else {
          v[q] = (c0[q].x + c0[q].y) + (c1[q].x + c1[q].y);
        }
      }
      finish(k, v);
    }
    if (N > 32) {                                 // rows 32 .. N-1: 8 lanes per row, chunks split
      const int g = lane >> 3, c = lane & 7, r = 32 + g;
      const int nch = NR / 4;
      float2 eh[NG], el[NG], ec[NG];
#pragma unroll
      for (int q = 0; q < NG; ++q) eh[q] = el[q] = ec[q] = make_float2(0.0f, 0.0f);
      if (r < N) {
#pragma unroll (kRoll ? 1 : 5)
        for (int sl = 0; sl < 5; ++sl) {
          if (!((pres >> sl) & 1)) continue;
          const TB* B = blk + sl * blk_elems;
          const float* z = zb + sl * NG * NR;
          const bool tr = (trm >> sl) & 1;
          for (int ch = c; ch < nch; ch += 8) {
            const int l = 4 * ch;
            if constexpr (kDF) {
              if (!tr) warp_chunk_df2<NG>(B + r * NP + l, 1, a.plane_elems, z + l, NR, zplane, eh, el);
              else warp_chunk_df2<NG>(B + l * NP + r, NP, a.plane_elems, z + l, NR, zplane, eh, el);
            } else {
              if (!tr) warp_chunk2<NG>(B + r * NP + l, 1, z + l, NR, ec);
              else warp_chunk2<NG>(B + l * NP + r, NP, z + l, NR, ec);
            }
          }
        }
      }
      Real v[NG];
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        float h, e;
        if constexpr (kDF) {
          df_two_sum(eh[q].x, eh[q].y, h, e);
          e += el[q].x + el[q].y;
        } else {
          h = ec[q].x + ec[q].y;
          e = 0.0f;
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {         // within the 8-lane group
          const float oh = __shfl_xor_sync(0xffffffffu, h, o), oe = __shfl_xor_sync(0xffffffffu, e, o);
          if constexpr (kDF) {
            float s, t;
            df_two_sum(h, oh, s, t);
            h = s;
            e = e + oe + t;
          } else {
            h += oh;
          }
        }
        if constexpr (kDF) v[q] = (double)h + (double)e;
        else v[q] = h;
      }
      if (c == 0 && r < N) finish(r, v);
    }
    __syncwarp();
    if (S == 1 && inx < a.ne) {                   // one stage: the next tet's copies start now
      gf_c = a.gface[inx]; gn_c = a.gnbr[inx];
      issue(inx, 0, gf_c, gn_c);
    }
  }
  if (a.dotpart) {                                // fixed order: lanes by shuffle, warps by index
    __shared__ float wdot[4][kMaxNg];
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      float v = dacc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) wdot[warp][q] = v;
    }
    __syncthreads();                              // every warp of the block reaches this point
    if (threadIdx.x < NG) {
      double t = 0.0;
      for (int w = 0; w < wpc; ++w) t += (double)wdot[w][threadIdx.x];
      a.dotpart[(size_t)blockIdx.x * NG + threadIdx.x] = t;
    }
  }
  if (abort) {
    if (lane == 0) atomicExch(a.err, 1);
    // bounded wait for this warp's copies in flight: the stage of iteration it and, when it was
    // issued, the stage of iteration it + 1
    const int st = S == 2 ? (it & 1) : 0;
    long spins = 0;
    while (!mbar_wait_hint(&bar[st], (uint32_t)((it / S) & 1)) && ++spins < kWarpSpin) {
    }
    if (next_issued) {
      spins = 0;
      while (!mbar_wait_hint(&bar[st ^ 1], (uint32_t)(((it + 1) / S) & 1)) && ++spins < kWarpSpin) {
      }
    }
  }
}

// The same operator with WPC warps sharing each staged tet, for the pair policy at N = 35, where the
// warp kernel fits only three warps per SM.  One CTA per stride of tets (persistent grid); S stages
// (two where two CTAs still fit: the next tet's copies land while this one computes).  Thread 0 stages the
// five blocks by 1-D TMA bulk copies, all threads stage the x rows by cp.async, on the stage's
// mbarrier.  The (block, four-column chunk) products of a tet are dealt out round robin: warp w
// takes products w, w + WPC, ..., one lane per output row 0..31, and for rows 32..N-1 one group of
// 8 lanes per row over the same products.  Each warp leaves its partial sums in shared memory;
// one thread per output row adds the WPC partials and finishes the row (time mixing, scale, mass
// term, pin, store, x.y partials).  Per tet: wait, prepare (pin; pair policy: x split into hi/lo
// planes), barrier, products, barrier, rows, barrier, refill the stage.  Every wait is bounded.
// component k (0..3) of an int4 by selects (no local-memory array for a runtime k)
__device__ __forceinline__ int pick4(const int4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
// the tet whose x slot sl (0: tet i itself, 1..4: the neighbour across face sl - 1) holds, or -1
__device__ __forceinline__ int slot_tet(int i, int sl, const int4& gf, const int4& gn) {
  return sl == 0 ? i : (pick4(gf, sl - 1) >= 0 ? pick4(gn, sl - 1) : -1);
}

template <typename W, int NG, int NC, int WPC>
__global__ void __launch_bounds__(32 * WPC) k_apply_cta(WarpArgs a, const typename W::XIn* __restrict__ x,
                                                       typename W::YOut* __restrict__ y) {
  using TB = typename W::TB;
  using XIn = typename W::XIn;
  using Real = typename W::Real;
  constexpr bool kDF = W::kPlanes == 2;
  using Part = typename std::conditional<kDF, float2, float>::type;
  constexpr int NT = 32 * WPC;
  extern __shared__ __align__(128) unsigned char csm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* zs = reinterpret_cast<float*>(csm + a.z_off);
  Part* red = reinterpret_cast<Part*>(csm + a.red_off);
  uint64_t* bar = reinterpret_cast<uint64_t*>(csm + a.bar_off);
  const int N = NC ? NC : a.N, NR = NC ? warp_nr_c(NC) : a.NR, NP = NC ? warp_np_c(NC) : a.NP;
  const int Nst = NC ? NC * NG : a.Nst, S = a.S;
  const int nch = NR / 4, npair = 5 * nch;
  const Real scale = (Real)a.scale;
  const bool has_mass = a.mass_coef != 0.0, kron = a.kron != 0, pinned = a.pinned != 0;
  const int zplane = 5 * NG * NR;
  __shared__ Real sT[NG * NG], sK[NG * NG];       // time matrices in the arithmetic type, converted once
  if (tid < NG * NG) { sT[tid] = (Real)a.Tacc[tid]; sK[tid] = (Real)a.Kmass[tid]; }
  if constexpr (kDF) {
    for (int e = tid; e < 2 * zplane; e += NT) zs[e] = 0.0f;             // padding entries stay 0
  } else {
    for (int st = 0; st < S; ++st) {
      float* xz = reinterpret_cast<float*>(csm + (size_t)st * a.stage_bytes + a.xraw_off);
      for (int e = tid; e < zplane; e += NT) xz[e] = 0.0f;
    }
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1 + NT);   // thread 0's expect_tx + NT cp.async arrivals
    fence_async_smem();
  }
  __syncthreads();

  auto issue = [&](int i, int st) {
    unsigned char* sb = csm + (size_t)st * a.stage_bytes;
    XIn* xr = reinterpret_cast<XIn*>(sb + a.xraw_off);
    const int4 gf = a.gface[i], gn = a.gnbr[i];
    const int fj[4] = {gf.x, gf.y, gf.z, gf.w};
    if (tid == 0) {
      uint32_t bytes = a.blk_bytes;
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (fj[f] >= 0) bytes += a.blk_bytes;
      fence_async_smem();                         // earlier generic reads of this stage before the copies
      mbar_expect_tx(&bar[st], bytes);
      tma_load_1d(sb, static_cast<const unsigned char*>(a.Bd) + (size_t)i * a.blk_bytes, a.blk_bytes, &bar[st]);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (fj[f] >= 0)
          tma_load_1d(sb + (size_t)(f + 1) * a.blk_bytes,
                      static_cast<const unsigned char*>(a.Ao) + (size_t)(fj[f] >> 1) * a.blk_bytes, a.blk_bytes,
                      &bar[st]);
    }
    if constexpr (kDF) {
      for (int idx = tid; idx < 5 * Nst; idx += NT) {
        const int sl = idx / Nst, o = idx - sl * Nst;
        const int nb = slot_tet(i, sl, gf, gn);
        if (nb >= 0) cp_async<sizeof(XIn)>(xr + idx, x + (size_t)nb * Nst + o);
      }
    } else {
      for (int idx = tid; idx < 5 * NG * N; idx += NT) {
        const int rw = idx / N, l = idx - rw * N, sl = rw / NG;   // row rw = (slot, time column)
        const int nb = slot_tet(i, sl, gf, gn);
        if (nb >= 0) cp_async<sizeof(XIn)>(xr + rw * NR + l, x + (size_t)nb * Nst + (rw - sl * NG) * N + l);
      }
    }
    cp_async_mbar_arrive_noinc(&bar[st]);
  };

  const int grid = gridDim.x;
  float dacc[NG];                                 // x_i . y_i of this thread's rows (dotpart)
#pragma unroll
  for (int q = 0; q < NG; ++q) dacc[q] = 0.0f;
  int i = blockIdx.x;
  for (int k = 0; k < S; ++k)
    if (i + k * grid < a.ne) issue(i + k * grid, k);
  bool abort = false;
  int it = 0;
  for (; i < a.ne; i += grid, ++it) {
    const int st = S == 2 ? (it & 1) : 0;
    {
      long spins = 0;
      const uint32_t par = (uint32_t)((it / S) & 1);
      while (!mbar_wait_hint(&bar[st], par))
        if (++spins > kWarpSpin) { abort = true; break; }
    }
    if (__syncthreads_or(abort)) { abort = true; break; }
    if (kDF && tid == 0 && i + S * grid < a.ne) {   // the blocks after the next staged tet: towards L2
      const int ip = i + S * grid;
      const int4 gp = a.gface[ip];
      const int fp[4] = {gp.x, gp.y, gp.z, gp.w};
      bulk_prefetch_l2(static_cast<const unsigned char*>(a.Bd) + (size_t)ip * a.blk_bytes, a.blk_bytes);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (fp[f] >= 0)
          bulk_prefetch_l2(static_cast<const unsigned char*>(a.Ao) + (size_t)(fp[f] >> 1) * a.blk_bytes, a.blk_bytes);
    }
    unsigned char* sb = csm + (size_t)st * a.stage_bytes;
    XIn* xr = reinterpret_cast<XIn*>(sb + a.xraw_off);
    const int4 gf = a.gface[i], gn = a.gnbr[i];
    const int fj[4] = {gf.x, gf.y, gf.z, gf.w};
    // pinned entries (constant mode of tet 0, every time column) read as 0
    if constexpr (kDF) {
      for (int idx = tid; idx < 5 * NG * N; idx += NT) {
        const int rw = idx / N, l = idx - rw * N, sl = rw / NG;
        const int nb = slot_tet(i, sl, gf, gn);
        if (nb < 0) continue;
        XIn v = xr[sl * Nst + (rw - sl * NG) * N + l];
        if (pinned && nb == 0 && l == 0) v = (XIn)0;
        const float2 hl = df_split(v);
        zs[rw * NR + l] = hl.x;
        zs[zplane + rw * NR + l] = hl.y;
      }
    } else if (pinned && tid < 5 * NG) {
      const int nb = slot_tet(i, tid / NG, gf, gn);
      if (nb == 0) xr[tid * NR] = (XIn)0;
    }
    __syncthreads();
    const float* zb = kDF ? zs : reinterpret_cast<const float*>(xr);   // z rows [slot][q][NR]
    const TB* blk = reinterpret_cast<const TB*>(sb);
    const int blk_elems = (int)(a.blk_bytes / sizeof(TB));
    int pres = 1, trm = 0;                        // per slot: block present / read transposed
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      pres |= (fj[f] >= 0 ? 1 : 0) << (f + 1);
      trm |= (fj[f] >= 0 && (fj[f] & 1) ? 1 : 0) << (f + 1);
    }
    // rows 0..31: lane k, this warp's share of the products
    if (lane < N) {
      const int k = lane;
      float2 dh[NG], dl[NG], c0[NG];
#pragma unroll
      for (int q = 0; q < NG; ++q) dh[q] = dl[q] = c0[q] = make_float2(0.0f, 0.0f);
#pragma unroll 1
      for (int pr = warp; pr < npair; pr += WPC) {
        const int sl = pr / nch, l = 4 * (pr - sl * nch);
        if (!((pres >> sl) & 1)) continue;
        const TB* B = blk + sl * blk_elems;
        const float* z = zb + sl * NG * NR + l;
        const bool tr = (trm >> sl) & 1;
        if constexpr (kDF) {
          if (!tr) warp_chunk_df2<NG>(B + k * NP + l, 1, a.plane_elems, z, NR, zplane, dh, dl);
          else warp_chunk_df2<NG>(B + l * NP + k, NP, a.plane_elems, z, NR, zplane, dh, dl);
        } else {
          if (!tr) warp_chunk2<NG>(B + k * NP + l, 1, z, NR, c0);
          else warp_chunk2<NG>(B + l * NP + k, NP, z, NR, c0);
        }
      }
      Part* rp = red + ((size_t)warp * NR + k) * NG;
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        if constexpr (kDF) {
          float s, t;
          df_two_sum(dh[q].x, dh[q].y, s, t);
          rp[q] = make_float2(s, t + (dl[q].x + dl[q].y));
        } else {
          rp[q] = c0[q].x + c0[q].y;
        }
      }
    }
    if (N > 32) {                                 // rows 32 .. N-1: 8 lanes per row over the warp's products
      const int g = lane >> 3, c = lane & 7, r = 32 + g;
      float2 eh[NG], el[NG], ec[NG];
#pragma unroll
      for (int q = 0; q < NG; ++q) eh[q] = el[q] = ec[q] = make_float2(0.0f, 0.0f);
      if (r < N) {
#pragma unroll 1
        for (int pr = warp + WPC * c; pr < npair; pr += 8 * WPC) {
          const int sl = pr / nch, l = 4 * (pr - sl * nch);
          if (!((pres >> sl) & 1)) continue;
          const TB* B = blk + sl * blk_elems;
          const float* z = zb + sl * NG * NR + l;
          const bool tr = (trm >> sl) & 1;
          if constexpr (kDF) {
            if (!tr) warp_chunk_df2<NG>(B + r * NP + l, 1, a.plane_elems, z, NR, zplane, eh, el);
            else warp_chunk_df2<NG>(B + l * NP + r, NP, a.plane_elems, z, NR, zplane, eh, el);
          } else {
            if (!tr) warp_chunk2<NG>(B + r * NP + l, 1, z, NR, ec);
            else warp_chunk2<NG>(B + l * NP + r, NP, z, NR, ec);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        float h, e;
        if constexpr (kDF) {
          df_two_sum(eh[q].x, eh[q].y, h, e);
          e += el[q].x + el[q].y;
        } else {
          h = ec[q].x + ec[q].y;
          e = 0.0f;
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {         // within the 8-lane group
          const float oh = __shfl_xor_sync(0xffffffffu, h, o), oe = __shfl_xor_sync(0xffffffffu, e, o);
          if constexpr (kDF) {
            float s, t;
            df_two_sum(h, oh, s, t);
            h = s;
            e = e + oe + t;
          } else {
            h += oh;
          }
        }
        if (c == 0 && r < N) {
          if constexpr (kDF) red[((size_t)warp * NR + r) * NG + q] = make_float2(h, e);
          else red[((size_t)warp * NR + r) * NG + q] = h;
        }
      }
    }
    __syncthreads();
    // output rows: the WPC partials of each, then time mixing, scale, mass term, pin, store, x.y
    for (int k = tid; k < N; k += NT) {
      Real v[NG];
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        if constexpr (kDF) {
          float h = 0.0f, e = 0.0f;
#pragma unroll
          for (int w = 0; w < WPC; ++w) {
            const float2 pw = red[((size_t)w * NR + k) * NG + q];
            float s, t;
            df_two_sum(h, pw.x, s, t);
            h = s;
            e += pw.y + t;
          }
          v[q] = (double)h + (double)e;
        } else {
          float h = 0.0f;
#pragma unroll
          for (int w = 0; w < WPC; ++w) h += red[((size_t)w * NR + k) * NG + q];
          v[q] = h;
        }
      }
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        Real o = v[q];
        if (!kron) {
          o = 0;
#pragma unroll
          for (int b = 0; b < NG; ++b) o += sT[q * NG + b] * v[b];
        }
        o *= scale;
        if (has_mass) {                           // x_i as staged (binary64 for the pair policy)
          Real m = 0;
#pragma unroll
          for (int b = 0; b < NG; ++b) m += sK[q * NG + b] * (Real)(kDF ? xr[b * N + k] : xr[b * NR + k]);
          o += (Real)(a.mass_coef * a.detJ[i]) * m;
        }
        if (pinned && i == 0 && k == 0) o = (Real)a.pin_diag * (Real)x[q * N];
        y[(size_t)i * Nst + q * N + k] = (typename W::YOut)o;
        if (a.dotpart) dacc[q] += (float)((Real)x[(size_t)i * Nst + q * N + k] * o);
      }
    }
    __syncthreads();                              // stage st and the partials are free again
    if (i + S * grid < a.ne) issue(i + S * grid, st);
  }
  if (a.dotpart) {                                // fixed order: lanes by shuffle, warps by index
    __shared__ float wdot[WPC][kMaxNg];
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      float v = dacc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) wdot[warp][q] = v;
    }
    __syncthreads();                              // every thread of the block reaches this point
    if (tid < NG) {
      double t = 0.0;
      for (int w = 0; w < WPC; ++w) t += (double)wdot[w][tid];
      a.dotpart[(size_t)blockIdx.x * NG + tid] = t;
    }
  }
  if (abort) {
    if (tid == 0) atomicExch(a.err, 1);
    // bounded wait for the copies in flight: the stages of iterations it .. it + S - 1 that were issued
    for (int k = 0; k < S; ++k) {
      if (i + k * grid >= a.ne) break;
      const int st = S == 2 ? ((it + k) & 1) : 0;
      long spins = 0;
      while (!mbar_wait_hint(&bar[st], (uint32_t)(((it + k) / S) & 1)) && ++spins < kWarpSpin) {
      }
    }
  }
}

// padded block copies: dst block b = planes x NR x NP, zero outside N x N
template <typename TB, int PLANES>
__global__ void k_to_padded(int64_t nblk, int N, int NR, int NP, const double* __restrict__ src, TB* __restrict__ dst,
                            const double* __restrict__ src2 = nullptr, double c2 = 0.0) {
  const int64_t per = (int64_t)PLANES * NR * NP;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nblk * per; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per;
    const int rem = (int)(e - b * per);
    const int plane = rem / (NR * NP);
    const int rc = rem - plane * NR * NP;
    const int r = rc / NP, c = rc - r * NP;
    double v = (r < N && c < N) ? src[b * N * N + r * N + c] : 0.0;
    if (src2 && r < N && c < N) v += c2 * src2[b * N * N + r * N + c];
    if constexpr (sizeof(TB) == 2) {
      dst[e] = __float2bfloat16_rn((float)v);
    } else if constexpr (PLANES == 2) {
      const float hi = (float)v;
      dst[e] = plane == 0 ? hi : (float)(v - (double)hi);
    } else {
      dst[e] = (float)v;
    }
  }
}

static int warp_np(int N) { int np = N; while (np % 8 != 4) ++np; return np; }
static int warp_nr(int N) { return (N + 3) / 4 * 4; }
static uint32_t a16(size_t b) { return (uint32_t)((b + 15) & ~(size_t)15); }

template <typename W>
static cudaError_t ensure_warp_blocks(stdg_solver* s, void** Bd, void** Ao) {
  if (*Bd) return cudaSuccess;
  using TB = typename W::TB;
  const int N = s->N, NR = warp_nr(N), NP = warp_np(N);
  const size_t per = (size_t)W::kPlanes * NR * NP;
  cudaError_t e = dev_alloc_cuda(s, Bd, (size_t)s->ne * per * sizeof(TB));
  if (e != cudaSuccess) return e;
  e = dev_alloc_cuda(s, Ao, (size_t)s->nf * per * sizeof(TB));
  if (e != cudaSuccess) return e;
  k_to_padded<TB, W::kPlanes><<<1216, 256, 0, s->stream>>>(s->ne, N, NR, NP, s->Bdiag, static_cast<TB*>(*Bd));
  k_to_padded<TB, W::kPlanes><<<1216, 256, 0, s->stream>>>(s->nf, N, NR, NP, s->Aoff, static_cast<TB*>(*Ao));
  s->nlaunch += 2;
  return cudaGetLastError();
}

// padded copy of the viscous diagonal blocks B_i - Bvisc_i (Eq. A1_mod, with the face blocks A_lr)
template <typename W>
static cudaError_t ensure_warp_visc_diag(stdg_solver* s, void** Bv) {
  if (*Bv || !s->Bvisc) return cudaSuccess;
  using TB = typename W::TB;
  const int N = s->N, NR = warp_nr(N), NP = warp_np(N);
  cudaError_t e = dev_alloc_cuda(s, Bv, (size_t)s->ne * W::kPlanes * NR * NP * sizeof(TB));
  if (e != cudaSuccess) return e;
  k_to_padded<TB, W::kPlanes><<<1216, 256, 0, s->stream>>>(s->ne, N, NR, NP, s->Bdiag, static_cast<TB*>(*Bv), s->Bvisc, -1.0);
  ++s->nlaunch;
  return cudaGetLastError();
}

// Per warp: S stages of [5 blocks | x], then (pair policy only) the (hi, lo) z planes, then the S
// mbarriers.  binary32 x is staged in rows of NR entries per time column, binary64 x as it is.
static WarpArgs warp_layout(const stdg_solver* s, size_t tb, int planes, size_t xin, int S) {
  WarpArgs a{};
  a.ne = (int)s->ne; a.N = s->N; a.NR = warp_nr(s->N); a.NP = warp_np(s->N); a.Nst = s->Nst; a.S = S;
  a.plane_elems = (uint32_t)(a.NR * a.NP);
  a.blk_bytes = (uint32_t)(planes * a.plane_elems * tb);
  a.xraw_off = 5 * a.blk_bytes;
  const bool df = planes == 2;
  a.stage_bytes = a.xraw_off + (df ? a16((size_t)5 * s->Nst * xin) : a16((size_t)5 * s->Ng * a.NR * xin));
  a.z_off = S * a.stage_bytes;
  a.bar_off = a.z_off + (df ? a16((size_t)planes * 5 * s->Ng * a.NR * sizeof(float)) : 0);
  a.warp_bytes = a16(a.bar_off + 2 * sizeof(uint64_t));
  return a;
}

// CTA kernels: the warp layout's stages and z planes, then the partial sums, then S mbarriers
// (warp_bytes: bytes per CTA)
static WarpArgs cta_layout(const stdg_solver* s, size_t tb, int planes, size_t xin, int S, int wpc) {
  WarpArgs a = warp_layout(s, tb, planes, xin, S);
  a.red_off = a.bar_off;
  a.bar_off = a16(a.red_off + (size_t)wpc * a.NR * s->Ng * (planes == 2 ? 8 : 4));
  a.warp_bytes = a16(a.bar_off + (size_t)S * sizeof(uint64_t));
  return a;
}

// warps per CTA of the CTA kernels (pair policy): one 72 KB stage each at N = 35, three CTAs per SM
constexpr int kCtaWarps = 4;

// The CTA kernels serve the pair policy at N > 20, where one tet's products are long enough to
// share among warps (N = 35: 19.2 -> 11.7 ms per application at 384,000 tets, the warp kernel fitting
// three warps per SM); for the binary32 policies and at N <= 20 the per-tet work is too short for
// three CTA barriers and the serial row pass (measured 1.4-2x slower), so the warp kernels serve.
template <typename W>
static bool use_cta(const stdg_solver* s) {
  return s->op_cta != 0 && W::kPlanes == 2 && s->N > 20;
}

template <typename W>
static WarpArgs warp_args(const stdg_solver* s) {
  if (use_cta<W>(s)) {
    // two stages when two CTAs fit on an SM with them, else one
    WarpArgs a = cta_layout(s, sizeof(typename W::TB), W::kPlanes, sizeof(typename W::XIn), 2, kCtaWarps);
    if ((size_t)a.warp_bytes * 2 > 226 * 1024)
      a = cta_layout(s, sizeof(typename W::TB), W::kPlanes, sizeof(typename W::XIn), 1, kCtaWarps);
    return a;
  }
  // two stages when ten warps fit on an SM with them, else one (more warps hide the latency)
  WarpArgs a = warp_layout(s, sizeof(typename W::TB), W::kPlanes, sizeof(typename W::XIn), 2);
  if ((size_t)a.warp_bytes * 10 > 228 * 1024) a = warp_layout(s, sizeof(typename W::TB), W::kPlanes, sizeof(typename W::XIn), 1);
  return a;
}

template <typename W>
static constexpr int warp_kind() { return W::kPlanes == 2 ? 2 : (sizeof(typename W::TB) == 4 ? 1 : 0); }

template <typename W>
using WarpKernel = void (*)(WarpArgs, const typename W::XIn*, typename W::YOut*);

// the instantiation for this N: compile-time N for p = 2, 3, 4, runtime N otherwise (CTA kernels:
// pair policy only, see use_cta)
template <typename W, int NG>
static WarpKernel<W> warp_kernel(int N, bool cta) {
  if constexpr (W::kPlanes == 2) {
    if (cta) return N == 35 ? k_apply_cta<W, NG, 35, kCtaWarps> : k_apply_cta<W, NG, 0, kCtaWarps>;
  }
  switch (N) {
    case 10: return k_apply_warp<W, NG, 10>;
    case 20: return k_apply_warp<W, NG, 20>;
    case 35: return k_apply_warp<W, NG, 35>;
    default: return k_apply_warp<W, NG, 0>;
  }
}

// Launch shape (warps per CTA, persistent grid) from the occupancy of this layout; sets the
// kernel's dynamic shared-memory limit.  Host-side setup: must not run during stream capture.
template <typename W, int NG>
static cudaError_t warp_configure(stdg_solver* s) {
  const WarpArgs a = warp_args<W>(s);
  const WarpKernel<W> kern = warp_kernel<W, NG>(s->N, use_cta<W>(s));
  int& grid = s->warp_grid[warp_kind<W>() * 8 + NG];
  int& wpc = s->warp_wpc[warp_kind<W>() * 8 + NG];
  if (grid != 0) return cudaSuccess;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  if (use_cta<W>(s)) {                            // fixed warps per CTA, as many CTAs as fit
    constexpr int C = kCtaWarps;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.warp_bytes);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * C, a.warp_bytes);
    if (e != cudaSuccess) return e;
    if (per == 0) return cudaErrorInvalidConfiguration;
    wpc = C;
    grid = nsm * per;
    return cudaSuccess;
  }
  int best = 0, bw = 1;
  for (int c : {4, 2, 1}) {
    const size_t smem = (size_t)c * a.warp_bytes;
    if (smem > 227 * 1024) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) continue;
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * c, smem);
    if (per * c > best) { best = per * c; bw = c; }
  }
  cudaGetLastError();
  if (best == 0) return cudaErrorInvalidConfiguration;      // the blocks of one tet do not fit on an SM
  wpc = bw;
  grid = nsm * (best / bw);
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((size_t)wpc * a.warp_bytes));
}

template <typename W>
static cudaError_t warp_prepare_t(stdg_solver* s, void** Bd, void** Ao) {
  cudaError_t e = ensure_warp_blocks<W>(s, Bd, Ao);
  if (e != cudaSuccess) return e;
  switch (s->Ng) {
    case 1: return warp_configure<W, 1>(s);
    case 2: return warp_configure<W, 2>(s);
    case 3: return warp_configure<W, 3>(s);
    case 4: return warp_configure<W, 4>(s);
    default: return warp_configure<W, 5>(s);
  }
}

template <typename W, int NG>
static cudaError_t launch_warp_ng(stdg_solver* s, const WarpArgs& a, const typename W::XIn* x, typename W::YOut* y) {
  const int grid = s->warp_grid[warp_kind<W>() * 8 + NG], wpc = s->warp_wpc[warp_kind<W>() * 8 + NG];
  if (grid == 0) return cudaErrorNotReady;                  // warp_prepare has not run
  const bool cta = use_cta<W>(s);
  const size_t smem = cta ? (size_t)a.warp_bytes : (size_t)wpc * a.warp_bytes;
  warp_kernel<W, NG>(s->N, cta)<<<grid, 32 * wpc, smem, s->stream>>>(a, x, y);
  return cudaGetLastError();
}

template <typename W>
static cudaError_t launch_warp(stdg_solver* s, const void* Bd, const void* Ao, const typename W::XIn* x,
                               typename W::YOut* y, int pinned, int kron, double scale, double pin_diag,
                               double mass_coef = 0.0, const double* Kmass = nullptr, double* dotpart = nullptr) {
  if (!Bd) return cudaErrorNotReady;
  WarpArgs a = warp_args<W>(s);
  a.gface = reinterpret_cast<const int4*>(s->gface);
  a.gnbr = reinterpret_cast<const int4*>(s->gnbr);
  a.Bd = Bd; a.Ao = Ao;
  a.pinned = pinned; a.kron = kron; a.scale = scale; a.pin_diag = pin_diag;
  for (int q = 0; q < s->Ng * s->Ng; ++q) a.Tacc[q] = s->tm.Tp[q];
  a.detJ = s->dm.detJ;
  a.mass_coef = Kmass ? mass_coef : 0.0;
  a.dotpart = dotpart;
  for (int q = 0; Kmass && q < s->Ng * s->Ng; ++q) a.Kmass[q] = Kmass[q];
  a.err = s->derr;
  switch (s->Ng) {
    case 1: return launch_warp_ng<W, 1>(s, a, x, y);
    case 2: return launch_warp_ng<W, 2>(s, a, x, y);
    case 3: return launch_warp_ng<W, 3>(s, a, x, y);
    case 4: return launch_warp_ng<W, 4>(s, a, x, y);
    default: return launch_warp_ng<W, 5>(s, a, x, y);
  }
}

}  // namespace stdg
