// Bodies of the second stage of an objective/gradient evaluation (finalize_kernel and
// finalize_reduce_kernel in reduce.cu), shared with kernels that fuse them with the step
// that consumes their result (the solver's line-search step, solver.cu).  The arithmetic and
// its order are the same wherever they run, so fused and separate launches give identical
// results.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace rpca {

// Gradient assembly.  Blocks [0, a.gu) handle the m x B side, FIN_EPT elements per thread
// (strided by the blocks of that side, so that each round is coalesced and all rounds' loads
// are in flight together): the column-split partials of PU are summed and
// G_U = lam_L U_t - PU (fg) or D Bv = -PU (apply) is written.  The other blocks handle the n x B side, 32 elements
// per block: eight groups of 32 threads each sum every eighth row-block partial of PV
// (coalesced across consecutive columns, loaded FIN_VB at a time, all in flight) and the
// groups are added in a fixed order.
// Elementwise work is float32 (the partial sums are float32 already); each block's dot
// products (||x_t||^2, g.d, ||g||^2) go to float-float for the fixed-order block sums.
// bid: this block's index in the launch's grid of a.gu + fin_grid_v(n, B) blocks.
RPCA_DEV void finalize_body(const FinArgs& a, const unsigned bid) {
  __shared__ float wsum[32][3];
  __shared__ float vs[8][32];
  __shared__ float alpha_s;
  // Conversions from float64 and 64-bit divisions run on the float64 pipe, which is narrow on
  // this GPU: the step is converted once per block, indices use 32-bit unsigned division
  // (m B and n B are below 2^31, checked when the context is created).
  if (threadIdx.x == 0) alpha_s = a.alpha_dev ? (float)*a.alpha_dev : a.alpha;
  __syncthreads();
  const float alpha = alpha_s;
  const float lam = a.lam_f;
  const unsigned mB = (unsigned)a.m * (unsigned)a.B, nB = (unsigned)a.n * (unsigned)a.B;
  float nrm_f = 0.f, gd_f = 0.f, gg_f = 0.f;
  if ((int)bid < a.gu && a.vec4) {
    // Four consecutive elements per thread (one row range of one column: m is a multiple of
    // 4), every array read and written as float4; the column-split partials are added in the
    // same order as below.
    const unsigned e = (bid * blockDim.x + threadIdx.x) * 4u;
    if (a.side != 2 && e < mB) {
      const int64_t cstride = (int64_t)a.B * a.mpad;
      const unsigned l = e / (unsigned)a.m, i = e - l * (unsigned)a.m;
      const float* pu = a.PU + (int64_t)l * a.mpad + i;
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
      for (int c = 0; c < a.ncs; ++c) {
        const float4 t = *reinterpret_cast<const float4*>(pu + c * cstride);
        s.x += t.x;
        s.y += t.y;
        s.z += t.z;
        s.w += t.w;
      }
      const float su[4] = {s.x, s.y, s.z, s.w};
      float uu[4] = {0.f, 0.f, 0.f, 0.f}, du[4] = {0.f, 0.f, 0.f, 0.f}, dir[4] = {0.f, 0.f, 0.f, 0.f};
      if (a.mode != FIN_APPLY) {
        const float4 u4 = *reinterpret_cast<const float4*>(a.U + e);
        uu[0] = u4.x, uu[1] = u4.y, uu[2] = u4.z, uu[3] = u4.w;
        if (a.dU) {
          const float4 d4 = *reinterpret_cast<const float4*>(a.dU + e);
          du[0] = d4.x, du[1] = d4.y, du[2] = d4.z, du[3] = d4.w;
        }
        if (a.DU) {
          const float4 d4 = *reinterpret_cast<const float4*>(a.DU + e);
          dir[0] = d4.x, dir[1] = d4.y, dir[2] = d4.z, dir[3] = d4.w;
        }
      }
      float xt[4] = {0.f, 0.f, 0.f, 0.f}, g[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (a.mode != FIN_APPLY) {
          xt[u] = a.dU ? fmaf(alpha, du[u], uu[u]) : uu[u];
          g[u] = a.mode == FIN_FG ? fmaf(lam, xt[u], -su[u]) : -su[u];
        } else {
          g[u] = -su[u];
        }
        nrm_f = fmaf(xt[u], xt[u], nrm_f);
        gd_f = fmaf(g[u], dir[u], gd_f);
        gg_f = fmaf(g[u], g[u], gg_f);
      }
      if (a.mode != FIN_APPLY && a.Ut) *reinterpret_cast<float4*>(a.Ut + e) = make_float4(xt[0], xt[1], xt[2], xt[3]);
      *reinterpret_cast<float4*>(a.GU + e) = make_float4(g[0], g[1], g[2], g[3]);
    }
  } else if ((int)bid < a.gu) {
    // Loads of all FIN_EPT elements first, stores after: a store between them would order
    // the next element's loads after it (the compiler cannot rule out aliasing).
    float su[FIN_EPT], uu[FIN_EPT], du[FIN_EPT], dir[FIN_EPT];
    const int64_t cstride = (int64_t)a.B * a.mpad;
#pragma unroll
    for (int u = 0; u < FIN_EPT; ++u) {
      const unsigned e = (bid + (unsigned)u * (unsigned)a.gu) * blockDim.x + threadIdx.x;
      su[u] = 0.f;
      uu[u] = 0.f;
      du[u] = 0.f;
      dir[u] = 0.f;
      if (a.side != 2 && e < mB) {
        const unsigned l = e / (unsigned)a.m, i = e - l * (unsigned)a.m;
        const float* pu = a.PU + (int64_t)l * a.mpad + i;
        float s = 0.f;
#pragma unroll 8
        for (int c = 0; c < a.ncs; ++c) s += pu[c * cstride];
        su[u] = s;
        if (a.mode != FIN_APPLY) {
          uu[u] = a.U[e];
          if (a.dU) du[u] = a.dU[e];
          if (a.DU) dir[u] = a.DU[e];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < FIN_EPT; ++u) {
      const unsigned e = (bid + (unsigned)u * (unsigned)a.gu) * blockDim.x + threadIdx.x;
      if (a.side != 2 && e < mB) {
        float g, xt = 0.f;
        if (a.mode != FIN_APPLY) {
          xt = a.dU ? fmaf(alpha, du[u], uu[u]) : uu[u];
          g = a.mode == FIN_FG ? fmaf(lam, xt, -su[u]) : -su[u];
          if (a.Ut) a.Ut[e] = xt;
        } else {
          g = -su[u];
        }
        a.GU[e] = g;
        nrm_f = fmaf(xt, xt, nrm_f);
        gd_f = fmaf(g, dir[u], gd_f);
        gg_f = fmaf(g, g, gg_f);
      }
    }
  } else {
    const int q = threadIdx.x >> 5, t = threadIdx.x & 31;
    const unsigned e2 = (bid - a.gu) * 32 + t;
    const bool live = a.side != 1 && e2 < nB;
    unsigned l = 0, j = 0;
    float s = 0.f;
    if (live) {
      l = e2 / (unsigned)a.n;
      j = e2 - l * (unsigned)a.n;
      const float* pv = a.PV + (int64_t)l * a.n + j;
      const int64_t rstride = (int64_t)a.B * a.n;
      for (int r0 = q; r0 < a.nrb; r0 += 8 * FIN_VB) {
        float tv[FIN_VB];
#pragma unroll
        for (int u = 0; u < FIN_VB; ++u) {
          const int r = r0 + 8 * u;
          tv[u] = r < a.nrb ? pv[r * rstride] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < FIN_VB; ++u) s += tv[u];
      }
    }
    vs[q][t] = s;
    __syncthreads();
    if (q == 0 && live) {
      s = ((vs[0][t] + vs[1][t]) + (vs[2][t] + vs[3][t])) + ((vs[4][t] + vs[5][t]) + (vs[6][t] + vs[7][t]));
      float g, xt = 0.f, dir = 0.f;
      if (a.vpart) {
        g = s;  // this row shard's D^T U; the shards' sum and lam_L V come later
      } else if (a.mode != FIN_APPLY) {
        xt = a.V[e2];
        if (a.dV) xt = fmaf(alpha, a.dV[e2], xt);
        g = a.mode == FIN_FG ? fmaf(lam, xt, s) : s;
        if (a.Vt) a.Vt[e2] = xt;
        if (a.DV) dir = a.DV[e2];
      } else {
        g = s;
      }
      a.GV[e2] = g;
      if (!a.vpart) {
        nrm_f = xt * xt;
        gd_f = g * dir;
        gg_f = g * g;
      }
    }
  }
  if (a.mode == FIN_APPLY) return;
  // Warp sums in float32, then the warps in float-float (a float64 sum over the warps, on
  // thread 0, was the longest step of the assembly on GB300).
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nrm_f += __shfl_xor_sync(0xffffffffu, nrm_f, o);
    gd_f += __shfl_xor_sync(0xffffffffu, gd_f, o);
    gg_f += __shfl_xor_sync(0xffffffffu, gg_f, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    wsum[w][0] = nrm_f;
    wsum[w][1] = gd_f;
    wsum[w][2] = gg_f;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int v = threadIdx.x;
    ff2 t = ff_make(wsum[0][v]);
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = ff_add(t, ff_make(wsum[i][v]));
    ff_store(&a.blk[3 * bid + v], t);
  }
}

// One block: fixed-order sums of the finalize partials and of the per-CTA psi sums, in
// float-float (each thread its blocks in order, a warp butterfly, the warps in order).
// out = {f, g.d, ||g||^2, ||x||^2} (written by thread 0).
RPCA_DEV void finalize_reduce_body(const FinArgs& a, int nblocks) {
  __shared__ ff2 wred[32][4];
  __shared__ double res[4];
  ff2 p[4] = {ff_make(0.f), ff_make(0.f), ff_make(0.f), ff_make(0.f)};  // ||x||^2, g.d, ||g||^2, psi
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {  // L2 reads: other blocks may have just written
#pragma unroll
    for (int v = 0; v < 3; ++v) p[v] = ff_add(p[v], ff_load_cg(&a.blk[3 * b + v]));
  }
  for (int b = threadIdx.x; b < a.nctas; b += blockDim.x) p[3] = ff_add(p[3], ff_load_cg(&a.Ppsi[b]));
#pragma unroll
  for (int v = 0; v < 4; ++v) p[v] = warp_ff_sum(p[v]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) wred[w][v] = p[v];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int v = threadIdx.x;
    ff2 t = wred[0][v];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = ff_add(t, wred[i][v]);
    res[v] = ff_to_d(t);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.out[0] = res[3] + 0.5 * a.lam_L * res[0];
    a.out[1] = res[1];
    a.out[2] = res[2];
    a.out[3] = res[0];
  }
}

}  // namespace rpca
