// Second stage of one objective/gradient evaluation, and small utility kernels.
//
// finalize_kernel sums the per-CTA partials of fg_kernel in a fixed order and adds the
// factor penalty of Eq. (Thm5):
//   G_U = D V + lam_L U,  G_V = D^T U + lam_L V,
//   f   = sum psi + lam_L/2 (||U||_F^2 + ||V||_F^2)       (sums over CTAs in float64)
// at the trial point (U + alpha dU, V + alpha dV).  It also returns, in float64, the
// directional derivative g.d along an optional direction and ||g||^2.  The last block to
// finish (atomic ticket) combines the per-block partials in index order, so the result is
// bitwise reproducible.
#include "common.cuh"
#include "kernels.h"

namespace rpca {

// Deterministic block sum of three doubles per thread; results valid in thread 0.
RPCA_DEV void block_sum3(double& x, double& y, double& z, double (*scr)[3]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
    z += __shfl_xor_sync(0xffffffffu, z, o);
  }
  __syncthreads();
  if (lane == 0) {
    scr[w][0] = x;
    scr[w][1] = y;
    scr[w][2] = z;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    x = y = z = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      x += scr[i][0];
      y += scr[i][1];
      z += scr[i][2];
    }
  }
}

// Blocks [0, a.gu) handle the m x B side (threads stride over elements, four independent
// loads in flight); blocks [a.gu, gridDim.x) handle the n x B side, one element per warp,
// the lanes splitting the row-block partials (fixed-order shuffle sum).  Each block writes
// its partial dot products; finalize_reduce_kernel combines them (no atomics, no fences).
__global__ void __launch_bounds__(256) finalize_kernel(FinArgs a) {
  __shared__ double scr[32][3];
  if (a.gate != nullptr && *a.gate == 0) return;
  const float alpha = a.alpha_dev ? (float)*a.alpha_dev : a.alpha;
  const float lam = (float)a.lam_L;
  const int64_t mB = (int64_t)a.m * a.B, nB = (int64_t)a.n * a.B;
  // Element-wise work in float32 (GB300's float64 pipe is ~1/64 of float32; the partial
  // sums are float32 already); each thread's dot products go to float64 once at the end.
  float nrm_f = 0.f, gd_f = 0.f, gg_f = 0.f;
  if ((int)blockIdx.x < a.gu) {
    const int64_t stride = (int64_t)a.gu * blockDim.x;
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a.side != 2 && e0 < mB; e0 += 4 * stride) {
      float sv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t e = e0 + u * stride;
        sv[u] = 0.f;
        if (e < mB) {
          const int l = (int)(e / a.m), i = (int)(e - (int64_t)l * a.m);
          for (int c = 0; c < a.ncs; ++c) sv[u] += a.PU[((int64_t)c * a.B + l) * a.mpad + i];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t e = e0 + u * stride;
        if (e >= mB) break;
        const float s = sv[u];
        float g, xt = 0.f, dir = 0.f;
        if (a.mode != FIN_APPLY) {
          xt = a.U[e];
          if (a.dU) xt = fmaf(alpha, a.dU[e], xt);
          g = a.mode == FIN_FG ? fmaf(lam, xt, -s) : -s;
          if (a.Ut) a.Ut[e] = xt;
          if (a.DU) dir = a.DU[e];
        } else {
          g = -s;
        }
        a.GU[e] = g;
        nrm_f = fmaf(xt, xt, nrm_f);
        gd_f = fmaf(g, dir, gd_f);
        gg_f = fmaf(g, g, gg_f);
      }
    }
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)(gridDim.x - a.gu) * (blockDim.x >> 5);
    for (int64_t e2 = (int64_t)(blockIdx.x - a.gu) * (blockDim.x >> 5) + (threadIdx.x >> 5); a.side != 1 && e2 < nB;
         e2 += warps) {
      const int l = (int)(e2 / a.n), j = (int)(e2 - (int64_t)l * a.n);
      float s = 0.f;
      for (int r = lane; r < a.nrb; r += 32) s += a.PV[((int64_t)r * a.B + l) * a.n + j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        float g, xt = 0.f, dir = 0.f;
        if (a.mode != FIN_APPLY) {
          xt = a.V[e2];
          if (a.dV) xt = fmaf(alpha, a.dV[e2], xt);
          g = a.mode == FIN_FG ? fmaf(lam, xt, s) : s;
          if (a.Vt) a.Vt[e2] = xt;
          if (a.DV) dir = a.DV[e2];
        } else {
          g = s;
        }
        a.GV[e2] = g;
        nrm_f = fmaf(xt, xt, nrm_f);
        gd_f = fmaf(g, dir, gd_f);
        gg_f = fmaf(g, g, gg_f);
      }
    }
  }
  if (a.mode == FIN_APPLY) return;
  double nrm = nrm_f, gd = gd_f, gg = gg_f;
  block_sum3(nrm, gd, gg, scr);
  if (threadIdx.x == 0) {
    a.blk[3 * blockIdx.x + 0] = nrm;
    a.blk[3 * blockIdx.x + 1] = gd;
    a.blk[3 * blockIdx.x + 2] = gg;
  }
}

// One block: fixed-order sums of the finalize partials and of the per-CTA psi sums.
// out = {f, g.d, ||g||^2, ||x||^2}.
__global__ void __launch_bounds__(256) finalize_reduce_kernel(FinArgs a, int nblocks) {
  __shared__ double scr[32][3];
  if (a.gate != nullptr && *a.gate == 0) return;
  double p0 = 0.0, p1 = 0.0, p2 = 0.0, ps = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    p0 += a.blk[3 * b + 0];
    p1 += a.blk[3 * b + 1];
    p2 += a.blk[3 * b + 2];
  }
  block_sum3(p0, p1, p2, scr);
  __syncthreads();
  for (int b = threadIdx.x; b < a.nctas; b += blockDim.x) ps += a.Ppsi[b];
  double d1 = 0.0, d2 = 0.0;
  block_sum3(ps, d1, d2, scr);
  if (threadIdx.x == 0) {
    a.out[0] = ps + 0.5 * a.lam_L * p0;
    a.out[1] = p1;
    a.out[2] = p2;
    a.out[3] = p0;
  }
}

// One warp per (word, column): bit b of word w of column j is mask(32 w + b, j) != 0.
__global__ void pack_mask_kernel(const uint8_t* mask, int64_t ldmask, int m, int n, int wpad, uint32_t* bits) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)wpad * n) return;
  const int j = (int)(gw / wpad), w = (int)(gw - (int64_t)j * wpad);
  const int row = w * 32 + lane;
  const bool on = row < m && mask[(int64_t)j * ldmask + row] != 0;
  const uint32_t word = __ballot_sync(0xffffffffu, on);
  if (lane == 0) bits[(int64_t)j * wpad + w] = word;
}

// Counts observed entries of X that are not finite, and observed entries overall.
__global__ void check_x_kernel(const float* X, int64_t ldx, const uint8_t* mask, int64_t ldmask, int m, int n,
                               unsigned long long* bad, unsigned long long* observed) {
  unsigned long long nb = 0, no = 0;
  const int64_t N = (int64_t)m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / m), i = (int)(e - (int64_t)j * m);
    const bool obs = mask == nullptr || mask[(int64_t)j * ldmask + i] != 0;
    if (obs) {
      ++no;
      if (!isfinite(X[(int64_t)j * ldx + i])) ++nb;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
    no += __shfl_xor_sync(0xffffffffu, no, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(bad, nb);
    atomicAdd(observed, no);
  }
}

}  // namespace rpca
