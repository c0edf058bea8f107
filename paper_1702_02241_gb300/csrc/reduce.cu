// Second stage of one objective/gradient evaluation, and small utility kernels.
//
// finalize_kernel sums the per-CTA partials of fg_kernel in a fixed order and adds the
// factor penalty of Eq. (Thm5):
//   G_U = D V + lam_L U,  G_V = D^T U + lam_L V,
//   f   = sum psi + lam_L/2 (||U||_F^2 + ||V||_F^2)       (all sums over CTAs in float64)
// at the trial point (U + alpha dU, V + alpha dV).  It also returns, in float64, the
// directional derivative g.d along an optional direction and ||g||^2.  The last block to
// finish (atomic ticket) combines the per-block partials in index order, so the result is
// bitwise reproducible.
#include "common.cuh"
#include "kernels.h"

namespace rpca {

__global__ void __launch_bounds__(256) finalize_kernel(FinArgs a) {
  __shared__ double scr[32];
  __shared__ bool is_last;
  if (a.gate != nullptr && *a.gate == 0) return;
  const int64_t mB = (int64_t)a.m * a.B, N = mB + (int64_t)a.n * a.B;
  const float alpha = a.alpha_dev ? (float)*a.alpha_dev : a.alpha;
  double nrm = 0.0, gd = 0.0, gg = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    float g, xt, dir = 0.f;
    if (e < mB) {
      const int l = (int)(e / a.m), i = (int)(e - (int64_t)l * a.m);
      double s = 0.0;
      for (int c = 0; c < a.ncs; ++c) s += (double)a.PU[((int64_t)c * a.B + l) * a.mpad + i];
      if (a.mode != FIN_APPLY) {
        xt = a.U[e];
        if (a.dU) xt = fmaf(alpha, a.dU[e], xt);
        g = a.mode == FIN_FG ? (float)(-s + a.lam_L * (double)xt) : (float)(-s);
        if (a.Ut) a.Ut[e] = xt;
        if (a.DU) dir = a.DU[e];
      } else {
        xt = 0.f;
        g = (float)(-s);
      }
      a.GU[e] = g;
    } else {
      const int64_t e2 = e - mB;
      const int l = (int)(e2 / a.n), j = (int)(e2 - (int64_t)l * a.n);
      double s = 0.0;
      for (int r = 0; r < a.nrb; ++r) s += (double)a.PV[((int64_t)r * a.B + l) * a.n + j];
      if (a.mode != FIN_APPLY) {
        xt = a.V[e2];
        if (a.dV) xt = fmaf(alpha, a.dV[e2], xt);
        g = a.mode == FIN_FG ? (float)(s + a.lam_L * (double)xt) : (float)s;
        if (a.Vt) a.Vt[e2] = xt;
        if (a.DV) dir = a.DV[e2];
      } else {
        xt = 0.f;
        g = (float)s;
      }
      a.GV[e2] = g;
    }
    nrm += (double)xt * (double)xt;
    gd += (double)g * (double)dir;
    gg += (double)g * (double)g;
  }
  if (a.mode == FIN_APPLY) return;
  const double s0 = block_sum_d(nrm, scr);
  const double s1 = block_sum_d(gd, scr);
  const double s2 = block_sum_d(gg, scr);
  if (threadIdx.x == 0) {
    a.blk[3 * blockIdx.x + 0] = s0;
    a.blk[3 * blockIdx.x + 1] = s1;
    a.blk[3 * blockIdx.x + 2] = s2;
    __threadfence();
    const unsigned t = atomicAdd(a.counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double p0 = 0.0, p1 = 0.0, p2 = 0.0, ps = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    p0 += __ldcg(&a.blk[3 * b + 0]);
    p1 += __ldcg(&a.blk[3 * b + 1]);
    p2 += __ldcg(&a.blk[3 * b + 2]);
  }
  for (int b = threadIdx.x; b < a.nctas; b += blockDim.x) ps += __ldcg(&a.Ppsi[b]);
  p0 = block_sum_d(p0, scr);
  p1 = block_sum_d(p1, scr);
  p2 = block_sum_d(p2, scr);
  ps = block_sum_d(ps, scr);
  if (threadIdx.x == 0) {
    a.out[0] = ps + 0.5 * a.lam_L * p0;
    a.out[1] = p1;
    a.out[2] = p2;
    a.out[3] = p0;
    *a.counter = 0u;
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
