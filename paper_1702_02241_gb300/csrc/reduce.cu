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
#include "fin.cuh"
#include "kernels.h"

namespace rpca {

__global__ void __launch_bounds__(256) finalize_kernel(FinArgs a) {
  if (a.gate != nullptr && *a.gate == 0) return;
  finalize_body(a, blockIdx.x);
}

__global__ void __launch_bounds__(256) finalize_reduce_kernel(FinArgs a, int nblocks) {
  if (a.gate != nullptr && *a.gate == 0) return;
  finalize_reduce_body(a, nblocks);
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
