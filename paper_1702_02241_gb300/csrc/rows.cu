// Row-partitioned evaluation of the objective and gradient (the multi-GPU form of the pass).
//
// With X = [X_1; ...; X_G] split by rows over G devices and U = [U_1; ...; U_G] split the same
// way (V shared), the objective of Eq. (Thm5) and its gradient (Sec. 3.2) separate as
//   F      = sum_g ( sum_{Omega_g} psi(U_g V^T - X_g) + lam_L/2 ||U_g||^2 ) + lam_L/2 ||V||^2,
//   G_{U_g} = D_g V + lam_L U_g                  (complete on device g),
//   G_V    = sum_g D_g^T U_g + lam_L V           (one sum over the devices),
// so one evaluation exchanges n k + 1 values: each device computes its shard's terms with the
// fused pass (rpca_fg_rows), the partials [D_g^T U_g | f_g] are summed over the devices (an
// all-reduce, done by the caller's communicator), and rpca_fg_rows_finish adds the shared V
// terms.  The paper scales the video problem by its row and column counts (Sec. 5.4); this is
// the data-parallel split of that pass.
#include <cmath>

#include "common.cuh"
#include "ctx.h"

namespace rpca {

// gV = PV + lam V and block partials of ||V||^2 (float32 within a thread's four elements,
// float64 across the block's warps).
__global__ void __launch_bounds__(256) rows_finish_kernel(const float* V, const float* PV, int64_t nk, float lam,
                                                         float* gV, double* blk) {
  __shared__ double scr[8];
  float acc = 0.f;
  const int64_t base = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 4;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t e = base + u;
    if (e < nk) {
      const float v = V[e];
      gV[e] = fmaf(lam, v, PV[e]);
      acc = fmaf(v, v, acc);
    }
  }
  double d = (double)acc;
  d = warp_sum_d(d);
  if ((threadIdx.x & 31) == 0) scr[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += scr[w];
    blk[blockIdx.x] = s;
  }
}

// Fixed-order sum of the block partials: out[0] = f_sum + lam_L / 2 ||V||^2.
__global__ void __launch_bounds__(256) rows_finish_reduce_kernel(const double* blk, int nblocks, double lam_L,
                                                                double f_sum, double* out) {
  __shared__ double scr[8];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 256) s += __ldcg(&blk[b]);
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) scr[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += scr[w];
    out[0] = f_sum + 0.5 * lam_L * t;
  }
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_fg_rows(rpca_ctx* c, const float* U, const float* V, double* f_part, float* gU,
                                    float* PV) {
  if (!c) return RPCA_EINVAL;
  if (!U || !V || !gU || !PV) return set_err(c, RPCA_EINVAL, "U, V, gU and PV are required");
  if (c->lk) return set_err(c, RPCA_EUNSUPPORTED, "the row-shard pass is built for k <= 16");
  FgLaunch L;
  L.U = U;
  L.V = V;
  L.GU = gU;
  L.GV = PV;
  L.out = c->ws.out;
  L.vpart = 1;
  rpca_status s = launch_fg(c, eval_plan(c), L, c->stream);
  if (s != RPCA_OK) return s;
  if (f_part) {
    RPCA_CUDA(c, cudaMemcpyAsync(f_part, c->ws.out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((s = check_dev_err(c)) != RPCA_OK) return s;
  }
  return RPCA_OK;
}

extern "C" rpca_status rpca_fg_rows_finish(rpca_ctx* c, const float* V, const float* PV_sum, double f_sum, double* f,
                                           float* gV) {
  if (!c) return RPCA_EINVAL;
  if (!V || !PV_sum || !gV) return set_err(c, RPCA_EINVAL, "V, PV_sum and gV are required");
  if (!std::isfinite(f_sum)) return set_err(c, RPCA_EINVAL, "f_sum is not finite");
  const int64_t nk = (int64_t)c->n * c->k;
  const int nb = (int)((nk + 1023) / 1024);
  if ((size_t)nb > c->ws.blk_n) return set_err(c, RPCA_EUNSUPPORTED, "workspace too small for the V side");
  rows_finish_kernel<<<nb, 256, 0, c->stream>>>(V, PV_sum, nk, (float)c->lam_L, gV, c->ws.blk);
  rows_finish_reduce_kernel<<<1, 256, 0, c->stream>>>(c->ws.blk, nb, c->lam_L, f_sum, c->ws.out);
  count_launches(c, 2);
  RPCA_CUDA(c, cudaGetLastError());
  if (f) {
    RPCA_CUDA(c, cudaMemcpyAsync(f, c->ws.out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
    if (*f < c->F_best) c->F_best = *f;
  }
  return RPCA_OK;
}
