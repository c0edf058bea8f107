// Frank-Wolfe method with marginalization (Sec. 6.2, Algorithm 1) on a dense L: the convex
// program min over ||L||_* <= t of lam_L t + phi(L), phi(L) = sum_Omega psi(L - X) (S
// marginalised).  One iteration:
//   G = P_Omega(clip(L - X, +-lam_S))                       (one pass: reads L, X, writes G)
//   top singular pair (sigma_1, u_1, v_1) of G                (power iteration on G, warm start)
//   V = -B u_1 v_1^T, Vt = B if sigma_1 > lam_L, else V = 0, Vt = 0    (B: the radius bound)
//   eta = clip(-(<G, V - L> + lam_L (Vt - t)) / ||P_Omega(V - L)||^2, 0, 1)  (exact line search
//         of the printed quadratic with S fixed; one pass over L for the denominator)
//   L <- (1 - eta) L + eta V,  t <- (1 - eta) t + eta Vt,  B <- B_0 + t (as printed)
// with the Frank-Wolfe gap <G, L - V> + lam_L (t - Vt) as the stopping test.  Every pass is a
// stream over m x n float32 arrays (HBM-bound); block partial sums are float64 in a fixed order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace rpca {

constexpr int FW_T = 128;          // threads per block; 4 rows per thread
constexpr int FW_ROWS = 4 * FW_T;  // rows per block
constexpr int FW_CCH = 8;          // column chunks of the D v product

RPCA_DEV double fw_block_sum(double v, double* scr) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) scr[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += scr[i];
  return s;
}

RPCA_DEV bool fw_obs(const uint8_t* mask, int64_t ldmask, int64_t i, int64_t j) {
  return mask == nullptr || mask[i + j * ldmask] != 0;
}

// G = P_Omega(clip(L - X)); partials: sum psi(L - X) and <G, L>.  Grid (row blocks, column
// blocks); each thread owns 4 consecutive rows (16-byte accesses; ld multiple of 4).
__global__ void __launch_bounds__(FW_T) fw_resid_kernel(const float* L, int64_t ldl, const float* X, int64_t ldx,
                                                        const uint8_t* mask, int64_t ldmask, int64_t m, int64_t n,
                                                        float lam, float* G, double* part) {
  __shared__ double scr[FW_T / 32];
  double psi = 0.0, gl = 0.0;
  const int64_t i0 = (int64_t)blockIdx.x * FW_ROWS + 4 * threadIdx.x;
  for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
    if (i0 >= m) break;
    float4 l, x;
    if (i0 + 3 < m) {
      l = *reinterpret_cast<const float4*>(L + i0 + j * ldl);
      x = *reinterpret_cast<const float4*>(X + i0 + j * ldx);
    } else {
      float lt[4] = {0, 0, 0, 0}, xt[4] = {0, 0, 0, 0};
      for (int q = 0; q < 4 && i0 + q < m; ++q) {
        lt[q] = L[i0 + q + j * ldl];
        xt[q] = X[i0 + q + j * ldx];
      }
      l = make_float4(lt[0], lt[1], lt[2], lt[3]);
      x = make_float4(xt[0], xt[1], xt[2], xt[3]);
    }
    float lv[4] = {l.x, l.y, l.z, l.w}, xv[4] = {x.x, x.y, x.z, x.w}, gv[4];
    float ps = 0.f, pg = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + q;
      const bool on = i < m && fw_obs(mask, ldmask, i, j);
      const float r = lv[q] - xv[q];
      const float d = on ? fminf(fmaxf(r, -lam), lam) : 0.f;
      gv[q] = d;
      ps += d * (r - 0.5f * d);  // psi(r) = d (r - d / 2) with d = clip(r)
      pg += d * lv[q];
    }
    psi += ps;
    gl += pg;
    if (i0 + 3 < m) {
      *reinterpret_cast<float4*>(G + i0 + j * ldl) = make_float4(gv[0], gv[1], gv[2], gv[3]);
    } else {
      for (int q = 0; q < 4 && i0 + q < m; ++q) G[i0 + q + j * ldl] = gv[q];
    }
  }
  const double a = fw_block_sum(psi, scr);
  const double b = fw_block_sum(gl, scr);
  if (threadIdx.x == 0) {
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    part[2 * blk + 0] = a;
    part[2 * blk + 1] = b;
  }
}

// Ypart[c][i] = sum over the columns of chunk c of G[i][j] v[j].
__global__ void __launch_bounds__(FW_T) fw_gemv_n_kernel(const float* G, int64_t ld, int64_t m, int64_t n,
                                                         const float* v, float* Ypart) {
  const int64_t i0 = (int64_t)blockIdx.x * FW_ROWS + 4 * threadIdx.x;
  if (i0 >= m) return;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t j0 = (int64_t)blockIdx.y * per, j1 = std::min<int64_t>(n, j0 + per);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  if (i0 + 3 < m) {
    for (int64_t j = j0; j < j1; ++j) {
      const float4 g = *reinterpret_cast<const float4*>(G + i0 + j * ld);
      const float vj = __ldg(v + j);
      a0 = fmaf(g.x, vj, a0);
      a1 = fmaf(g.y, vj, a1);
      a2 = fmaf(g.z, vj, a2);
      a3 = fmaf(g.w, vj, a3);
    }
  } else {
    for (int64_t j = j0; j < j1; ++j) {
      const float vj = __ldg(v + j);
      a0 = fmaf(G[i0 + j * ld], vj, a0);
      if (i0 + 1 < m) a1 = fmaf(G[i0 + 1 + j * ld], vj, a1);
      if (i0 + 2 < m) a2 = fmaf(G[i0 + 2 + j * ld], vj, a2);
    }
  }
  float* y = Ypart + (int64_t)blockIdx.y * m;
  y[i0] = a0;
  if (i0 + 1 < m) y[i0 + 1] = a1;
  if (i0 + 2 < m) y[i0 + 2] = a2;
  if (i0 + 3 < m) y[i0 + 3] = a3;
}

// y = sum of the chunks (fixed order); partials of ||y||^2.
__global__ void fw_ysum_kernel(const float* Ypart, int nch, int64_t m, float* y, double* part) {
  __shared__ double scr[32];
  double s2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int c = 0; c < nch; ++c) a += Ypart[(int64_t)c * m + i];
    y[i] = a;
    s2 += (double)a * a;
  }
  const double t = fw_block_sum(s2, scr);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// z[j] = sum_i G[i][j] y[i]: one block per column (grid-stride over columns).
__global__ void __launch_bounds__(256) fw_gemv_t_kernel(const float* G, int64_t ld, int64_t m, int64_t n,
                                                        const float* y, float* z) {
  __shared__ double scr[8];
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    float a = 0.f;
    const float* g = G + j * ld;
    const int64_t m4 = m & ~(int64_t)3;
    for (int64_t i = 4 * (int64_t)threadIdx.x; i < m4; i += 4 * (int64_t)blockDim.x) {
      const float4 gv = *reinterpret_cast<const float4*>(g + i);
      const float4 yv = *reinterpret_cast<const float4*>(y + i);
      a = fmaf(gv.x, yv.x, a);
      a = fmaf(gv.y, yv.y, a);
      a = fmaf(gv.z, yv.z, a);
      a = fmaf(gv.w, yv.w, a);
    }
    for (int64_t i = m4 + threadIdx.x; i < m; i += blockDim.x) a = fmaf(g[i], y[i], a);
    const double s = fw_block_sum((double)a, scr);
    if (threadIdx.x == 0) z[j] = (float)s;
    __syncthreads();
  }
}

// v = z / ||z|| (one block).
__global__ void __launch_bounds__(1024) fw_normalize_kernel(const float* z, int64_t n, float* v) {
  __shared__ double scr[32];
  __shared__ double nrm;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s += (double)z[j] * z[j];
  s = fw_block_sum(s, scr);
  if (threadIdx.x == 0) nrm = s > 0.0 ? sqrt(s) : 1.0;
  __syncthreads();
  const float inv = (float)(1.0 / nrm);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) v[j] = z[j] * inv;
}

// Partials of ||P_Omega(c y v^T - L)||^2 (c = 0: ||P_Omega L||^2).
__global__ void __launch_bounds__(FW_T) fw_quad_kernel(const float* L, int64_t ldl, const uint8_t* mask,
                                                       int64_t ldmask, int64_t m, int64_t n, const float* y,
                                                       const float* v, float c, double* part) {
  __shared__ double scr[FW_T / 32];
  double acc = 0.0;
  const int64_t i0 = (int64_t)blockIdx.x * FW_ROWS + 4 * threadIdx.x;
  float yi[4] = {0, 0, 0, 0};
  for (int q = 0; q < 4; ++q)
    if (i0 + q < m) yi[q] = y[i0 + q];
  for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
    if (i0 >= m) break;
    const float cv = c * __ldg(v + j);
    float s = 0.f;
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + q;
      if (i < m && fw_obs(mask, ldmask, i, j)) {
        const float w = cv * yi[q] - L[i + j * ldl];
        s = fmaf(w, w, s);
      }
    }
    acc += s;
  }
  const double a = fw_block_sum(acc, scr);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = a;
}

// L <- (1 - eta) L + eta c y v^T.
__global__ void __launch_bounds__(FW_T) fw_update_kernel(float* L, int64_t ldl, int64_t m, int64_t n, const float* y,
                                                         const float* v, float c, float eta) {
  const int64_t i0 = (int64_t)blockIdx.x * FW_ROWS + 4 * threadIdx.x;
  if (i0 >= m) return;
  float yi[4] = {0, 0, 0, 0};
  for (int q = 0; q < 4; ++q)
    if (i0 + q < m) yi[q] = y[i0 + q];
  const float a = 1.f - eta;
  for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
    const float b = eta * c * __ldg(v + j);
    if (i0 + 3 < m) {
      float4* p = reinterpret_cast<float4*>(L + i0 + j * ldl);
      float4 l = *p;
      l.x = fmaf(a, l.x, b * yi[0]);
      l.y = fmaf(a, l.y, b * yi[1]);
      l.z = fmaf(a, l.z, b * yi[2]);
      l.w = fmaf(a, l.w, b * yi[3]);
      *p = l;
    } else {
      for (int q = 0; q < 4 && i0 + q < m; ++q) L[i0 + q + j * ldl] = fmaf(a, L[i0 + q + j * ldl], b * yi[q]);
    }
  }
}

__global__ void fw_fill_kernel(float* v, int64_t n, float val) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    v[j] = val;
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_fw_solve(rpca_ctx* c, float* L, int64_t ldl, int max_iter, double gap_tol,
                                     int power_iters, double* log, rpca_fw_result* res) {
  if (!c) return RPCA_EINVAL;
  if (!L || ldl < c->m || (ldl * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(L) & 15) != 0)
    return set_err(c, RPCA_EINVAL, "L must be 16-byte aligned with ldl >= m a multiple of 4");
  if (max_iter < 0 || power_iters < 1 || !(gap_tol >= 0.0))
    return set_err(c, RPCA_EINVAL, "max_iter >= 0, power_iters >= 1, gap_tol >= 0");
  if (c->xq_dt != 0) return set_err(c, RPCA_EUNSUPPORTED, "Frank-Wolfe reads float32 X");
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t m = c->m, n = c->n;
  cudaStream_t st = c->stream;
  const float lam = std::isinf(c->lam_S) ? INFINITY : (float)c->lam_S;
  const double lamL = c->lam_L;
  const int gx = (int)((m + FW_ROWS - 1) / FW_ROWS);
  const int gy = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)std::max(1, 4 * c->nsm / std::max(gx, 1))));
  const int nblk = gx * gy;
  const int ysum_grid = (int)std::min<int64_t>(256, (m + 255) / 256);
  const int gt_grid = (int)std::min<int64_t>(n, 16 * (int64_t)c->nsm);
  // Scratch: G (same layout as L), Ypart (FW_CCH x m), y (m), z (n), v (n), partials.
  float* buf = nullptr;
  double* part = nullptr;
  const size_t nf = (size_t)ldl * n + (size_t)FW_CCH * m + m + 2 * (size_t)n;
  RPCA_CUDA(c, cudaMalloc(&buf, sizeof(float) * nf));
  const size_t np = 2 * (size_t)nblk + 256 + 8;
  if (cudaMalloc(&part, sizeof(double) * np) != cudaSuccess) {
    cudaFree(buf);
    return set_err(c, RPCA_ENOMEM, "cudaMalloc");
  }
  float* G = buf;
  float* Yp = G + (size_t)ldl * n;
  float* y = Yp + (size_t)FW_CCH * m;
  float* z = y + m;
  float* v = z + n;
  std::vector<double> hp(np);
  auto fail = [&](rpca_status s) {
    cudaStreamSynchronize(st);
    cudaFree(buf);
    cudaFree(part);
    return s;
  };
  auto read_parts = [&](size_t count) -> bool {
    if (cudaMemcpyAsync(hp.data(), part, sizeof(double) * count, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return false;
    return cudaStreamSynchronize(st) == cudaSuccess;
  };
  const dim3 g2(gx, gy);
  RPCA_CUDA(c, cudaMemsetAsync(y, 0, sizeof(float) * m, st));
  fw_fill_kernel<<<std::max<int64_t>(1, std::min<int64_t>(256, (n + 255) / 256)), 256, 0, st>>>(
      v, n, (float)(1.0 / std::sqrt((double)n)));
  count_launches(c, 1);
  double t = 0.0, B = 0.0, B0 = 0.0, F = 0.0, gap = INFINITY, eta = 0.0, s1 = 0.0;
  int it = 0;
  for (;; ++it) {
    fw_resid_kernel<<<g2, FW_T, 0, st>>>(L, ldl, c->X, c->ldx, c->mask, c->ldmask, m, n, lam, G, part);
    count_launches(c, 1);
    if (!read_parts(2 * (size_t)nblk)) return fail(cuda_err(c, cudaGetLastError(), "rpca_fw_solve"));
    double psi = 0.0, gl = 0.0;
    for (int b = 0; b < nblk; ++b) {
      psi += hp[2 * b];
      gl += hp[2 * b + 1];
    }
    F = psi + lamL * t;
    if (it == 0) {
      // B_0 = (1 / (2 lam_L)) ||P_Omega(L_0 + S_0 - X)||^2 = ||G_0||^2 / (2 lam_L).
      fw_quad_kernel<<<g2, FW_T, 0, st>>>(G, ldl, nullptr, 0, m, n, y, v, 0.f, part);
      count_launches(c, 1);
      if (!read_parts(nblk)) return fail(cuda_err(c, cudaGetLastError(), "rpca_fw_solve"));
      double gg = 0.0;
      for (int b = 0; b < nblk; ++b) gg += hp[b];
      B0 = 0.5 * gg / lamL;
      B = B0;
    }
    if (it >= max_iter) break;
    // Top singular pair of G: power iterations from the previous v (unit), then y = G v.
    for (int p = 0; p <= power_iters; ++p) {
      fw_gemv_n_kernel<<<dim3(gx, FW_CCH), FW_T, 0, st>>>(G, ldl, m, n, v, Yp);
      fw_ysum_kernel<<<ysum_grid, 256, 0, st>>>(Yp, FW_CCH, m, y, part);
      count_launches(c, 2);
      if (p == power_iters) break;
      fw_gemv_t_kernel<<<gt_grid, 256, 0, st>>>(G, ldl, m, n, y, z);
      fw_normalize_kernel<<<1, 1024, 0, st>>>(z, n, v);
      count_launches(c, 2);
    }
    if (!read_parts(ysum_grid)) return fail(cuda_err(c, cudaGetLastError(), "rpca_fw_solve"));
    double yy = 0.0;
    for (int b = 0; b < ysum_grid; ++b) yy += hp[b];
    s1 = std::sqrt(yy);  // = u^T G v with u = y / ||y||
    // Vertex of the linear subproblem: V = cc y v^T with cc = -B / sigma_1 (= -B u v^T).
    const bool move = s1 > lamL && s1 > 0.0;
    const double Vt = move ? B : 0.0;
    const float cc = move ? (float)(-B / s1) : 0.f;
    const double gv = move ? -B * s1 : 0.0;  // <G, V>
    gap = (gl - gv) + lamL * (t - Vt);
    if (log) {
      log[4 * it + 0] = F;
      log[4 * it + 1] = gap;
      log[4 * it + 2] = s1;
    }
    if (gap <= gap_tol * std::max(1.0, std::fabs(F))) {
      if (log) log[4 * it + 3] = 0.0;
      break;
    }
    fw_quad_kernel<<<g2, FW_T, 0, st>>>(L, ldl, c->mask, c->ldmask, m, n, y, v, cc, part);
    count_launches(c, 1);
    if (!read_parts(nblk)) return fail(cuda_err(c, cudaGetLastError(), "rpca_fw_solve"));
    double ww = 0.0;
    for (int b = 0; b < nblk; ++b) ww += hp[b];
    const double num = -((gv - gl) + lamL * (Vt - t));
    eta = ww > 0.0 ? std::min(std::max(num / ww, 0.0), 1.0) : 0.0;
    if (log) log[4 * it + 3] = eta;
    fw_update_kernel<<<g2, FW_T, 0, st>>>(L, ldl, m, n, y, v, cc, (float)eta);
    count_launches(c, 1);
    const double t_old = t;
    t = (1.0 - eta) * t + eta * Vt;
    B = B0 + t_old;
  }
  const rpca_status s = fail(check_dev_err(c));
  if (res) {
    memset(res, 0, sizeof *res);
    res->F = F;
    res->t = t;
    res->gap = gap;
    res->sigma1 = s1;
    res->iters = it;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return s;
}
