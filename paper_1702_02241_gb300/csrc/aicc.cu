// Corrected Akaike information criterion of a solution (Sec. 5.2), as the paper defines it
// for SPCP: with S = shrink(X - L, lam_S) on the observed set and Z = L + S - X,
//   sigma^2 = ||X||^2 / N, b = ||S||_1 / N, b_* = ||L||_* / rank(L)            (N observed)
//   ell = -(N/2) log(2 pi sigma^2) - ||Z||^2 / (2 sigma^2) - N log(2 b) - ||S||_1 / (2 b)
//         - rank(L) log(2 b_*) - ||L||_* / (2 b_*)
//   p   = r (m + n - r) + nnz(S) + (||Z||^2 / ||X||^2) N,   AIC_c = 2 (p - ell) + 2 p (p+1) / (N - p - 1).
// One pass over X forms the sums (L = U V^T entry by entry, or from the GEMM buffer for large
// ranks); the singular values of L come from the k x k Grams (sigma^2 = eig(R_U V^T V R_U^T),
// U^T U = R_U^T R_U by eigen-decomposition), float64, one CTA.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "smallla.cuh"

namespace rpca {

constexpr int AI_T = 256;
constexpr int AI_KMAX = 256;

// Per-block sums: ||Z||^2, ||S||_1, ||X||^2, nnz(S), observed count (float64).
__global__ void __launch_bounds__(AI_T) aicc_elem_kernel(const float* X, int64_t ldx, const uint32_t* bits, int wpad,
                                                         int64_t m, int64_t n, const float* U, const float* V, int k,
                                                         const float* Lbuf, int64_t ldl, float lam, double* part) {
  __shared__ double scr[5][AI_T / 32];
  double acc[5] = {0, 0, 0, 0, 0};
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    const bool on = bits == nullptr || ((bits[(size_t)j * wpad + (i >> 5)] >> (i & 31)) & 1u);
    if (!on) continue;
    float l = 0.f;
    if (Lbuf) {
      l = Lbuf[i + j * ldl];
    } else {
      for (int q = 0; q < k; ++q) l = fmaf(U[i + q * m], V[j + q * n], l);
    }
    const float x = X[i + j * ldx];
    const float r = l - x;
    const float s = fmaxf(fabsf(r) - lam, 0.f);  // |S_ij|
    const float z = fminf(fmaxf(r, -lam), lam);   // Z_ij = L + S - X
    acc[0] += (double)z * z;
    acc[1] += s;
    acc[2] += (double)x * x;
    acc[3] += s > 0.f ? 1.0 : 0.0;
    acc[4] += 1.0;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = 0; q < 5; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) scr[q][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0.0;
    for (int i = 0; i < AI_T / 32; ++i) v += scr[threadIdx.x][i];
    part[(size_t)blockIdx.x * 5 + threadIdx.x] = v;
  }
}

// G = A^T A (k x k, float64) for A rows x k (column-major): one warp per entry.
__global__ void aicc_gram_kernel(const float* A, int64_t rows, int k, double* G) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = wid; e < (int64_t)k * k; e += nw) {
    const int a = (int)(e % k), b = (int)(e / k);
    if (a > b) continue;
    double s = 0.0;
    for (int64_t i = lane; i < rows; i += 32) s += (double)A[i + a * rows] * (double)A[i + b * rows];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      G[a + b * k] = s;
      G[b + a * k] = s;
    }
  }
}

// Singular values of L = U V^T (descending) from AU = U^T U and AV = V^T V; W, T: k x k
// scratch (float64, global).  One CTA.
__global__ void __launch_bounds__(1024) aicc_spectrum_kernel(double* AU, const double* AV, int k, double* W,
                                                             double* T, double* sig) {
  __shared__ double ev[AI_KMAX];
  __shared__ int ord[AI_KMAX];
  __shared__ int flag;
  cta_jacobi_svd<double>(AU, k, k, k, W, k, ev, &flag, 60, 1e-13, 4.0 * k * 1.1e-16);
  double emax = 0.0;
  for (int i = 0; i < k; ++i) emax = fmax(emax, ev[i]);
  // R_U = diag(sqrt(ev)) W^T (rows with negligible eigenvalues dropped): store R_U^T in AU.
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e % k, c = e / k;  // R_U[c][a] = sqrt(ev_c) W[a][c]
    AU[a + c * k] = ev[c] > 1e-14 * emax ? sqrt(ev[c]) * W[a + c * k] : 0.0;
  }
  __syncthreads();
  // T = AV R_U^T (k x k), then M = R_U T stored in W (symmetric PSD).
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e % k, c = e / k;
    double s = 0.0;
    for (int q = 0; q < k; ++q) s += AV[a + q * k] * AU[q + c * k];
    T[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e % k, c = e / k;
    double s = 0.0;
    for (int q = 0; q < k; ++q) s += AU[q + a * k] * T[q + c * k];
    W[e] = s;
  }
  __syncthreads();
  cta_jacobi_svd<double>(W, k, k, k, T, k, ev, &flag, 60, 1e-13, 4.0 * k * 1.1e-16);
  cta_sort_desc<double>(ev, k, ord);
  for (int i = threadIdx.x; i < k; i += blockDim.x) sig[i] = sqrt(fmax(ev[ord[i]], 0.0));
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_aicc(rpca_ctx* c, const float* U, const float* V, rpca_aicc_result* out) {
  if (!c) return RPCA_EINVAL;
  if (!U || !V || !out) return set_err(c, RPCA_EINVAL, "U, V and out are required");
  if (c->xq_dt != 0) return set_err(c, RPCA_EUNSUPPORTED, "AIC_c reads float32 X");
  const int64_t m = c->m, n = c->n;
  const int k = c->k;
  cudaStream_t st = c->stream;
  const float* Lbuf = nullptr;
  int64_t ldl = 0;
  if (c->lk) {  // large ranks: L = U V^T by GEMM into the context's m x n buffer
    rpca_status s = lk_product(c, U, V, &Lbuf, &ldl);
    if (s != RPCA_OK) return s;
  }
  const int nblk = (int)std::min<int64_t>(8 * (int64_t)c->nsm, (m * n + AI_T - 1) / AI_T);
  double* dbuf = nullptr;
  const size_t nd = (size_t)nblk * 5 + 4 * (size_t)k * k + k;
  RPCA_CUDA(c, cudaMalloc(&dbuf, sizeof(double) * nd));
  double* part = dbuf;
  double* AU = part + (size_t)nblk * 5;
  double* AV = AU + (size_t)k * k;
  double* W = AV + (size_t)k * k;
  double* T = W + (size_t)k * k;
  double* sig = T + (size_t)k * k;
  auto done = [&](rpca_status s) {
    cudaStreamSynchronize(st);
    cudaFree(dbuf);
    return s;
  };
  const float lam = std::isinf(c->lam_S) ? INFINITY : (float)c->lam_S;
  aicc_elem_kernel<<<nblk, AI_T, 0, st>>>(c->X, c->ldx, c->bits, c->wpad, m, n, U, V, k, Lbuf, ldl, lam, part);
  const int gg = (int)std::min<int64_t>(4 * (int64_t)c->nsm, ((int64_t)k * k * 32 + 255) / 256);
  aicc_gram_kernel<<<gg, 256, 0, st>>>(U, m, k, AU);
  aicc_gram_kernel<<<gg, 256, 0, st>>>(V, n, k, AV);
  aicc_spectrum_kernel<<<1, 1024, 0, st>>>(AU, AV, k, W, T, sig);
  count_launches(c, 4);
  RPCA_CUDA(c, cudaGetLastError());
  std::vector<double> hp((size_t)nblk * 5), hs(k);
  RPCA_CUDA(c, cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
  RPCA_CUDA(c, cudaMemcpyAsync(hs.data(), sig, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  RPCA_CUDA(c, cudaStreamSynchronize(st));
  double q[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblk; ++b)
    for (int i = 0; i < 5; ++i) q[i] += hp[(size_t)b * 5 + i];
  const double resid2 = q[0], s_l1 = q[1], x2 = q[2], nnz = q[3], N = q[4];
  int r = 0;
  double nuc = 0.0;
  for (int i = 0; i < k; ++i)
    if (hs[0] > 0.0 && hs[i] > 1e-6 * hs[0]) {
      ++r;
      nuc += hs[i];
    }
  const double sigma2 = x2 / N, b = s_l1 / N;
  double ell = -(N / 2.0) * std::log(2.0 * M_PI * sigma2) - resid2 / (2.0 * sigma2);
  if (b > 0.0) ell += -N * std::log(2.0 * b) - s_l1 / (2.0 * b);
  if (r > 0) {
    const double bs = nuc / r;
    ell += -r * std::log(2.0 * bs) - nuc / (2.0 * bs);
  }
  const double p = (double)r * (double)(m + n - r) + nnz + (resid2 / x2) * N;
  memset(out, 0, sizeof *out);
  out->aicc = 2.0 * (p - ell) + 2.0 * p * (p + 1.0) / (N - p - 1.0);
  out->loglik = ell;
  out->dof = p;
  out->rank = r;
  out->nuclear = nuc;
  out->s_l1 = s_l1;
  out->nnz_s = (int64_t)nnz;
  out->resid2 = resid2;
  out->x2 = x2;
  out->count = (int64_t)N;
  return done(check_dev_err(c));
}
