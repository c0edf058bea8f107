// Objective/gradient pass for factor ranks above the fused kernel's (k > 16), e.g. the
// k = 200 synthetic problem of Sec. 5.3.  There the products U V^T, D V and D^T U are dense
// contractions of depth k, so they run as GEMMs on the tensor cores (cuBLAS with float32
// emulated by three bfloat16 terms: float32 accuracy), with the elementwise part in this
// file's kernels:
//   R  = Ut Vt^T - X                      (GEMM onto a copy of X)
//   D  = P_Omega(clip(R, +-lam_S)), psi   (one pass over R: D in place, per-block psi sums)
//   PU = -D Vt,  PV = D^T Ut              (GEMMs into the fused kernel's partial-sum layout)
// and the fused path's finalize kernels complete G_U, G_V, f and the line-search dots, so the
// solver sees the same interface for every k.  (Ut, Vt) is the trial point U + alpha dU,
// V + alpha dV when a direction is given.  R costs m n floats of extra memory.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "ctx.h"
#include "smallla.cuh"

namespace rpca {

struct LargeK {
  cublasHandle_t h = nullptr;
  float* R = nullptr;  // m x n, ld mpad
  float* Ut = nullptr;
  float* Vt = nullptr;
  int nblk = 0;  // blocks of the elementwise pass (= psi partials)
};

constexpr int LK_T = 256;

// Ut = U + alpha dU, Vt = V + alpha dV (alpha from the device when given); skipped when the
// gate is closed.
__global__ void lk_trial_kernel(const float* U, const float* dU, const float* V, const float* dV, int64_t mk,
                                int64_t nk, float alpha, const double* alpha_dev, const int* gate, float* Ut,
                                float* Vt) {
  if (gate != nullptr && *gate == 0) return;
  const float a = alpha_dev ? (float)*alpha_dev : alpha;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < mk + nk; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < mk) Ut[e] = dU ? fmaf(a, dU[e], U[e]) : U[e];
    else Vt[e - mk] = dV ? fmaf(a, dV[e - mk], V[e - mk]) : V[e - mk];
  }
}

// D = P_Omega(clip(R)) in place; per-block sums of psi(R) over Omega (psi(r) = d (r - d / 2)).
__global__ void __launch_bounds__(LK_T) lk_resid_kernel(float* R, int64_t ldr, int64_t m, int64_t n,
                                                        const uint32_t* bits, int wpad, float lam, const int* gate,
                                                        double* psi_part) {
  if (gate != nullptr && *gate == 0) return;
  __shared__ double scr[LK_T / 32];
  float acc_s = 0.f, acc_c = 0.f;  // Kahan pair; float-float across lanes and warps
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    float* p = R + i + j * ldr;
    const float r = *p;
    const bool on = bits == nullptr || ((bits[(size_t)j * wpad + (i >> 5)] >> (i & 31)) & 1u);
    const float d = on ? fminf(fmaxf(r, -lam), lam) : 0.f;
    *p = d;
    const float y = d * (r - 0.5f * d) - acc_c;
    const float t = acc_s + y;
    acc_c = (t - acc_s) - y;
    acc_s = t;
  }
  const ff2 w = warp_ff_sum(ff_from_kahan(acc_s, acc_c));
  if ((threadIdx.x & 31) == 0) ff_store(&scr[threadIdx.x >> 5], w);
  __syncthreads();
  if (threadIdx.x == 0) {
    ff2 s = ff_load(&scr[0]);
    for (int q = 1; q < LK_T / 32; ++q) s = ff_add(s, ff_load(&scr[q]));
    ff_store(&psi_part[blockIdx.x], s);
  }
}

static rpca_status lk_cublas(rpca_ctx* c, cublasStatus_t s, const char* what) {
  if (s == CUBLAS_STATUS_SUCCESS) return RPCA_OK;
  char buf[160];
  snprintf(buf, sizeof buf, "%s failed (cuBLAS status %d)", what, (int)s);
  return set_err(c, RPCA_ECUDA, buf);
}

// C (rows x cols, ldc) = alpha op(A) op(B) + beta C, float32 emulated on the tensor cores.
static cublasStatus_t lk_gemm(LargeK* lk, cublasOperation_t ta, cublasOperation_t tb, int64_t rows, int64_t cols,
                              int64_t depth, float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                              float beta, float* C, int64_t ldc) {
  return cublasGemmEx(lk->h, ta, tb, (int)rows, (int)cols, (int)depth, &alpha, A, CUDA_R_32F, (int)lda, B, CUDA_R_32F,
                      (int)ldb, &beta, C, CUDA_R_32F, (int)ldc, CUBLAS_COMPUTE_32F_EMULATED_16BFX9,
                      CUBLAS_GEMM_DEFAULT);
}

rpca_status lk_setup(rpca_ctx* c) {
  LargeK* lk = new (std::nothrow) LargeK();
  if (!lk) return set_err(c, RPCA_ENOMEM, "host allocation failed");
  c->lk = lk;
  rpca_status s;
  if ((s = lk_cublas(c, cublasCreate(&lk->h), "cublasCreate")) != RPCA_OK) return s;
  if ((s = lk_cublas(c, cublasSetStream(lk->h, c->stream), "cublasSetStream")) != RPCA_OK) return s;
  if ((s = lk_cublas(c, cublasSetMathMode(lk->h, CUBLAS_FP32_EMULATED_BF16X9_MATH), "cublasSetMathMode")) != RPCA_OK)
    return s;
  const int64_t m = c->m, n = c->n, k = c->k;
  RPCA_CUDA(c, cudaMalloc(&lk->R, sizeof(float) * (size_t)c->mpad * n));
  RPCA_CUDA(c, cudaMalloc(&lk->Ut, sizeof(float) * (size_t)(m + n) * k));
  lk->Vt = lk->Ut + m * k;
  lk->nblk = (int)std::min<int64_t>(8 * (int64_t)c->nsm, (m * n + LK_T - 1) / LK_T);
  // The plan: one "row block" and one "column split" for the finalize's partial-sum layout.
  FgPlan& P = c->fg_plan;
  P = FgPlan();
  P.valid = true;
  P.large = true;
  P.K = P.B = (int)k;
  P.same = true;
  P.masked = c->bits != nullptr;
  P.nrb = 1;
  P.ncs = 1;
  P.fin_gu = fin_grid_u(c->m, (int)k);
  P.fin_gv = fin_grid_v(c->n, (int)k);
  P.fin_grid = P.fin_gu + P.fin_gv;
  Workspace& w = c->ws;
  RPCA_CUDA(c, cudaMalloc(&w.PU, sizeof(float) * (size_t)c->mpad * k));
  w.PU_n = (size_t)c->mpad * k;
  RPCA_CUDA(c, cudaMalloc(&w.PV, sizeof(float) * (size_t)n * k));
  w.PV_n = (size_t)n * k;
  RPCA_CUDA(c, cudaMalloc(&w.Ppsi, sizeof(double) * lk->nblk));
  w.Ppsi_n = lk->nblk;
  RPCA_CUDA(c, cudaMalloc(&w.blk, sizeof(double) * 3 * P.fin_grid));
  w.blk_n = 3 * (size_t)P.fin_grid;
  return RPCA_OK;
}

void lk_free(rpca_ctx* c) {
  LargeK* lk = c->lk;
  if (!lk) return;
  if (lk->h) cublasDestroy(lk->h);
  cudaFree(lk->R);
  cudaFree(lk->Ut);
  delete lk;
  c->lk = nullptr;
}

// L = U V^T into the context's m x n buffer (ld mpad); *Lp, *ldl receive it.
rpca_status lk_product(rpca_ctx* c, const float* U, const float* V, const float** Lp, int64_t* ldl) {
  LargeK* lk = c->lk;
  if (!lk) return set_err(c, RPCA_EINVAL, "no large-rank state on this context");
  rpca_status s;
  if ((s = lk_cublas(c, cublasSetStream(lk->h, c->stream), "cublasSetStream")) != RPCA_OK) return s;
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_N, CUBLAS_OP_T, c->m, c->n, c->k, 1.f, U, c->m, V, c->n, 0.f, lk->R,
                                c->mpad),
                     "GEMM U V^T")) != RPCA_OK)
    return s;
  *Lp = lk->R;
  *ldl = c->mpad;
  return RPCA_OK;
}

rpca_status launch_fg_large(rpca_ctx* c, const FgPlan& P, const FgLaunch& L, cudaStream_t stream) {
  LargeK* lk = c->lk;
  if (!lk) return set_err(c, RPCA_EINVAL, "no large-rank state on this context");
  if (L.fin_mode != FIN_FG) return set_err(c, RPCA_EUNSUPPORTED, "k > 16: only the objective/gradient pass");
  const int64_t m = c->m, n = c->n, k = c->k, ldr = c->mpad;
  rpca_status s;
  if ((s = lk_cublas(c, cublasSetStream(lk->h, stream), "cublasSetStream")) != RPCA_OK) return s;
  const float* Ut = L.U;
  const float* Vt = L.V;
  if (L.dU || L.dV) {
    const int grid = (int)std::min<int64_t>(4 * (int64_t)c->nsm, ((m + n) * k + 255) / 256);
    lk_trial_kernel<<<grid, 256, 0, stream>>>(L.U, L.dU, L.V, L.dV, m * k, n * k, L.alpha, L.alpha_dev, L.gate,
                                              lk->Ut, lk->Vt);
    count_launches(c, 1);
    Ut = lk->Ut;
    Vt = lk->Vt;
  }
  // R = Ut Vt^T - X.
  RPCA_CUDA(c, cudaMemcpy2DAsync(lk->R, ldr * sizeof(float), c->X, c->ldx * sizeof(float), m * sizeof(float), n,
                                 cudaMemcpyDeviceToDevice, stream));
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_N, CUBLAS_OP_T, m, n, k, 1.f, Ut, m, Vt, n, -1.f, lk->R, ldr),
                     "GEMM U V^T")) != RPCA_OK)
    return s;
  const float lam = std::isinf(c->lam_S) ? INFINITY : (float)c->lam_S;
  lk_resid_kernel<<<lk->nblk, LK_T, 0, stream>>>(lk->R, ldr, m, n, c->bits, c->wpad, lam, L.gate, c->ws.Ppsi);
  count_launches(c, 1);
  // PU = -D Vt (m x k, ld mpad), PV = D^T Ut (n x k, ld n).
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_N, CUBLAS_OP_N, m, k, n, -1.f, lk->R, ldr, Vt, n, 0.f, c->ws.PU, ldr),
                     "GEMM D V")) != RPCA_OK)
    return s;
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_T, CUBLAS_OP_N, n, k, m, 1.f, lk->R, ldr, Ut, m, 0.f, c->ws.PV, n),
                     "GEMM D^T U")) != RPCA_OK)
    return s;
  FinArgs f;
  memset(&f, 0, sizeof f);
  f.m = c->m;
  f.n = c->n;
  f.B = (int)k;
  f.mpad = c->mpad;
  f.nrb = 1;
  f.ncs = 1;
  f.nctas = lk->nblk;
  f.gu = P.fin_gu;
  f.PU = c->ws.PU;
  f.PV = c->ws.PV;
  f.Ppsi = c->ws.Ppsi;
  f.mode = FIN_FG;
  f.side = 0;
  f.U = L.U;
  f.V = L.V;
  f.dU = L.dU;
  f.dV = L.dV;
  f.alpha = L.alpha;
  f.alpha_dev = L.alpha_dev;
  f.gate = L.gate;
  f.lam_L = c->lam_L;
  f.lam_f = (float)c->lam_L;
  f.GU = L.GU;
  f.GV = L.GV;
  f.Ut = L.Ut;
  f.Vt = L.Vt;
  f.DU = L.DU;
  f.DV = L.DV;
  f.blk = c->ws.blk;
  f.counter = c->ws.counter;
  f.out = L.out ? L.out : c->ws.out;
  f.vec4 = fin_vec4(f);
  finalize_kernel<<<P.fin_grid, 256, 0, stream>>>(f);
  finalize_reduce_kernel<<<1, 256, 0, stream>>>(f, P.fin_grid);
  count_launches(c, 2);
  RPCA_CUDA(c, cudaGetLastError());
  return RPCA_OK;
}

// ---- randomized SVD for large sketches (l = k + p > 32) --------------------------------------
void fill_normal(float* out, int64_t count, uint64_t seed, float scale, cudaStream_t s);  // solve.cu

constexpr int LKS_LMAX = 224;  // float32 l x l Cholesky in shared memory (<= 196 KB)

// A*(X) = P_Omega(X) / p_hat into R (m x n, ld ldr).
__global__ void lk_sample_kernel(const float* X, int64_t ldx, const uint32_t* bits, int wpad, int64_t m, int64_t n,
                                 float inv_p, float* R, int64_t ldr) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    const bool on = bits == nullptr || ((bits[(size_t)j * wpad + (i >> 5)] >> (i & 31)) & 1u);
    R[i + j * ldr] = on ? X[i + j * ldx] * inv_p : 0.f;
  }
}

// G (l x l, symmetric, column-major) -> R^{-1} (upper triangular, zeros below) of the Cholesky
// factor of G + shift I, shift = 1e-6 max diag (float32, one CTA, in shared memory).  A pivot
// that falls below 1e-6 of the largest diagonal marks its column as collapsed: its column
// of R^{-1} is zero (the corresponding column of Y R^{-1} vanishes).
__global__ void __launch_bounds__(1024) lk_chol_inv_kernel(float* G, int l) {
  extern __shared__ float A[];  // l x l, column-major
  __shared__ float col[LKS_LMAX];
  __shared__ float dmax;
  __shared__ int dead[LKS_LMAX];
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < l * l; e += nt) A[e] = G[e];
  __syncthreads();
  if (t == 0) {
    float d = 0.f;
    for (int i = 0; i < l; ++i) d = fmaxf(d, A[i + i * l]);
    dmax = fmaxf(d, 1e-30f);
  }
  __syncthreads();
  const float shift = 1e-6f * dmax;
  for (int i = t; i < l; i += nt) A[i + i * l] += shift;
  __syncthreads();
  // Upper Cholesky A = R^T R in place (R in the upper triangle), right-looking.
  for (int j = 0; j < l; ++j) {
    if (t == 0) {
      const float p = A[j + j * l];
      dead[j] = !(p > 1e-6f * dmax);
      A[j + j * l] = dead[j] ? 1.f : sqrtf(p);
    }
    __syncthreads();
    const float r = A[j + j * l];
    for (int c = j + 1 + t; c < l; c += nt) A[j + c * l] = dead[j] ? 0.f : A[j + c * l] / r;
    __syncthreads();
    // Trailing update A[a][c] -= R[j][a] R[j][c] for j < a <= c.
    const int w = l - j - 1;
    for (int e = t; e < w * w; e += nt) {
      const int a = j + 1 + e % w, c = j + 1 + e / w;
      if (a <= c) A[a + c * l] -= A[j + a * l] * A[j + c * l];
    }
    __syncthreads();
  }
  // In-place inverse of the upper triangular R, column by column.
  for (int j = 0; j < l; ++j) {
    for (int i = t; i <= j; i += nt) col[i] = A[i + j * l];
    __syncthreads();
    const float rjj = 1.f / col[j];
    for (int i = t; i < j; i += nt) {
      float s = 0.f;
      for (int q = i; q < j; ++q) s = fmaf(A[i + q * l], col[q], s);  // (R^{-1})[i][q] R[q][j]
      A[i + j * l] = -s * rjj;
    }
    if (t == 0) A[j + j * l] = rjj;
    __syncthreads();
  }
  for (int e = t; e < l * l; e += nt) {
    const int a = e % l, c = e / l;
    G[e] = (a > c || dead[c] || dead[a]) ? 0.f : A[e];
  }
}

// Eigen-decomposition of the Gram B B^T (l x l, in global memory) by one-sided Jacobi (float32),
// then C1 = W[:, :k] Sigma^{1/2}, C2 = W[:, :k] Sigma^{-1/2} (l x k), Sigma = sqrt(eigenvalues),
// descending.
__global__ void __launch_bounds__(1024) lk_eig_kernel(float* A, float* W, int l, int k, float* C1, float* C2) {
  __shared__ float ev[LKS_LMAX];
  __shared__ int ord[LKS_LMAX];
  __shared__ int flag;
  cta_jacobi_svd<float>(A, l, l, l, W, l, ev, &flag, 30, 1e-6f, 2.0f * l * 6e-8f);
  cta_sort_desc<float>(ev, l, ord);
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) {
    const int a = e % l, c = e / l;
    const float lam = ev[ord[c]];
    const float sg = lam > 0.f ? sqrtf(lam) : 0.f;
    const float u = W[a + ord[c] * l];
    C1[e] = u * sqrtf(sg);
    C2[e] = sg > 0.f ? u / sqrtf(sg) : 0.f;
  }
}

rpca_status sketch_init_large(rpca_ctx* c, const float* Omega, float* U, float* V) {
  LargeK* lk = c->lk;
  if (!lk) return set_err(c, RPCA_EINVAL, "no large-rank state on this context");
  const int64_t m = c->m, n = c->n, k = c->k;
  const int l = (int)std::min<int64_t>(std::min<int64_t>(k + std::max(0, c->opt.sketch_oversample), LKS_LMAX),
                                       std::min(m, n));
  if (l < k) return set_err(c, RPCA_EUNSUPPORTED, "the large sketch holds at most 224 columns");
  const int q = std::max(0, c->opt.sketch_power);
  cudaStream_t st = c->stream;
  rpca_status s;
  if ((s = lk_cublas(c, cublasSetStream(lk->h, st), "cublasSetStream")) != RPCA_OK) return s;
  // A*(X): X itself when fully observed, else the rescaled observed entries (in R).
  const float* Xs = c->X;
  int64_t ldxs = c->ldx;
  if (c->bits) {
    lk_sample_kernel<<<4 * c->nsm, 256, 0, st>>>(c->X, c->ldx, c->bits, c->wpad, m, n,
                                                 (float)(1.0 / std::max(c->p_hat, 1e-30)), lk->R, c->mpad);
    count_launches(c, 1);
    Xs = lk->R;
    ldxs = c->mpad;
  }
  float* buf = nullptr;
  const size_t nf = (size_t)n * l + (size_t)m * l + (size_t)n * l + (size_t)l * l * 2 + (size_t)2 * l * k;
  RPCA_CUDA(c, cudaMalloc(&buf, sizeof(float) * nf));
  float* Om = buf;
  float* Y = Om + (size_t)n * l;   // m x l
  float* Z = Y + (size_t)m * l;    // n x l
  float* G = Z + (size_t)n * l;    // l x l
  float* Gi = G + (size_t)l * l;   // l x l (W of the eigen-decomposition)
  float* C1 = Gi + (size_t)l * l;  // l x k
  float* C2 = C1 + (size_t)l * k;  // l x k
  auto done = [&](rpca_status r) {
    cudaStreamSynchronize(st);
    cudaFree(buf);
    return r;
  };
  const size_t chol_smem = sizeof(float) * (size_t)l * l;
  if (!allow_smem((const void*)lk_chol_inv_kernel, chol_smem))
    return done(set_err(c, RPCA_EUNSUPPORTED, "shared memory for the sketch's Cholesky"));
  if (Omega) {
    RPCA_CUDA(c, cudaMemcpyAsync(Om, Omega, sizeof(float) * n * l, cudaMemcpyDeviceToDevice, st));
  } else {
    fill_normal(Om, n * l, 0xC0FFEEULL ^ (c->opt.seed * 0x9E3779B97F4A7C15ULL), 1.f, st);
    count_launches(c, 1);
  }
  // Orthonormalise the columns of A (rows x l): two passes of shifted CholeskyQR, the product
  // A R^{-1} going through a scratch buffer of the larger height.
  float* scratch = nullptr;
  RPCA_CUDA(c, cudaMalloc(&scratch, sizeof(float) * (size_t)std::max(m, n) * l));
  auto orth2 = [&](float* A, int64_t rows) -> rpca_status {
    for (int pass = 0; pass < 2; ++pass) {
      rpca_status r;
      if ((r = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_T, CUBLAS_OP_N, l, l, rows, 1.f, A, rows, A, rows, 0.f, G, l),
                         "GEMM sketch Gram")) != RPCA_OK)
        return r;
      lk_chol_inv_kernel<<<1, 1024, chol_smem, st>>>(G, l);
      count_launches(c, 1);
      if ((r = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_N, CUBLAS_OP_N, rows, l, l, 1.f, A, rows, G, l, 0.f, scratch,
                                    rows),
                         "GEMM sketch orth")) != RPCA_OK)
        return r;
      RPCA_CUDA(c, cudaMemcpyAsync(A, scratch, sizeof(float) * rows * l, cudaMemcpyDeviceToDevice, st));
    }
    return RPCA_OK;
  };
  auto fin = [&](rpca_status r) {
    cudaStreamSynchronize(st);
    cudaFree(scratch);
    return done(r);
  };
  // Y = A*(X) Omega, orthonormalised; q power iterations through A*(X)^T and A*(X).
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_N, CUBLAS_OP_N, m, l, n, 1.f, Xs, ldxs, Om, n, 0.f, Y, m),
                     "GEMM X Omega")) != RPCA_OK)
    return fin(s);
  if ((s = orth2(Y, m)) != RPCA_OK) return fin(s);
  for (int it = 0; it < q; ++it) {
    if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_T, CUBLAS_OP_N, n, l, m, 1.f, Xs, ldxs, Y, m, 0.f, Z, n),
                       "GEMM X^T Q")) != RPCA_OK)
      return fin(s);
    if ((s = orth2(Z, n)) != RPCA_OK) return fin(s);
    if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_N, CUBLAS_OP_N, m, l, n, 1.f, Xs, ldxs, Z, n, 0.f, Y, m),
                       "GEMM X Z")) != RPCA_OK)
      return fin(s);
    if ((s = orth2(Y, m)) != RPCA_OK) return fin(s);
  }
  // B^T = A*(X)^T Q (n x l); Gram B B^T = (B^T)^T B^T (l x l); its eigen-decomposition.
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_T, CUBLAS_OP_N, n, l, m, 1.f, Xs, ldxs, Y, m, 0.f, Z, n),
                     "GEMM X^T Q")) != RPCA_OK)
    return fin(s);
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_T, CUBLAS_OP_N, l, l, n, 1.f, Z, n, Z, n, 0.f, G, l), "GEMM B B^T")) !=
      RPCA_OK)
    return fin(s);
  lk_eig_kernel<<<1, 1024, 0, st>>>(G, Gi, l, (int)k, C1, C2);
  count_launches(c, 1);
  // U0 = Q W Sigma^{1/2}, V0 = B^T W Sigma^{-1/2}.
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_N, CUBLAS_OP_N, m, k, l, 1.f, Y, m, C1, l, 0.f, U, m), "GEMM U0")) !=
      RPCA_OK)
    return fin(s);
  if ((s = lk_cublas(c, lk_gemm(lk, CUBLAS_OP_N, CUBLAS_OP_N, n, k, l, 1.f, Z, n, C2, l, 0.f, V, n), "GEMM V0")) !=
      RPCA_OK)
    return fin(s);
  RPCA_CUDA(c, cudaGetLastError());
  return fin(check_dev_err(c));
}

}  // namespace rpca
