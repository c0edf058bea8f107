// Randomized-SVD initialisation (Sec. 4.2): U0 = U_k Sigma^1/2, V0 = V_k Sigma^1/2 from the
// SVD of A*(X) (observed entries, rescaled by 1/p_hat when a mask is present), computed with
// a rank-(k + p) sketch and q power iterations (Halko, Martinsson & Tropp; p = 10, q = 2 by
// default).  Products with A*(X) and its transpose are passes of the fused kernel in apply
// mode with no forming factors and no clipping (then D = -A*(X)); orthonormalisation is
// CholeskyQR2 with float64 Grams; the small SVD is a float32 one-sided Jacobi on the Gram of
// B^T = A*(X)^T Q.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "ctx.h"
#include "smallla.cuh"
#include "tsla_ctx.h"

namespace rpca {

constexpr int SK_LMAX = 32;
constexpr int SK_CHUNK = 8;  // columns per product pass (the chunk buffers' width)

struct SketchState {
  double G[SK_LMAX * SK_LMAX];
  double R[SK_LMAX * SK_LMAX], Rinv[SK_LMAX * SK_LMAX];
  double C1[SK_LMAX * SK_LMAX], C2[SK_LMAX * SK_LMAX];
  int bad;
};

void fill_normal(float* out, int64_t count, uint64_t seed, float scale, cudaStream_t s);

// Factors the l x l Gram st->G (summed over the row blocks by ts_gram's multi-block reduction:
// float64 runs at a few operations per clock per SM on this GPU, so one CTA summing every
// block's partials was the larger part of this step); collapsed columns (the sketch of a matrix
// of rank < l) are flagged and left uncoupled.
constexpr int SK_CHOL_THREADS = 256;
__global__ void __launch_bounds__(SK_CHOL_THREADS) sk_gram_chol_kernel(SketchState* st, int l) {
  __shared__ double G[SK_LMAX * SK_LMAX], W[SK_LMAX * SK_LMAX], R[SK_LMAX * SK_LMAX], Ri[SK_LMAX * SK_LMAX];
  __shared__ double rd[SK_LMAX];
  __shared__ int bad;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) G[e] = st->G[e];
  __syncthreads();
  const int mask = cta_chol_masked(G, l, 1e-10, nullptr, W, R, Ri, rd, &bad);
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    st->G[e] = G[e];
    st->R[e] = R[e];
    st->Rinv[e] = Ri[e];
  }
  if (threadIdx.x == 0) st->bad = mask;
}

// Zero the flagged columns of Y (rows x l).
__global__ void sk_zero_cols_kernel(float* Y, int64_t rows, int l, const SketchState* st) {
  const int mask = st->bad;
  if (mask == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * l; i += (int64_t)gridDim.x * blockDim.x)
    if ((mask >> (int)(i / rows)) & 1) Y[i] = 0.f;
}

// Right singular vectors and singular values of Z = D^T Q (n x l, the Gram st->G = Z^T Z);
// C1 = U_B[:, :k] Sigma^{1/2} and C2 = U_B[:, :k] Sigma^{-1/2}, both l x k (ld l).  The Gram is
// factored in float64 (G = R^T R, masked Cholesky: a collapsed column gives a zero row of R),
// and R, whose singular values are Z's (not their squares), goes through a float32 one-sided
// Jacobi on one warp: float64 Jacobi sweeps on this GPU's narrow float64 pipe took ten times as
// long, and the start needs no more than float32 singular vectors.
__global__ void __launch_bounds__(256) sk_small_svd_kernel(SketchState* st, int l, int k, float* sig_out,
                                                            float inv_p) {
  __shared__ double G[SK_LMAX * SK_LMAX], Wd[SK_LMAX * SK_LMAX], R[SK_LMAX * SK_LMAX], Ri[SK_LMAX * SK_LMAX];
  __shared__ double rd[SK_LMAX], ev[SK_LMAX];
  __shared__ float A[SK_LMAX * SK_LMAX], W[SK_LMAX * SK_LMAX], evf[SK_LMAX];
  __shared__ int ord[SK_LMAX];
  __shared__ int bad;
  for (int i = threadIdx.x; i < l * l; i += blockDim.x) G[i] = st->G[i];
  __syncthreads();
  const int mask = cta_chol_masked(G, l, 1e-12, nullptr, Wd, R, Ri, rd, &bad);
  for (int i = threadIdx.x; i < l * l; i += blockDim.x) {
    const int row = i % l;
    A[i] = ((mask >> row) & 1) ? 0.f : (float)R[i];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const float tol = fmaxf(1e-6f, 4.0f * l * 1.2e-7f), noise = 2.0f * l * 6e-8f;
    if (l <= 16) warp_jacobi_svd<float, 16, 16>(A, l, l, l, W, l, evf, 40, tol, noise);
    else warp_jacobi_svd<float, SK_LMAX, SK_LMAX>(A, l, l, l, W, l, evf, 40, tol, noise);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < l; i += blockDim.x) ev[i] = (double)evf[i] * (double)evf[i];  // sigma^2
  __syncthreads();
  cta_sort_desc<double>(ev, l, ord);
  for (int i = threadIdx.x; i < l * k; i += blockDim.x) {
    const int a = i % l, c = i / l;
    const double lam = ev[ord[c]];                 // sigma_c^2
    const double sg = lam > 0.0 ? sqrt(lam) : 0.0;  // sigma_c
    const double u = W[a + ord[c] * l];
    st->C1[a + c * l] = u * sqrt(sg);
    st->C2[a + c * l] = sg > 0.0 ? u / sqrt(sg) : 0.0;
  }
  // The sketch's singular values of A*(X), descending (the Gram's eigenvalues carry p_hat^2).
  for (int c = threadIdx.x; c < l; c += blockDim.x) {
    const double lam = ev[ord[c]];
    sig_out[c] = (float)((lam > 0.0 ? sqrt(lam) : 0.0) * inv_p);
  }
}

struct SketchBuffers {
  float* buf = nullptr;
  int l = 0;   // sketch width the buffers were made for
  int lp = 0;  // columns of Om, Y, Z: l rounded up to the products' chunk width
  int lw = 0;  // the current call's l rounded up to its chunk width (<= lp)
  float *Om, *Y, *Z, *BVc, *BUc, *Y1c, *Y2c;
  SketchState* st = nullptr;
  TsScratch ts;
};

static void free_sketch_buffers(SketchBuffers& b) {
  dev_free(b.buf);
  dev_free(b.st);
  dev_free(b.ts.part);
  b.buf = nullptr;
  b.st = nullptr;
  b.ts.part = nullptr;
  b.l = 0;
  b.lp = 0;
}

void sk_free(rpca_ctx* c) {
  if (!c->sk) return;
  cudaStreamSynchronize(c->stream);
  free_sketch_buffers(*c->sk);
  delete c->sk;
  c->sk = nullptr;
}

// The context's sketch scratch for width l (made on first use, kept until rpca_destroy).
static rpca_status ensure_sketch(rpca_ctx* c, int l, SketchBuffers** out) {
  if (!c->sk) c->sk = new SketchBuffers();
  SketchBuffers& b = *c->sk;
  const int64_t m = c->m, n = c->n;
  const int lp = (l + SK_CHUNK - 1) / SK_CHUNK * SK_CHUNK;
  if (b.buf == nullptr || b.l < l || b.lp < lp) {
    if (b.buf) {
      cudaStreamSynchronize(c->stream);
      free_sketch_buffers(b);
    }
    const int64_t nf = (n + m + n) * (int64_t)lp + (n + m + m + n) * (int64_t)SK_CHUNK;
    if (dev_alloc(&b.buf, sizeof(float) * nf) != cudaSuccess) {
      b.buf = nullptr;
      return set_err(c, RPCA_ENOMEM, "cudaMalloc");
    }
    if (dev_alloc(&b.st, sizeof(SketchState)) != cudaSuccess) {
      b.st = nullptr;
      free_sketch_buffers(b);
      return set_err(c, RPCA_ENOMEM, "cudaMalloc");
    }
    b.ts.grid = 2 * c->nsm;
    b.ts.part_n = (size_t)b.ts.grid * 2304;
    if (dev_alloc(&b.ts.part, sizeof(double) * b.ts.part_n) != cudaSuccess) {
      b.ts.part = nullptr;
      free_sketch_buffers(b);
      return set_err(c, RPCA_ENOMEM, "cudaMalloc");
    }
    b.l = l;
    b.lp = lp;
  }
  b.lw = lp;
  b.Om = b.buf;
  b.Y = b.Om + n * b.lp;
  b.Z = b.Y + m * b.lp;
  b.BVc = b.Z + n * b.lp;
  b.BUc = b.BVc + n * SK_CHUNK;
  b.Y1c = b.BUc + m * SK_CHUNK;
  b.Y2c = b.Y1c + m * SK_CHUNK;
  *out = &b;
  return RPCA_OK;
}

#define SK_CUDA(call)                                     \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(c, e_, #call); \
  } while (0)

// Y1 (m x l) = -A*(X) BV (BV n x l),  or  Y2 (n x l) = -A*(X)^T BU (BU m x l), in chunks of
// 16 columns while at least 16 remain (one pass of the 16-column apply kernel, where it has a
// launch configuration), then of 8 (the 8-column kernel), each one pass over X with no forming
// factors.  A full chunk writes its columns of Y in place; a ragged last chunk (l not a
// multiple of 8) goes through a zero-padded copy.
static rpca_status sk_apply(rpca_ctx* c, SketchBuffers& b, int l, const float* BV, const float* BU, float* Y1,
                            float* Y2) {
  const int side = BV ? 1 : 2;
  const FgPlan* P8 = apply_plan(c, 0, side);
  if (!P8) return RPCA_EUNSUPPORTED;
  const FgPlan* P16 = l >= 16 ? apply_plan16(c, side) : nullptr;
  const int64_t m = c->m, n = c->n;
  for (int c0 = 0; c0 < l;) {
    const bool wide = P16 != nullptr && l - c0 >= 16;
    const FgPlan* P = wide ? P16 : P8;
    const int W = wide ? 16 : SK_CHUNK;
    const int w = std::min(W, l - c0);
    const float* bv = BV ? BV + n * c0 : b.BVc;
    const float* bu = BU ? BU + m * c0 : b.BUc;
    if (w < W) {  // ragged last chunk: zero-padded copy
      if (BV) {
        SK_CUDA(cudaMemsetAsync(b.BVc, 0, sizeof(float) * n * W, c->stream));
        SK_CUDA(cudaMemcpyAsync(b.BVc, bv, sizeof(float) * n * w, cudaMemcpyDeviceToDevice, c->stream));
        bv = b.BVc;
      } else {
        SK_CUDA(cudaMemsetAsync(b.BUc, 0, sizeof(float) * m * W, c->stream));
        SK_CUDA(cudaMemcpyAsync(b.BUc, bu, sizeof(float) * m * w, cudaMemcpyDeviceToDevice, c->stream));
        bu = b.BUc;
      }
    }
    const bool direct = w == W;  // the product's W columns go straight to Y
    FgLaunch L;
    L.U = b.BUc;  // not read: no forming factors
    L.V = b.BVc;
    L.BU = bu;
    L.BV = bv;
    L.fin_mode = FIN_APPLY;
    L.GU = (direct && Y1) ? Y1 + m * c0 : b.Y1c;
    L.GV = (direct && Y2) ? Y2 + n * c0 : b.Y2c;
    L.lam = INFINITY;
    rpca_status s = launch_fg(c, *P, L, c->stream);
    if (s != RPCA_OK) return s;
    if (!direct && Y1) SK_CUDA(cudaMemcpyAsync(Y1 + m * c0, b.Y1c, sizeof(float) * m * w, cudaMemcpyDeviceToDevice, c->stream));
    if (!direct && Y2) SK_CUDA(cudaMemcpyAsync(Y2 + n * c0, b.Y2c, sizeof(float) * n * w, cudaMemcpyDeviceToDevice, c->stream));
    c0 += W;
  }
  return RPCA_OK;
}

// CholeskyQR2; columns that collapse in the first pass are zeroed (rank of the sketch < l).
// The first pass's masked factor leaves a collapsed column uncoupled (its column of R^-1 is the
// unit vector), so Y R^-1 keeps it as it was and zeroing it afterwards gives what zeroing it
// first and factoring again would.
static rpca_status sk_orth(rpca_ctx* c, SketchBuffers& b, float* Y, int64_t rows, int l) {
  for (int pass = 0; pass < 2; ++pass) {
    if (ts_gram_c(c, Y, rows, l, Y, rows, l, rows, b.st->G, b.ts, c->stream) != cudaSuccess)
      return set_err(c, RPCA_ECUDA, "ts_gram");
    sk_gram_chol_kernel<<<1, SK_CHOL_THREADS, 0, c->stream>>>(b.st, l);
    count_launches(c, 1);
    SK_CUDA(cudaGetLastError());
    SK_CUDA(ts_mul_c(c, Y, rows, l, b.st->Rinv, l, l, Y, rows, rows, 1.f, 0.f, c->stream));
    if (pass == 0) {
      sk_zero_cols_kernel<<<256, 256, 0, c->stream>>>(Y, rows, l, b.st);
      count_launches(c, 1);
    }
  }
  return RPCA_OK;
}

rpca_status sketch_init_large(rpca_ctx* c, const float* Omega, float* U, float* V);  // largek.cu

rpca_status sketch_init(rpca_ctx* c, const float* Omega, float* U, float* V) {
  if (c->lk) return sketch_init_large(c, Omega, U, V);  // k > 16: sketches wider than 32
  const int k = c->k;
  const int l = std::min(std::min(k + std::max(0, c->opt.sketch_oversample), SK_LMAX), std::min(c->m, c->n));
  const int q = std::max(0, c->opt.sketch_power);
  const int64_t m = c->m, n = c->n;
  SketchBuffers* bp = nullptr;
  {
    const rpca_status es = ensure_sketch(c, l, &bp);
    if (es != RPCA_OK) return es;
  }
  SketchBuffers& b = *bp;
  // Om, Y and Z carry lp >= l columns, a multiple of the products' chunk width: the extra
  // columns are zero (so are their products), and every product is whole chunks written in
  // place, without the padded copies of a ragged chunk.
  const int lp = b.lw;
  if (lp > l) {
    SK_CUDA(cudaMemsetAsync(b.Om + n * l, 0, sizeof(float) * n * (lp - l), c->stream));
    SK_CUDA(cudaMemsetAsync(b.Y + m * l, 0, sizeof(float) * m * (lp - l), c->stream));
    SK_CUDA(cudaMemsetAsync(b.Z + n * l, 0, sizeof(float) * n * (lp - l), c->stream));
  }
  if (Omega) cudaMemcpyAsync(b.Om, Omega, sizeof(float) * n * l, cudaMemcpyDeviceToDevice, c->stream);
  else {
    fill_normal(b.Om, n * l, 0xC0FFEEULL ^ (c->opt.seed * 0x9E3779B97F4A7C15ULL), 1.f, c->stream);
    count_launches(c, 1);
  }
  rpca_status s;
  if ((s = sk_apply(c, b, lp, b.Om, nullptr, b.Y, nullptr)) != RPCA_OK) return s;
  if ((s = sk_orth(c, b, b.Y, m, l)) != RPCA_OK) return s;
  for (int it = 0; it < q; ++it) {
    if ((s = sk_apply(c, b, lp, nullptr, b.Y, nullptr, b.Z)) != RPCA_OK) return s;
    if ((s = sk_orth(c, b, b.Z, n, l)) != RPCA_OK) return s;
    if ((s = sk_apply(c, b, lp, b.Z, nullptr, b.Y, nullptr)) != RPCA_OK) return s;
    if ((s = sk_orth(c, b, b.Y, m, l)) != RPCA_OK) return s;
  }
  // B^T = A*(X)^T Q = -(D^T Q) / p_hat.
  if ((s = sk_apply(c, b, lp, nullptr, b.Y, nullptr, b.Z)) != RPCA_OK) return s;
  if (ts_gram_c(c, b.Z, n, l, b.Z, n, l, n, b.st->G, b.ts, c->stream) != cudaSuccess)
    return set_err(c, RPCA_ECUDA, "ts_gram");
  if (!c->sk_sigma && dev_alloc(&c->sk_sigma, sizeof(float) * SK_LMAX) != cudaSuccess)
    return set_err(c, RPCA_ENOMEM, "cudaMalloc");
  const float inv_p = (float)(1.0 / std::max(c->p_hat, 1e-30));
  sk_small_svd_kernel<<<1, 256, 0, c->stream>>>(b.st, l, k, c->sk_sigma, inv_p);
  count_launches(c, 1);
  c->sk_l = l;
  // The Gram was formed from D^T Q = -p_hat B^T: its eigenvalues are p_hat^2 sigma^2, so
  // sqrt(sigma) picks up sqrt(p_hat) -- rescale both factors accordingly.
  const float su = std::sqrt(inv_p);
  if (ts_mul_c(c, b.Y, m, l, b.st->C1, l, k, U, m, m, su, 0.f, c->stream) != cudaSuccess ||
      ts_mul_c(c, b.Z, n, l, b.st->C2, l, k, V, n, n, -su, 0.f, c->stream) != cudaSuccess)
    return set_err(c, RPCA_ECUDA, "ts_mul");
  return check_dev_err(c);
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_init_sketch(rpca_ctx* c, const float* Omega, float* U, float* V) {
  if (!c) return RPCA_EINVAL;
  if (!U || !V) return set_err(c, RPCA_EINVAL, "U and V are required");
  return sketch_init(c, Omega, U, V);
}
