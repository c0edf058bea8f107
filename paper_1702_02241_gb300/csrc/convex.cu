// The convex baseline of Sec. 6.1: FISTA on the Lagrangian SPCP program with S marginalised,
//   min_L lam_L ||L||_* + phi(L),   phi(L) = sum_Omega psi(L - X),   grad phi 1-Lipschitz,
// whose prox (singular-value thresholding) is taken on a rank-l randomized SVD with every QR a
// TSQR.  Dense m x n float32 iterates; one iteration (q power iterations):
//   pass   Z = Y - P_Omega clip(Y - X),  Y = L + beta (L - L_prev),  A = Z Omega      (fused;
//          also phi(L), ||L - L_prev||^2, ||L||^2 for the objective and the stopping test)
//   rSVD   Q = tsqr(A); q times {Q_w = tsqr(Z^T Q), Q = tsqr(Z Q_w)}; W = Z^T Q = Q_w R_w;
//          R_w = U_r diag(s) V_r^T (one-warp Jacobi)
//   prox   L_new = (Q V_r diag(max(s - lam_L, 0))) (Q_w U_r)^T   (rank-l product pass)
// and Omega for the next iteration = Q_w U_r (the right singular basis found).  Every pass over
// an m x n array is a stream through HBM (4 rows per thread, 16-byte accesses); the sketch
// products keep the l-wide operand in registers and reduce across lanes with a butterfly
// reduce-scatter.  Deterministic: every reduction is in a fixed order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "smallla.cuh"
#include "tsqr.h"

namespace rpca {

constexpr int CV_T = 128;          // threads per block of the passes
constexpr int CV_ROWS = 4 * CV_T;  // rows per block
constexpr int CV_NB = 8;           // column groups per shared-memory flush of the Z^T Q pass

RPCA_DEV double cv_block_sum(double v, double* scr) {
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

RPCA_DEV void cv_load4(const float* p, bool full, int64_t left, float* v) {
  if (full) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = r < left ? p[r] : 0.f;
  }
}

RPCA_DEV void cv_store4(float* p, bool full, int64_t left, const float* v) {
  if (full) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (r < left) p[r] = v[r];
  }
}

// GRAD: Z = Y - P_Omega clip(Y - X) written, partials {phi(L), ||L - Lp||^2, ||L||^2} per block.
// Otherwise Z is read.  Both: Apart[blockIdx.y] (l x mp, column-major) = Z[:, chunk] Om[chunk, :]
// with Om row-major (row j at Om + j LP, zero past l).  Grid (row blocks, column chunks).
template <int LP, bool GRAD>
__global__ void __launch_bounds__(CV_T) cv_sketch_kernel(const float* L, const float* Lp, const float* X, int64_t ldx,
                                                         const uint8_t* mask, int64_t ldmask, int64_t m, int64_t n,
                                                         float beta, float lam, float* Z, int64_t ldz,
                                                         const float* Om, int l, float* Apart, int64_t mp,
                                                         double* part) {
  __shared__ double scr[CV_T / 32];
  const int64_t i0 = (int64_t)blockIdx.x * CV_ROWS + 4 * threadIdx.x;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t j0 = (int64_t)blockIdx.y * per, j1 = std::min<int64_t>(n, j0 + per);
  float acc[4][LP];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < LP; ++c) acc[r][c] = 0.f;
  double phi = 0.0, dl2 = 0.0, l2 = 0.0;
  if (i0 < m) {
    const bool full = i0 + 3 < m;
    const int64_t left = m - i0;
    for (int64_t j = j0; j < j1; ++j) {
      float z[4];
      if (GRAD) {
        float lv[4], pv[4], xv[4];
        cv_load4(L + i0 + j * ldz, full, left, lv);
        cv_load4(Lp + i0 + j * ldz, full, left, pv);
        cv_load4(X + i0 + j * ldx, full, left, xv);
        float ph = 0.f, d2 = 0.f, n2 = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const bool on = r < left && (mask == nullptr || mask[i0 + r + j * ldmask] != 0);
          const float y = fmaf(beta, lv[r] - pv[r], lv[r]);
          const float dy = on ? fminf(fmaxf(y - xv[r], -lam), lam) : 0.f;
          z[r] = y - dy;
          const float rl = lv[r] - xv[r];
          const float dl = on ? fminf(fmaxf(rl, -lam), lam) : 0.f;
          ph = fmaf(dl, rl - 0.5f * dl, ph);  // psi(r) = d (r - d / 2), d = clip(r)
          const float df = lv[r] - pv[r];
          d2 = fmaf(df, df, d2);
          n2 = fmaf(lv[r], lv[r], n2);
        }
        cv_store4(Z + i0 + j * ldz, full, left, z);
        phi += ph;
        dl2 += d2;
        l2 += n2;
      } else {
        cv_load4(Z + i0 + j * ldz, full, left, z);
      }
      const float4* o4 = reinterpret_cast<const float4*>(Om + j * LP);
#pragma unroll
      for (int c4 = 0; c4 < LP / 4; ++c4) {
        const float4 o = __ldg(o4 + c4);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          acc[r][4 * c4 + 0] = fmaf(z[r], o.x, acc[r][4 * c4 + 0]);
          acc[r][4 * c4 + 1] = fmaf(z[r], o.y, acc[r][4 * c4 + 1]);
          acc[r][4 * c4 + 2] = fmaf(z[r], o.z, acc[r][4 * c4 + 2]);
          acc[r][4 * c4 + 3] = fmaf(z[r], o.w, acc[r][4 * c4 + 3]);
        }
      }
    }
    float* ap = Apart + (size_t)blockIdx.y * l * mp;
#pragma unroll
    for (int c = 0; c < LP; ++c) {
      if (c < l) {
        const float v[4] = {acc[0][c], acc[1][c], acc[2][c], acc[3][c]};
        cv_store4(ap + (size_t)c * mp + i0, full, left, v);
      }
    }
  }
  if (GRAD) {
    const double a = cv_block_sum(phi, scr);
    const double b = cv_block_sum(dl2, scr);
    const double c = cv_block_sum(l2, scr);
    if (threadIdx.x == 0) {
      const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
      part[3 * blk + 0] = a;
      part[3 * blk + 1] = b;
      part[3 * blk + 2] = c;
    }
  }
}

// Wpart[blockIdx.x] (l x n, column-major) = (rows of the block)^T: Z[rows, chunk]^T Q[rows, :].
// Each thread keeps its 4 rows of Q in registers; 32 / LP columns at a time, the 32 per-lane
// partial products are summed over the warp by a butterfly reduce-scatter (lane e ends with
// output e), the warps' sums are added through shared memory every CV_NB column groups.
template <int LP>
__global__ void __launch_bounds__(CV_T) cv_left_kernel(const float* Z, int64_t ldz, int64_t m, int64_t n,
                                                       const float* Q, int64_t ldq, int l, float* Wpart) {
  constexpr int NC = 32 / LP;
  __shared__ float red[CV_T / 32][CV_NB][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * CV_ROWS + 4 * threadIdx.x;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t j0 = (int64_t)blockIdx.y * per, j1 = std::min<int64_t>(n, j0 + per);
  const bool full = i0 + 3 < m;
  const int64_t left = m - i0;
  float q[4][LP];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < LP; ++c) q[r][c] = (r < left && c < l) ? Q[i0 + r + (int64_t)c * ldq] : 0.f;
  for (int64_t jb = j0; jb < j1; jb += NC * CV_NB) {
#pragma unroll 1
    for (int g = 0; g < CV_NB; ++g) {
      float v[32];
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        const int64_t j = jb + g * NC + s;
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (j < j1 && left > 0) cv_load4(Z + i0 + j * ldz, full, left, z);
#pragma unroll
        for (int c = 0; c < LP; ++c) {
          float t = z[0] * q[0][c];
          t = fmaf(z[1], q[1][c], t);
          t = fmaf(z[2], q[2][c], t);
          v[s * LP + c] = fmaf(z[3], q[3][c], t);
        }
      }
#pragma unroll
      for (int o = 16, h = 16; o >= 1; o >>= 1, h >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int t = 0; t < h; ++t) {
          const float send = up ? v[t] : v[t + h];
          const float keep = up ? v[t + h] : v[t];
          v[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      red[w][g][lane] = v[0];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * CV_NB; t += CV_T) {
      const int g = t >> 5, e = t & 31;
      float s = 0.f;
#pragma unroll
      for (int ww = 0; ww < CV_T / 32; ++ww) s += red[ww][g][e];
      const int64_t j = jb + g * NC + e / LP;
      const int c = e % LP;
      if (j < j1 && c < l) Wpart[(size_t)blockIdx.x * l * n + (size_t)c * n + j] = s;
    }
    __syncthreads();
  }
}

// W (n x l, column-major, ld n) = sum over nb blocks of Wpart, in a fixed order: each block
// takes 32 consecutive outputs, 8 threads per output sum every 8th partial, then the 8 sums
// are added in order.
__global__ void __launch_bounds__(256) cv_wsum_kernel(const float* Wpart, int nb, int64_t nl, float* W) {
  __shared__ float part[8][32];
  const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
  for (int64_t e0 = (int64_t)blockIdx.x * 32; e0 < nl; e0 += (int64_t)gridDim.x * 32) {
    const int64_t e = e0 + o;
    float s = 0.f;
    if (e < nl)
      for (int b = g; b < nb; b += 8) s += Wpart[(size_t)b * nl + e];
    part[g][o] = s;
    __syncthreads();
    if (g == 0 && e < nl) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += part[q][o];
      W[e] = t;
    }
    __syncthreads();
  }
}

// Out = A C with A rows x l (column-major, lda) and C l x l (column-major, ld l): column-major
// out (ld ldo) or, when rowmajor, row i at Out + i * ldo with the entries past l zeroed.
template <int LP>
__global__ void __launch_bounds__(256) cv_mul_kernel(const float* A, int64_t lda, int64_t rows, int l, const float* C,
                                                     float* Out, int64_t ldo, int rowmajor) {
  __shared__ float Cs[LP * LP];
  for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
    const int a = e % LP, c = e / LP;
    Cs[e] = (a < l && c < l) ? C[a + c * l] : 0.f;
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    float a[LP];
#pragma unroll
    for (int t = 0; t < LP; ++t) a[t] = t < l ? A[i + t * lda] : 0.f;
#pragma unroll
    for (int c = 0; c < LP; ++c) {
      float v = 0.f;
#pragma unroll
      for (int t = 0; t < LP; ++t) v = fmaf(a[t], Cs[t + c * LP], v);
      if (rowmajor) {
        if (c < ldo) Out[i * ldo + c] = v;
      } else if (c < l) {
        Out[i + c * ldo] = v;
      }
    }
  }
}

// Lout = P Vr^T: P m x l (column-major, ld mp), Vr row-major (row j at Vr + j LP, zero past l).
template <int LP>
__global__ void __launch_bounds__(CV_T) cv_recon_kernel(const float* P, int64_t mp, int64_t m, int64_t n, int l,
                                                        const float* Vr, float* Lout, int64_t ldl) {
  const int64_t i0 = (int64_t)blockIdx.x * CV_ROWS + 4 * threadIdx.x;
  if (i0 >= m) return;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t j0 = (int64_t)blockIdx.y * per, j1 = std::min<int64_t>(n, j0 + per);
  const bool full = i0 + 3 < m;
  const int64_t left = m - i0;
  float p[4][LP];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < LP; ++c) p[r][c] = (r < left && c < l) ? P[i0 + r + (int64_t)c * mp] : 0.f;
  for (int64_t j = j0; j < j1; ++j) {
    const float4* v4 = reinterpret_cast<const float4*>(Vr + j * LP);
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c4 = 0; c4 < LP / 4; ++c4) {
      const float4 v = __ldg(v4 + c4);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        o[r] = fmaf(p[r][4 * c4 + 0], v.x, o[r]);
        o[r] = fmaf(p[r][4 * c4 + 1], v.y, o[r]);
        o[r] = fmaf(p[r][4 * c4 + 2], v.z, o[r]);
        o[r] = fmaf(p[r][4 * c4 + 3], v.w, o[r]);
      }
    }
    cv_store4(Lout + i0 + j * ldl, full, left, o);
  }
}

// SVD of R_w (l x l) by one-sided Jacobi in float32 on one warp (lane j holds column j; no
// barriers), sorted descending: Cl = V_r diag(s_thr) and Cr = U_r (both l x l, column-major),
// s_thr = max(s - lam_L, 0); info = {sum s_thr, rank (s_thr > 0), s_1, s_l}.  One warp.
template <int LP>
__global__ void __launch_bounds__(32) cv_small_svd_kernel(const float* Rw, int l, double lamL, float* Cl, float* Cr,
                                                          double* sv, double* info) {
  __shared__ float A[LP * LP], V[LP * LP], sig[LP];
  __shared__ int ord[LP];
  for (int e = threadIdx.x; e < l * l; e += 32) A[e] = Rw[e];
  __syncwarp();
  const float eps = 6e-8f;
  warp_jacobi_svd<float, LP, LP>(A, l, l, l, V, l, sig, 40, 8.f * l * eps, 4.f * l * eps);
  cta_sort_desc<float>(sig, l, ord);
  for (int e = threadIdx.x; e < l * l; e += 32) {
    const int a = e % l, o = e / l;
    const int c = ord[o];
    const float s = sig[c];
    const float st = (double)s > lamL ? (float)((double)s - lamL) : 0.f;
    Cl[e] = V[a + c * l] * st;
    Cr[e] = s > 0.f ? A[a + c * l] / s : 0.f;
  }
  if (threadIdx.x == 0) {
    double tot = 0.0;
    int r = 0;
    for (int o = 0; o < l; ++o) {
      const double s = (double)sig[ord[o]];
      sv[o] = s;
      if (s > lamL) {
        tot += s - lamL;
        ++r;
      }
    }
    info[0] = tot;
    info[1] = r;
    info[2] = (double)sig[ord[0]];
    info[3] = (double)sig[ord[l - 1]];
  }
}

// Omega in the row-major padded layout from an n x l column-major device matrix.
__global__ void cv_rowmajor_kernel(const float* A, int64_t lda, int64_t n, int l, int LP, float* Out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * LP; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / LP;
    const int c = (int)(e % LP);
    Out[e] = c < l ? A[j + c * lda] : 0.f;
  }
}

template <int LP>
void cv_launch_sketch(bool grad, dim3 g, cudaStream_t st, const float* L, const float* Lp, const float* X, int64_t ldx,
                      const uint8_t* mask, int64_t ldmask, int64_t m, int64_t n, float beta, float lam, float* Z,
                      int64_t ldz, const float* Om, int l, float* Apart, int64_t mp, double* part) {
  if (grad)
    cv_sketch_kernel<LP, true><<<g, CV_T, 0, st>>>(L, Lp, X, ldx, mask, ldmask, m, n, beta, lam, Z, ldz, Om, l, Apart,
                                                   mp, part);
  else
    cv_sketch_kernel<LP, false><<<g, CV_T, 0, st>>>(L, Lp, X, ldx, mask, ldmask, m, n, beta, lam, Z, ldz, Om, l,
                                                    Apart, mp, part);
}

// Scratch of the solver, kept on the context between solves of the same shape.
struct ConvexBuffers {
  int l = 0, LP = 0, gx = 0, gy = 0, gyl = 0;  // gyl: column chunks of the Z^T Q pass
  int64_t ldl = 0, mp = 0;
  TsqrPlan pm, pn;
  float* buf = nullptr;
  double* dbl = nullptr;    // block partials, singular values, info
  double* host = nullptr;   // pinned copy of dbl
  size_t nd = 0;
  float *L1 = nullptr, *L2 = nullptr, *Z = nullptr, *Ap = nullptr, *Q = nullptr, *P = nullptr, *Wp = nullptr,
        *W = nullptr, *Qw = nullptr, *Om = nullptr, *Ow = nullptr, *Cl = nullptr, *Cr = nullptr, *Rw = nullptr,
        *Tm = nullptr, *Tn = nullptr;
};

void cvx_free(rpca_ctx* c) {
  if (!c->cvx) return;
  cudaFree(c->cvx->buf);
  cudaFree(c->cvx->dbl);
  cudaFreeHost(c->cvx->host);
  delete c->cvx;
  c->cvx = nullptr;
}

static rpca_status cvx_setup(rpca_ctx* c, int l, int64_t ldl) {
  if (c->cvx && c->cvx->l == l && c->cvx->ldl == ldl) return RPCA_OK;
  cvx_free(c);
  const int64_t m = c->m, n = c->n;
  auto* b = new ConvexBuffers;
  b->l = l;
  b->LP = l <= 8 ? 8 : (l <= 16 ? 16 : 32);
  b->ldl = ldl;
  b->mp = (m + 3) & ~(int64_t)3;
  b->gx = (int)((m + CV_ROWS - 1) / CV_ROWS);
  b->gy = (int)std::max<int64_t>(1, std::min<int64_t>({n, 16, (int64_t)(4 * c->nsm + b->gx - 1) / b->gx}));
  b->gyl = b->gy;
  b->pm = tsqr_plan(m, l, c->nsm);
  b->pn = tsqr_plan(n, l, c->nsm);
  // Two more iterate buffers and Z (ldl x n each), A partials (gy x l x mp), Q and P (mp x l),
  // W partials (gx x l x n), W and Q_w (n x l), Omega and Omega_w (n x LP, row-major), the
  // small coefficient matrices, the TSQR workspaces.
  size_t off = 0;
  auto take = [&](size_t nf) {
    const size_t o = off;
    off += (nf + 63) & ~(size_t)63;
    return o;
  };
  const size_t big = (size_t)ldl * n;
  const size_t oL1 = take(big), oL2 = take(big), oZ = take(big), oAp = take((size_t)b->gy * l * b->mp),
               oQ = take((size_t)b->mp * l), oP = take((size_t)b->mp * l), oWp = take((size_t)b->gx * l * n),
               oW = take((size_t)n * l), oQw = take((size_t)n * l), oOm = take((size_t)n * b->LP),
               oOw = take((size_t)n * b->LP), oCl = take((size_t)l * l), oCr = take((size_t)l * l),
               oRw = take((size_t)l * l), oTm = take(b->pm.ws_floats), oTn = take(b->pn.ws_floats);
  b->nd = 3 * (size_t)b->gx * b->gy + TQ_LMAX + 8;
  if (cudaMalloc(&b->buf, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&b->dbl, sizeof(double) * b->nd) != cudaSuccess ||
      cudaMallocHost(&b->host, sizeof(double) * b->nd) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->buf);
    cudaFree(b->dbl);
    delete b;
    return set_err(c, RPCA_ENOMEM, "the convex solver's scratch does not fit");
  }
  float* f = b->buf;
  b->L1 = f + oL1;
  b->L2 = f + oL2;
  b->Z = f + oZ;
  b->Ap = f + oAp;
  b->Q = f + oQ;
  b->P = f + oP;
  b->Wp = f + oWp;
  b->W = f + oW;
  b->Qw = f + oQw;
  b->Om = f + oOm;
  b->Ow = f + oOw;
  b->Cl = f + oCl;
  b->Cr = f + oCr;
  b->Rw = f + oRw;
  b->Tm = f + oTm;
  b->Tn = f + oTn;
  c->cvx = b;
  return RPCA_OK;
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_convex_solve(rpca_ctx* c, float* L, int64_t ldl, int l, int power_iters,
                                         const float* Omega0, int max_iter, double tol, int profile, double* log,
                                         rpca_convex_result* res) {
  if (!c) return RPCA_EINVAL;
  if (!L || ldl < c->m || (ldl * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(L) & 15) != 0)
    return set_err(c, RPCA_EINVAL, "L must be 16-byte aligned with ldl >= m a multiple of 4");
  if (l < 1 || l > TQ_LMAX || l > c->m || l > c->n)
    return set_err(c, RPCA_EINVAL, "the sketch width l must lie in [1, min(32, m, n)]");
  if (!Omega0 || power_iters < 0 || power_iters > 16 || max_iter < 0 || !(tol >= 0.0))
    return set_err(c, RPCA_EINVAL, "Omega0 required; 0 <= power_iters <= 16; max_iter, tol >= 0");
  if (c->xq_dt != 0) return set_err(c, RPCA_EUNSUPPORTED, "the convex solver reads float32 X");
  if (!tsqr_allow_smem()) return set_err(c, RPCA_ECUDA, "TSQR shared-memory opt-in failed");
  const auto t0 = std::chrono::steady_clock::now();
  rpca_status s0 = cvx_setup(c, l, ldl);
  if (s0 != RPCA_OK) return s0;
  ConvexBuffers& B = *c->cvx;
  const int64_t m = c->m, n = c->n;
  cudaStream_t st = c->stream;
  const float lam = std::isinf(c->lam_S) ? INFINITY : (float)c->lam_S;
  const double lamL = c->lam_L;
  const int LP = B.LP, gx = B.gx, gy = B.gy;
  const int64_t mp = B.mp;
  const int nblk = gx * gy;
  const size_t nd = B.nd;
  double* part = B.dbl;
  double* sv = part + 3 * (size_t)nblk;
  double* info = sv + TQ_LMAX;
  const double* hp = B.host;
  float* Lb[3] = {L, B.L1, B.L2};
  // Events: [0, 1] the pass, [2] the host copy of its sums, then two alternating sets (one per
  // iteration parity) of {rSVD start, after the coefficient products, after the
  // reconstruction, TSQR start / end pairs}: an iteration's set is read at the next one's wait.
  const int nq = 2 * power_iters + 2;
  const int per_set = 3 + 2 * nq;
  std::vector<cudaEvent_t> ev(3 + 2 * (size_t)per_set);
  for (size_t i = 0; i < ev.size(); ++i)
    if (cudaEventCreateWithFlags(&ev[i], (profile || i == 2) ? cudaEventDefault : cudaEventDisableTiming) !=
        cudaSuccess) {
      for (size_t j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
      return set_err(c, RPCA_ECUDA, "cudaEventCreate");
    }
  auto finish = [&](rpca_status s) {
    cudaStreamSynchronize(st);
    for (auto& e : ev) cudaEventDestroy(e);
    return s;
  };
  const dim3 g2(gx, gy);
  const int mul_grid_m = (int)std::min<int64_t>(4 * c->nsm, (m + 255) / 256);
  const int mul_grid_n = (int)std::min<int64_t>(4 * c->nsm, (n + 255) / 256);
  const int ws_grid = (int)std::min<int64_t>(8 * c->nsm, ((int64_t)n * l + 31) / 32);
  auto sketch = [&](bool grad, const float* Lc, const float* Lpv, float beta, const float* Omx) {
    if (LP == 8)
      cv_launch_sketch<8>(grad, g2, st, Lc, Lpv, c->X, c->ldx, c->mask, c->ldmask, m, n, beta, lam, B.Z, ldl, Omx,
                          l, B.Ap, mp, part);
    else if (LP == 16)
      cv_launch_sketch<16>(grad, g2, st, Lc, Lpv, c->X, c->ldx, c->mask, c->ldmask, m, n, beta, lam, B.Z, ldl, Omx,
                           l, B.Ap, mp, part);
    else
      cv_launch_sketch<32>(grad, g2, st, Lc, Lpv, c->X, c->ldx, c->mask, c->ldmask, m, n, beta, lam, B.Z, ldl, Omx,
                           l, B.Ap, mp, part);
    count_launches(c, 1);
  };
  const dim3 gl2(gx, B.gyl);
  auto left = [&](const float* Qm) {  // W = Z^T Q
    if (LP == 8)
      cv_left_kernel<8><<<gl2, CV_T, 0, st>>>(B.Z, ldl, m, n, Qm, mp, l, B.Wp);
    else if (LP == 16)
      cv_left_kernel<16><<<gl2, CV_T, 0, st>>>(B.Z, ldl, m, n, Qm, mp, l, B.Wp);
    else
      cv_left_kernel<32><<<gl2, CV_T, 0, st>>>(B.Z, ldl, m, n, Qm, mp, l, B.Wp);
    cv_wsum_kernel<<<ws_grid, 256, 0, st>>>(B.Wp, gx, (int64_t)n * l, B.W);
    count_launches(c, 2);
  };
  auto mul = [&](const float* A, int64_t lda, int64_t rows, const float* C, float* Out, int64_t ldo, int rm,
                 int grid) {
    if (LP == 8)
      cv_mul_kernel<8><<<grid, 256, 0, st>>>(A, lda, rows, l, C, Out, ldo, rm);
    else if (LP == 16)
      cv_mul_kernel<16><<<grid, 256, 0, st>>>(A, lda, rows, l, C, Out, ldo, rm);
    else
      cv_mul_kernel<32><<<grid, 256, 0, st>>>(A, lda, rows, l, C, Out, ldo, rm);
    count_launches(c, 1);
  };
  auto recon = [&](float* Lout) {
    if (LP == 8)
      cv_recon_kernel<8><<<g2, CV_T, 0, st>>>(B.P, mp, m, n, l, B.Om, Lout, ldl);
    else if (LP == 16)
      cv_recon_kernel<16><<<g2, CV_T, 0, st>>>(B.P, mp, m, n, l, B.Om, Lout, ldl);
    else
      cv_recon_kernel<32><<<g2, CV_T, 0, st>>>(B.P, mp, m, n, l, B.Om, Lout, ldl);
    count_launches(c, 1);
  };
  int set = 0, qi = 0;
  auto evs = [&](int which, int i) -> cudaEvent_t& { return ev[3 + (size_t)which * per_set + i]; };
  auto tsqr = [&](const TsqrPlan& p, const float* A, int64_t lda, int npart, int64_t ps, float* Qo, int64_t ldq,
                  bool rm, float* R, float* ws) -> cudaError_t {
    count_launches(c, p.launches);
    if (profile) cudaEventRecord(evs(set, 3 + 2 * qi), st);
    const cudaError_t e = tsqr_run(p, A, lda, npart, ps, Qo, ldq, rm, R, ws, st);
    if (profile) cudaEventRecord(evs(set, 4 + 2 * qi), st);
    ++qi;
    return e;
  };
  auto elapsed = [&](cudaEvent_t a, cudaEvent_t b) {
    float x = 0.f;
    cudaEventElapsedTime(&x, a, b);
    return (double)x;
  };
  // Start: L = L_prev = 0, Omega = Omega0.
  RPCA_CUDA(c, cudaMemset2DAsync(Lb[0], sizeof(float) * ldl, 0, sizeof(float) * m, n, st));
  RPCA_CUDA(c, cudaMemset2DAsync(Lb[1], sizeof(float) * ldl, 0, sizeof(float) * m, n, st));
  cv_rowmajor_kernel<<<mul_grid_n, 256, 0, st>>>(Omega0, n, n, l, LP, B.Om);
  count_launches(c, 1);
  int cur = 0, prev = 1, spare = 2;
  double t_prev = 1.0, t = 1.0, nuc = 0.0, F = 0.0, phi = 0.0, rel = 0.0;
  double info_h[4] = {0, 0, 0, 0};
  double ms_tot[4] = {0, 0, 0, 0};  // pass, rSVD, TSQR (part of the rSVD), reconstruction
  int k = 0, qi_prev = 0;
  for (;; ++k) {
    // The pass at L_k and the host copy of its sums; then, speculatively, the prox of iteration
    // k (it writes only the spare iterate buffer and the sketch scratch) while the host waits
    // for the sums and takes the stopping decision.
    const double beta = k == 0 ? 0.0 : (t_prev - 1.0) / t;
    if (profile) cudaEventRecord(ev[0], st);
    sketch(true, Lb[cur], Lb[prev], (float)beta, B.Om);
    if (profile) cudaEventRecord(ev[1], st);
    RPCA_CUDA(c, cudaMemcpyAsync(B.host, part, sizeof(double) * nd, cudaMemcpyDeviceToHost, st));
    RPCA_CUDA(c, cudaEventRecord(ev[2], st));
    cudaError_t e = cudaSuccess;
    if (k < max_iter) {
      set = k & 1;
      qi = 0;
      if (profile) cudaEventRecord(evs(set, 0), st);
      e = tsqr(B.pm, B.Ap, mp, gy, (int64_t)l * mp, B.Q, mp, false, nullptr, B.Tm);
      for (int p = 0; p < power_iters && e == cudaSuccess; ++p) {
        left(B.Q);
        e = tsqr(B.pn, B.W, n, 1, 0, B.Ow, LP, true, nullptr, B.Tn);
        if (e != cudaSuccess) break;
        sketch(false, nullptr, nullptr, 0.f, B.Ow);
        e = tsqr(B.pm, B.Ap, mp, gy, (int64_t)l * mp, B.Q, mp, false, nullptr, B.Tm);
      }
      if (e == cudaSuccess) {
        left(B.Q);
        e = tsqr(B.pn, B.W, n, 1, 0, B.Qw, n, false, B.Rw, B.Tn);
      }
      if (e == cudaSuccess) {
        if (LP == 8)
          cv_small_svd_kernel<8><<<1, 32, 0, st>>>(B.Rw, l, lamL, B.Cl, B.Cr, sv, info);
        else if (LP == 16)
          cv_small_svd_kernel<16><<<1, 32, 0, st>>>(B.Rw, l, lamL, B.Cl, B.Cr, sv, info);
        else
          cv_small_svd_kernel<32><<<1, 32, 0, st>>>(B.Rw, l, lamL, B.Cl, B.Cr, sv, info);
        count_launches(c, 1);
        // Prox: P = Q Cl, Omega <- Q_w Cr (the right basis: the next sketch's test matrix),
        // L_{k+1} = P Omega^T.
        mul(B.Q, mp, m, B.Cl, B.P, mp, 0, mul_grid_m);
        mul(B.Qw, n, n, B.Cr, B.Om, LP, 1, mul_grid_n);
        if (profile) cudaEventRecord(evs(set, 1), st);
        recon(Lb[spare]);
        if (profile) cudaEventRecord(evs(set, 2), st);
        e = cudaGetLastError();
      }
    }
    if (e != cudaSuccess) return finish(cuda_err(c, e, "rpca_convex_solve"));
    e = cudaEventSynchronize(ev[2]);
    if (e != cudaSuccess) return finish(cuda_err(c, e, "rpca_convex_solve"));
    if (profile) {
      ms_tot[0] += elapsed(ev[0], ev[1]);
      if (k > 0) {  // the previous iteration's prox ran before this pass
        const int ps = (k - 1) & 1;
        ms_tot[1] += elapsed(evs(ps, 0), evs(ps, 1));
        ms_tot[3] += elapsed(evs(ps, 1), evs(ps, 2));
        for (int i = 0; i < qi_prev; ++i) ms_tot[2] += elapsed(evs(ps, 3 + 2 * i), evs(ps, 4 + 2 * i));
      }
    }
    qi_prev = qi;
    double s_phi = 0.0, s_dl = 0.0, s_l = 0.0;
    for (int b = 0; b < nblk; ++b) {
      s_phi += hp[3 * b];
      s_dl += hp[3 * b + 1];
      s_l += hp[3 * b + 2];
    }
    if (k > 0) {
      for (int i = 0; i < 4; ++i) info_h[i] = hp[3 * (size_t)nblk + TQ_LMAX + i];
      nuc = info_h[0];  // ||L_k||_*: the thresholded singular values that formed L_k
    }
    phi = s_phi;
    F = lamL * nuc + phi;
    rel = std::sqrt(s_dl) / std::max(1.0, std::sqrt(s_l));
    if (log) {
      log[4 * k + 0] = F;
      log[4 * k + 1] = rel;
      log[4 * k + 2] = k > 0 ? info_h[1] : 0.0;
      log[4 * k + 3] = k > 0 ? info_h[3] : 0.0;
    }
    if ((k > 0 && rel <= tol) || k >= max_iter) break;
    const int old_prev = prev;
    prev = cur;
    cur = spare;
    spare = old_prev;
    t_prev = t;
    t = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
  }
  if (cur != 0)
    RPCA_CUDA(c, cudaMemcpy2DAsync(L, sizeof(float) * ldl, Lb[cur], sizeof(float) * ldl, sizeof(float) * m, n,
                                   cudaMemcpyDeviceToDevice, st));
  const rpca_status s = finish(check_dev_err(c));
  if (res) {
    memset(res, 0, sizeof *res);
    res->F = F;
    res->phi = phi;
    res->nuclear = nuc;
    res->rel_change = rel;
    res->iters = k;
    res->rank = k > 0 ? (int)info_h[1] : 0;
    res->truncated = k > 0 && info_h[3] > lamL ? 1 : 0;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    res->ms_pass = ms_tot[0];
    res->ms_rsvd = ms_tot[1];
    res->ms_tsqr = ms_tot[2];
    res->ms_recon = ms_tot[3];
  }
  return s;
}
