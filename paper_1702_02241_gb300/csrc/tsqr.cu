// TSQR (Sec. 6.1, after Demmel, Grigori, Hoemmen and Langou): the QR factorisation of a
// tall-skinny float32 matrix A (rows x l, l <= 32) by a reduction tree.
//   leaves  one CTA per row block (b rows, the last one up to 2b - 1): Householder QR in shared
//           memory, R_p (l x l) out, the block's explicit Q_p into a column-major scratch;
//   levels  one CTA per group of up to G stacked R's: Householder QR of the stack, its R up a
//           level, its explicit Q (G l x l) kept;
//   root    R = D R_root with D = sign(diag R_root), so that R has a non-negative diagonal (the
//           unique QR of a full-rank A);
//   expand  top-down, each node's l x l multiplier E_child = (slice of the parent's Q) E_parent,
//           E_root = D;
//   apply   Q rows of leaf p = Q_p E_p.
// The QRs run in float32 (the GPU's float64 rate is a few operations per clock per SM): a
// Householder QR is backward stable, so Q is orthonormal and Q R = A to a few float32 ulps
// times a modest factor of the size, whatever A's condition.  Every reduction is in a fixed
// order (deterministic).
#include <algorithm>

#include "common.cuh"
#include "ctx.h"
#include "tsqr.h"

namespace rpca {

constexpr int TQ_T = 256;

// Sum over the CTA, returned to every thread.  red: 32 shared floats.
RPCA_DEV float tq_cta_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Householder QR of A (rows x cols, rows >= cols, column-major, ld) in shared memory, by the
// CTA.  On return the upper triangle holds R (R[j][j] = beta_j), the strict lower part of
// column j the reflector v_j (v_j[j] = 1 implied), tau[j] its coefficient: H_j = I - tau v v^T
// maps the column's trailing part x to beta_j e_1 with beta_j = -sign(x_1) ||x|| (tau = 0 and
// beta_j = x_1 when the part below the diagonal is zero).
__device__ void tq_house_qr(float* A, int rows, int cols, int ld, float* tau, float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < cols; ++j) {
    float* a = A + (size_t)j * ld;
    float s = 0.f;
    for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) s = fmaf(a[i], a[i], s);
    s = tq_cta_sum(s, red);
    const float alpha = a[j];
    float t = 0.f, beta = alpha, scale = 0.f;
    if (s > 0.f) {
      const float nrm = sqrtf(fmaf(alpha, alpha, s));
      beta = alpha >= 0.f ? -nrm : nrm;
      t = (beta - alpha) / beta;
      scale = 1.f / (alpha - beta);
    }
    for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) a[i] *= scale;
    __syncthreads();
    // b <- H_j b for the columns right of j: d = tau (b_j + v^T b), b -= d v.
    for (int cc = j + 1 + w; cc < cols; cc += nw) {
      float* b = A + (size_t)cc * ld;
      const float bj = b[j];
      float d = 0.f;
      float d1 = 0.f;
      int i = j + 1 + lane;
#pragma unroll 2
      for (; i + 32 < rows; i += 64) {
        d = fmaf(a[i], b[i], d);
        d1 = fmaf(a[i + 32], b[i + 32], d1);
      }
      if (i < rows) d = fmaf(a[i], b[i], d);
      d += d1;
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      d = t * (d + bj);
#pragma unroll 4
      for (int i2 = j + 1 + lane; i2 < rows; i2 += 32) b[i2] = fmaf(-d, a[i2], b[i2]);
      if (lane == 0) b[j] = bj - d;
    }
    if (threadIdx.x == 0) {
      a[j] = beta;
      tau[j] = t;
    }
    __syncthreads();
  }
}

// The explicit Q = H_0 H_1 ... H_{cols-1} [I; 0] (rows x cols), formed in place from the
// reflectors left by tq_house_qr, last reflector first (column j of Q takes its final value at
// step j; the columns to its right are updated by H_j).
__device__ void tq_house_q(float* A, int rows, int cols, int ld, const float* tau) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = cols - 1; j >= 0; --j) {
    float* a = A + (size_t)j * ld;
    const float t = tau[j];
    for (int cc = j + 1 + w; cc < cols; cc += nw) {
      float* b = A + (size_t)cc * ld;
      const float bj = b[j];
      float d = 0.f;
      float d1 = 0.f;
      int i = j + 1 + lane;
#pragma unroll 2
      for (; i + 32 < rows; i += 64) {
        d = fmaf(a[i], b[i], d);
        d1 = fmaf(a[i + 32], b[i + 32], d1);
      }
      if (i < rows) d = fmaf(a[i], b[i], d);
      d += d1;
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      d = t * (d + bj);
#pragma unroll 4
      for (int i2 = j + 1 + lane; i2 < rows; i2 += 32) b[i2] = fmaf(-d, a[i2], b[i2]);
      if (lane == 0) b[j] = bj - d;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) a[i] = i > j ? -t * a[i] : (i == j ? 1.f - t : 0.f);
    __syncthreads();
  }
}

// Writes the upper triangle of the factored S (rows x l, ld) as an l x l column-major R.
RPCA_DEV void tq_store_r(const float* S, int ld, int l, float* R) {
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int a = e % l, c = e / l;
    R[e] = a <= c ? S[a + (size_t)c * ld] : 0.f;
  }
}

// Leaf p: rows [p b, p b + nb) of A (the sum of npart partials), QR, R_p and Q_p out.
__global__ void __launch_bounds__(TQ_T) tq_leaf_kernel(const float* A, int64_t lda, int npart, int64_t pstride,
                                                       int64_t rows, int l, int b, int P, float* Qt, float* Rl) {
  extern __shared__ float tq_smem[];
  __shared__ float tau[TQ_LMAX], red[32];
  const int p = blockIdx.x;
  const int64_t r0 = (int64_t)p * b;
  const int nb = (int)(p == P - 1 ? rows - r0 : b);
  float* S = tq_smem;
  // Unrolled so that the loads of several elements and partials are in flight together (the
  // partials are added in order).
#pragma unroll 4
  for (int e = threadIdx.x; e < nb * l; e += blockDim.x) {
    const int i = e % nb, c = e / nb;
    const float* src = A + (r0 + i) + (int64_t)c * lda;
    float v = 0.f;
#pragma unroll 4
    for (int t = 0; t < npart; ++t) v += src[(int64_t)t * pstride];
    S[e] = v;
  }
  __syncthreads();
  tq_house_qr(S, nb, l, nb, tau, red);
  tq_store_r(S, nb, l, Rl + (size_t)p * l * l);
  __syncthreads();
  tq_house_q(S, nb, l, nb, tau);
  for (int e = threadIdx.x; e < nb * l; e += blockDim.x) {
    const int i = e % nb, c = e / nb;
    Qt[(r0 + i) + (int64_t)c * rows] = S[e];
  }
}

// Node p of a level: children [p G, p G + g) of the level below, their R's stacked.
__global__ void __launch_bounds__(TQ_T) tq_node_kernel(const float* Rin, int nin, int l, int G, float* Qn,
                                                       float* Rout) {
  extern __shared__ float tq_smem[];
  __shared__ float tau[TQ_LMAX], red[32];
  const int p = blockIdx.x;
  const int c0 = p * G;
  const int g = min(G, nin - c0);
  const int rows = g * l;
  float* S = tq_smem;
  for (int e = threadIdx.x; e < rows * l; e += blockDim.x) {
    const int i = e % rows, c = e / rows;
    const int s = i / l, a = i % l;
    S[e] = Rin[(size_t)(c0 + s) * l * l + a + (size_t)c * l];
  }
  __syncthreads();
  tq_house_qr(S, rows, l, rows, tau, red);
  tq_store_r(S, rows, l, Rout + (size_t)p * l * l);
  __syncthreads();
  tq_house_q(S, rows, l, rows, tau);
  const int ldn = G * l;
  for (int e = threadIdx.x; e < rows * l; e += blockDim.x) {
    const int i = e % rows, c = e / rows;
    Qn[(size_t)p * ldn * l + i + (size_t)c * ldn] = S[e];
  }
}

// R = D R_root, E_root = D with D = sign(diag R_root) (+1 for a zero diagonal entry).
__global__ void tq_root_kernel(const float* Rr, int l, float* R, float* E) {
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int a = e % l, c = e / l;
    const float d = Rr[a + (size_t)a * l] < 0.f ? -1.f : 1.f;
    if (R) R[e] = d * Rr[e];
    E[e] = a == c ? d : 0.f;
  }
}

// E of child ch (parent ch / G, slot s = ch % G): rows [s l, s l + l) of the parent's Q times
// the parent's E.
__global__ void tq_expand_kernel(const float* Qn, const float* Ep, int l, int G, float* Ec) {
  const int ch = blockIdx.x;
  const int p = ch / G, s = ch % G;
  const int ldn = G * l;
  const float* Q = Qn + (size_t)p * ldn * l;
  const float* E = Ep + (size_t)p * l * l;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int a = e % l, c = e / l;
    float v = 0.f;
    for (int t = 0; t < l; ++t) v = fmaf(Q[s * l + a + (size_t)t * ldn], E[t + (size_t)c * l], v);
    Ec[(size_t)ch * l * l + e] = v;
  }
}

// Rows of leaf p: Q = Q_p E_p, one row per thread.
template <int LP>
__global__ void __launch_bounds__(TQ_T) tq_apply_kernel(const float* Qt, int64_t rows, int l, int b, int P,
                                                        const float* El, float* Q, int64_t ldq, int rowmajor) {
  __shared__ float E[LP * LP];
  const int p = blockIdx.x;
  for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
    const int a = e % LP, c = e / LP;
    E[e] = (a < l && c < l) ? El[(size_t)p * l * l + a + (size_t)c * l] : 0.f;
  }
  __syncthreads();
  const int64_t r0 = (int64_t)p * b;
  const int64_t r1 = p == P - 1 ? rows : r0 + b;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    float q[LP];
#pragma unroll
    for (int t = 0; t < LP; ++t) q[t] = t < l ? Qt[i + (int64_t)t * rows] : 0.f;
#pragma unroll
    for (int c = 0; c < LP; ++c) {
      float v = 0.f;
#pragma unroll
      for (int t = 0; t < LP; ++t) v = fmaf(q[t], E[t + c * LP], v);
      if (rowmajor) {
        if (c < ldq) Q[i * ldq + c] = v;  // zero past l (E is zero-padded)
      } else if (c < l) {
        Q[i + (int64_t)c * ldq] = v;
      }
    }
    if (rowmajor)
      for (int64_t c = LP; c < ldq; ++c) Q[i * ldq + c] = 0.f;
  }
}

TsqrPlan tsqr_plan(int64_t rows, int l, int nsm) {
  TsqrPlan p;
  p.rows = rows;
  p.l = l;
  if (l < 1 || l > TQ_LMAX || rows < l) return p;
  const int64_t bmax = std::max<int64_t>(l, (TQ_SMEM_FLOATS / l + 1) / 2);
  int64_t b = std::max<int64_t>(32, (rows + 2 * (int64_t)nsm - 1) / (2 * (int64_t)nsm));
  b = std::max<int64_t>(l, std::min(b, bmax));
  p.b = (int)b;
  p.P = (int)std::max<int64_t>(1, rows / b);
  p.G = std::max(2, std::min(32, TQ_SMEM_FLOATS / (l * l)));
  p.cnt[0] = p.P;
  while (p.cnt[p.nlev] > 1 && p.nlev < TQ_MAXLEV) {
    p.cnt[p.nlev + 1] = (p.cnt[p.nlev] + p.G - 1) / p.G;
    ++p.nlev;
  }
  size_t off = 0;
  auto take = [&](size_t nf) {
    const size_t o = off;
    off += (nf + 63) & ~(size_t)63;
    return o;
  };
  p.offQt = take((size_t)rows * l);
  for (int v = 0; v <= p.nlev; ++v) {
    p.offR[v] = take((size_t)p.cnt[v] * l * l);
    p.offE[v] = take((size_t)p.cnt[v] * l * l);
    if (v > 0) p.offQn[v] = take((size_t)p.cnt[v] * p.G * l * l);
  }
  p.ws_floats = off;
  const int64_t maxblk = std::max<int64_t>(b, rows - (int64_t)(p.P - 1) * b);
  p.smem_leaf = sizeof(float) * (size_t)maxblk * l;
  p.smem_node = sizeof(float) * (size_t)p.G * l * l;
  p.launches = 3 + 2 * p.nlev;
  return p;
}

bool tsqr_allow_smem() {
  static int ok = -1;
  if (ok < 0) {
    const size_t bytes = sizeof(float) * TQ_SMEM_FLOATS;
    ok = allow_smem((const void*)tq_leaf_kernel, bytes) && allow_smem((const void*)tq_node_kernel, bytes);
  }
  return ok == 1;
}

cudaError_t tsqr_run(const TsqrPlan& p, const float* A, int64_t lda, int npart, int64_t part_stride, float* Q,
                     int64_t ldq, bool rowmajor, float* R, float* ws, cudaStream_t st) {
  if (p.P < 1) return cudaErrorInvalidValue;
  const int l = p.l;
  float* Qt = ws + p.offQt;
  tq_leaf_kernel<<<p.P, TQ_T, p.smem_leaf, st>>>(A, lda, npart, part_stride, p.rows, l, p.b, p.P, Qt, ws + p.offR[0]);
  for (int v = 1; v <= p.nlev; ++v)
    tq_node_kernel<<<p.cnt[v], TQ_T, p.smem_node, st>>>(ws + p.offR[v - 1], p.cnt[v - 1], l, p.G, ws + p.offQn[v],
                                                         ws + p.offR[v]);
  tq_root_kernel<<<1, 256, 0, st>>>(ws + p.offR[p.nlev], l, R, ws + p.offE[p.nlev]);
  for (int v = p.nlev; v >= 1; --v)
    tq_expand_kernel<<<p.cnt[v - 1], 256, 0, st>>>(ws + p.offQn[v], ws + p.offE[v], l, p.G, ws + p.offE[v - 1]);
  const int rm = rowmajor ? 1 : 0;
  if (l <= 8)
    tq_apply_kernel<8><<<p.P, TQ_T, 0, st>>>(Qt, p.rows, l, p.b, p.P, ws + p.offE[0], Q, ldq, rm);
  else if (l <= 16)
    tq_apply_kernel<16><<<p.P, TQ_T, 0, st>>>(Qt, p.rows, l, p.b, p.P, ws + p.offE[0], Q, ldq, rm);
  else
    tq_apply_kernel<32><<<p.P, TQ_T, 0, st>>>(Qt, p.rows, l, p.b, p.P, ws + p.offE[0], Q, ldq, rm);
  return cudaGetLastError();
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_tsqr(rpca_ctx* c, const float* A, int64_t lda, int64_t rows, int l, float* Q,
                                 int64_t ldq, float* R) {
  if (!c) return RPCA_EINVAL;
  if (!A || !Q || l < 1 || l > TQ_LMAX || rows < l || lda < rows || ldq < rows)
    return set_err(c, RPCA_EINVAL, "rpca_tsqr: 1 <= l <= 32, rows >= l, lda and ldq >= rows, A and Q required");
  if (!tsqr_allow_smem()) return set_err(c, RPCA_ECUDA, "rpca_tsqr: shared-memory opt-in failed");
  const TsqrPlan p = tsqr_plan(rows, l, c->nsm);
  float* ws = nullptr;
  RPCA_CUDA(c, cudaMallocAsync(&ws, sizeof(float) * p.ws_floats, c->stream));
  const cudaError_t e = tsqr_run(p, A, lda, 1, 0, Q, ldq, false, R, ws, c->stream);
  count_launches(c, p.launches);
  cudaFreeAsync(ws, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "rpca_tsqr");
  RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_dev_err(c);
}
