// Learned warm start: a three-layer network maps features of the randomized sketch's spectrum
// to the share w_j of each sketch component that the solution keeps; the start is then
// U0 = U_s diag(sqrt(w)), V0 = V_s diag(sqrt(w)) from the sketch start (U_s, V_s) of Sec. 4.2.
// The paper compares SVD, randomized-SVD and random starts only; the network, its training on
// the plain solver's solutions and the fallback to the sketch start when the objective at the
// learned start is not lower are this library's.
//
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3, w = sigmoid(z);
// FEAT = 40 inputs, HID = 256, OUT = 16.  float32 master parameters (packed: W1 | b1 | W2T |
// b2 | W3 | b3, W2T[i][u] = W2[u][i]); the weight matrices are used rounded to bfloat16 (two
// copies of W2: transposed for the forward pass, plain for the backward pass), float32
// arithmetic.  Training: per-CTA partial gradients of 16 samples, summed in a fixed order by
// the Adam kernel (deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "ctx.h"
#include "tsla_ctx.h"

namespace rpca {

constexpr int WS_FEAT = 40, WS_HID = 256, WS_OUT = 16, WS_TB = 16;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + WS_HID * WS_FEAT, OFF_W2T = OFF_B1 + WS_HID;
constexpr int OFF_B2 = OFF_W2T + WS_HID * WS_HID, OFF_W3 = OFF_B2 + WS_HID, OFF_B3 = OFF_W3 + WS_OUT * WS_HID;
constexpr int WS_NPARAM = OFF_B3 + WS_OUT;
// bfloat16 copies: W1 | W2T | W3 | W2 (plain).
constexpr int Q_W1 = 0, Q_W2T = Q_W1 + WS_HID * WS_FEAT, Q_W3 = Q_W2T + WS_HID * WS_HID, Q_W2 = Q_W3 + WS_OUT * WS_HID;
constexpr int WS_NQ = Q_W2 + WS_HID * WS_HID;
constexpr int H_LD = WS_HID + 1;  // padded rows of the activations in shared memory

__global__ void ws_quantize_kernel(const float* theta, __nv_bfloat16* q) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < WS_NQ; i += gridDim.x * blockDim.x) {
    float v;
    if (i < Q_W2T) v = theta[OFF_W1 + i];
    else if (i < Q_W3) v = theta[OFF_W2T + (i - Q_W2T)];
    else if (i < Q_W2) v = theta[OFF_W3 + (i - Q_W3)];
    else {
      const int e = i - Q_W2, u = e / WS_HID, ii = e % WS_HID;  // W2[u][ii] = W2T[ii][u]
      v = theta[OFF_W2T + ii * WS_HID + u];
    }
    q[i] = __float2bfloat16_rn(v);
  }
}

// Shared-memory working set of one CTA (16 samples).
struct WsSmem {
  float x[WS_TB][WS_FEAT];
  float h1[WS_TB][H_LD];
  float h2[WS_TB][H_LD];
  float w[WS_TB][WS_OUT];
  float dz[WS_TB][WS_OUT];
};

// Forward pass of samples [b0, b0 + 16) of X (B x FEAT) into S (rows >= B are zero).
__device__ void ws_forward_tile(const float* theta, const __nv_bfloat16* q, const float* X, int B, int b0, WsSmem& S) {
  const int t = threadIdx.x;
  for (int e = t; e < WS_TB * WS_FEAT; e += blockDim.x) {
    const int s = e / WS_FEAT, i = e % WS_FEAT;
    S.x[s][i] = (b0 + s < B) ? X[(int64_t)(b0 + s) * WS_FEAT + i] : 0.f;
  }
  __syncthreads();
  {  // layer 1: thread u
    const int u = t;
    float acc[WS_TB];
    const float b = theta[OFF_B1 + u];
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) acc[s] = b;
    for (int i = 0; i < WS_FEAT; ++i) {
      const float wv = __bfloat162float(q[Q_W1 + u * WS_FEAT + i]);
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) acc[s] = fmaf(wv, S.x[s][i], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) S.h1[s][u] = fmaxf(acc[s], 0.f);
  }
  __syncthreads();
  {  // layer 2: thread u, W2T[i][u] coalesced over u
    const int u = t;
    float acc[WS_TB];
    const float b = theta[OFF_B2 + u];
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) acc[s] = b;
    for (int i = 0; i < WS_HID; ++i) {
      const float wv = __bfloat162float(q[Q_W2T + i * WS_HID + u]);
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) acc[s] = fmaf(wv, S.h1[s][i], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) S.h2[s][u] = fmaxf(acc[s], 0.f);
  }
  __syncthreads();
  {  // layer 3: warp wp owns outputs 2wp, 2wp + 1; lanes stride over the hidden units
    const int wp = t >> 5, lane = t & 31;
    for (int oo = 0; oo < 2; ++oo) {
      const int o = 2 * wp + oo;
      float acc[WS_TB];
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) acc[s] = 0.f;
      for (int i = lane; i < WS_HID; i += 32) {
        const float wv = __bfloat162float(q[Q_W3 + o * WS_HID + i]);
#pragma unroll
        for (int s = 0; s < WS_TB; ++s) acc[s] = fmaf(wv, S.h2[s][i], acc[s]);
      }
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) {
        float v = acc[s];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) {
          const float z = v + theta[OFF_B3 + o];
          S.w[s][o] = 1.f / (1.f + expf(-z));
        }
      }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) ws_forward_kernel(const float* theta, const __nv_bfloat16* q, const float* X,
                                                         int B, float* W) {
  __shared__ WsSmem S;
  const int b0 = blockIdx.x * WS_TB;
  ws_forward_tile(theta, q, X, B, b0, S);
  for (int e = threadIdx.x; e < WS_TB * WS_OUT; e += blockDim.x) {
    const int s = e / WS_OUT, o = e % WS_OUT;
    if (b0 + s < B) W[(int64_t)(b0 + s) * WS_OUT + o] = S.w[s][o];
  }
}

// Forward + backward of 16 samples: the CTA's partial gradient (packed layout) and its loss.
__global__ void __launch_bounds__(256) ws_train_kernel(const float* theta, const __nv_bfloat16* q, const float* X,
                                                       const float* T, const int* K, int B, float* part,
                                                       float* loss_part) {
  __shared__ WsSmem S;
  __shared__ float red[8];
  const int t = threadIdx.x, b0 = blockIdx.x * WS_TB;
  ws_forward_tile(theta, q, X, B, b0, S);
  float* g = part + (int64_t)blockIdx.x * WS_NPARAM;
  const float inv_b = 1.f / (float)B;
  {  // dz = (2 / B) (w - t) w (1 - w) on valid outputs; the loss
    const int s = t / WS_OUT, o = t % WS_OUT;
    float l = 0.f;
    float d = 0.f;
    if (b0 + s < B && o < K[b0 + s]) {
      const float w = S.w[s][o];
      const float e = w - T[(int64_t)(b0 + s) * WS_OUT + o];
      l = e * e * inv_b;
      d = 2.f * inv_b * e * w * (1.f - w);
    }
    S.dz[s][o] = d;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((t & 31) == 0) red[t >> 5] = l;
  }
  __syncthreads();
  if (t == 0) {
    float l = 0.f;
    for (int i = 0; i < 8; ++i) l += red[i];
    loss_part[blockIdx.x] = l;
  }
  {  // dW3[o][i], db3; then dh2 (in place of h2, thread i owns column i)
    const int i = t;
    float hcol[WS_TB];
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) hcol[s] = S.h2[s][i];
    for (int o = 0; o < WS_OUT; ++o) {
      float a = 0.f;
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) a = fmaf(S.dz[s][o], hcol[s], a);
      g[OFF_W3 + o * WS_HID + i] = a;
    }
    if (i < WS_OUT) {
      float a = 0.f;
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) a += S.dz[s][i];
      g[OFF_B3 + i] = a;
    }
    float wcol[WS_OUT];
#pragma unroll
    for (int o = 0; o < WS_OUT; ++o) wcol[o] = __bfloat162float(q[Q_W3 + o * WS_HID + i]);
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) {
      float a = 0.f;
#pragma unroll
      for (int o = 0; o < WS_OUT; ++o) a = fmaf(wcol[o], S.dz[s][o], a);
      S.h2[s][i] = hcol[s] > 0.f ? a : 0.f;  // dh2
    }
  }
  __syncthreads();
  {  // dW2T[i][u] = sum_s h1[s][i] dh2[s][u] (thread u), db2
    const int u = t;
    float dcol[WS_TB];
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) dcol[s] = S.h2[s][u];
    for (int i = 0; i < WS_HID; ++i) {
      float a = 0.f;
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) a = fmaf(S.h1[s][i], dcol[s], a);
      g[OFF_W2T + i * WS_HID + u] = a;
    }
    float a = 0.f;
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) a += dcol[s];
    g[OFF_B2 + u] = a;
  }
  __syncthreads();
  {  // dh1[s][i] = (h1 > 0) sum_u W2[u][i] dh2[s][u] (thread i, W2 plain copy coalesced over i)
    const int i = t;
    float a[WS_TB];
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) a[s] = 0.f;
    for (int u = 0; u < WS_HID; ++u) {
      const float wv = __bfloat162float(q[Q_W2 + u * WS_HID + i]);
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) a[s] = fmaf(wv, S.h2[s][u], a[s]);
    }
    __syncthreads();  // every thread has read dh2 before dh1 overwrites h1 below
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) S.h1[s][i] = S.h1[s][i] > 0.f ? a[s] : 0.f;  // dh1
  }
  __syncthreads();
  {  // dW1[u][i] = sum_s dh1[s][u] x[s][i] (thread u), db1
    const int u = t;
    float dcol[WS_TB];
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) dcol[s] = S.h1[s][u];
    for (int i = 0; i < WS_FEAT; ++i) {
      float a = 0.f;
#pragma unroll
      for (int s = 0; s < WS_TB; ++s) a = fmaf(dcol[s], S.x[s][i], a);
      g[OFF_W1 + u * WS_FEAT + i] = a;
    }
    float a = 0.f;
#pragma unroll
    for (int s = 0; s < WS_TB; ++s) a += dcol[s];
    g[OFF_B1 + u] = a;
  }
}

// Sum of the CTA partial gradients in CTA order, Adam update of the masters (Kingma & Ba:
// m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, theta -= lr m^ / (sqrt(v^) + eps) with the
// bias corrections m^ = m / (1 - b1^t), v^ = v / (1 - b2^t)); the gradient is also written
// out (grad may be NULL).
__global__ void ws_adam_kernel(float* theta, float* m, float* v, const float* part, int nblk, float* grad, float lr,
                               float beta1, float beta2, float eps, float corr1, float corr2) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < WS_NPARAM; p += gridDim.x * blockDim.x) {
    float gsum = 0.f;
    for (int b = 0; b < nblk; ++b) gsum += part[(int64_t)b * WS_NPARAM + p];
    if (grad) grad[p] = gsum;
    const float mm = beta1 * m[p] + (1.f - beta1) * gsum;
    const float vv = beta2 * v[p] + (1.f - beta2) * gsum * gsum;
    m[p] = mm;
    v[p] = vv;
    theta[p] -= lr * (mm / corr1) / (sqrtf(vv / corr2) + eps);
  }
}

// Features of the sketch spectrum s (l values, descending), see the header.
__global__ void ws_features_kernel(const float* sig, int l, int k, double lam_L, double lam_S, double m, double n,
                                   float* x) {
  const int i = threadIdx.x;
  if (i >= WS_FEAT) return;
  const double s_ref = fmax(fmax((double)sig[l - 1], 1e-30 * (double)sig[0]), 1e-300);
  double v = 0.0;
  if (i < l) v = log(fmax((double)sig[i], 1e-300) / s_ref);
  else if (i == 32) v = log(lam_L / s_ref);
  else if (i == 33) v = isinf(lam_S) ? 0.0 : log(lam_S * sqrt(m * n) / s_ref);
  else if (i == 34) v = k / 16.0;
  else if (i == 35) v = l / 32.0;
  else if (i == 36) v = log(m / n) / 4.0;
  else if (i == 37) v = log(m * n) / 20.0;
  if (i >= l && i < 32) v = 0.0;
  x[i] = (float)v;
}

// w*_j = clip(sum_c Gu[j][c] Gv[j][c] / s_j^2, 0, 1), Gu = Us^T U (k x k), Gv = Vs^T V.
__global__ void ws_targets_kernel(const double* Gu, const double* Gv, const float* sig, int k, float* wstar) {
  const int j = threadIdx.x;
  if (j >= WS_OUT) return;
  float r = 0.f;
  if (j < k) {
    double a = 0.0;
    for (int c = 0; c < k; ++c) a += Gu[j + c * k] * Gv[j + c * k];
    const double s = sig[j];
    r = s > 0.0 ? (float)fmin(fmax(a / (s * s), 0.0), 1.0) : 0.f;
  }
  wstar[j] = r;
}

// Y[:, j] = A[:, j] sqrt(w_j) (rows x k, column-major).
__global__ void ws_scale_cols_kernel(const float* A, float* Y, int64_t rows, int k, const float* w) {
  const int64_t total = rows * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = A[e] * sqrtf(fmaxf(w[e / rows], 0.f));
}

}  // namespace rpca

struct rpca_ws {
  float* theta = nullptr;  // WS_NPARAM masters
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* q = nullptr;
  float* part = nullptr;
  float* loss_part = nullptr;
  int part_blocks = 0;
  int t = 0;  // Adam steps taken
  cudaStream_t stream = nullptr;
  std::string err;
};

using namespace rpca;

namespace {
thread_local char g_ws_err[256];
rpca_status ws_fail(rpca_ws* w, rpca_status s, const char* msg) {
  if (w) w->err = msg;
  snprintf(g_ws_err, sizeof g_ws_err, "%s", msg);
  return s;
}
#define WS_CUDA(w, call)                                                  \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return ws_fail(w, RPCA_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

rpca_status ws_requantize(rpca_ws* w) {
  ws_quantize_kernel<<<256, 256, 0, w->stream>>>(w->theta, w->q);
  WS_CUDA(w, cudaGetLastError());
  return RPCA_OK;
}
}  // namespace

extern "C" {

int rpca_ws_nparam(void) { return WS_NPARAM; }

rpca_status rpca_ws_create(rpca_ws** out, const float* theta, void* cuda_stream) {
  if (!out || !theta) return ws_fail(nullptr, RPCA_EINVAL, "rpca_ws_create: out and theta are required");
  *out = nullptr;
  rpca_ws* w = new (std::nothrow) rpca_ws();
  if (!w) return RPCA_ENOMEM;
  w->stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t pb = sizeof(float) * WS_NPARAM;
  if (cudaMalloc(&w->theta, pb) != cudaSuccess || cudaMalloc(&w->m, pb) != cudaSuccess ||
      cudaMalloc(&w->v, pb) != cudaSuccess || cudaMalloc(&w->grad, pb) != cudaSuccess ||
      cudaMalloc(&w->q, sizeof(__nv_bfloat16) * WS_NQ) != cudaSuccess) {
    rpca_ws_destroy(w);
    return ws_fail(nullptr, RPCA_ENOMEM, "rpca_ws_create: cudaMalloc");
  }
  const rpca_status s = rpca_ws_set_params(w, theta);
  if (s != RPCA_OK) {
    rpca_ws_destroy(w);
    return s;
  }
  *out = w;
  return RPCA_OK;
}

rpca_status rpca_ws_set_params(rpca_ws* w, const float* theta) {
  if (!w || !theta) return ws_fail(w, RPCA_EINVAL, "rpca_ws_set_params: model and theta are required");
  const size_t pb = sizeof(float) * WS_NPARAM;
  WS_CUDA(w, cudaMemcpyAsync(w->theta, theta, pb, cudaMemcpyHostToDevice, w->stream));
  WS_CUDA(w, cudaMemsetAsync(w->m, 0, pb, w->stream));
  WS_CUDA(w, cudaMemsetAsync(w->v, 0, pb, w->stream));
  WS_CUDA(w, cudaMemsetAsync(w->grad, 0, pb, w->stream));
  w->t = 0;
  rpca_status s = ws_requantize(w);
  if (s != RPCA_OK) return s;
  WS_CUDA(w, cudaStreamSynchronize(w->stream));
  return RPCA_OK;
}

rpca_status rpca_ws_get_params(rpca_ws* w, float* theta, float* grad) {
  if (!w || !theta) return ws_fail(w, RPCA_EINVAL, "rpca_ws_get_params: model and theta are required");
  WS_CUDA(w, cudaMemcpyAsync(theta, w->theta, sizeof(float) * WS_NPARAM, cudaMemcpyDeviceToHost, w->stream));
  if (grad) WS_CUDA(w, cudaMemcpyAsync(grad, w->grad, sizeof(float) * WS_NPARAM, cudaMemcpyDeviceToHost, w->stream));
  WS_CUDA(w, cudaStreamSynchronize(w->stream));
  return RPCA_OK;
}

rpca_status rpca_ws_predict(rpca_ws* w, const float* X, int B, float* W) {
  if (!w || !X || !W || B < 0) return ws_fail(w, RPCA_EINVAL, "rpca_ws_predict: bad arguments");
  if (B == 0) return RPCA_OK;
  ws_forward_kernel<<<(B + WS_TB - 1) / WS_TB, 256, 0, w->stream>>>(w->theta, w->q, X, B, W);
  WS_CUDA(w, cudaGetLastError());
  return RPCA_OK;
}

rpca_status rpca_ws_train_step(rpca_ws* w, const float* X, const float* T, const int* K, int B, float lr,
                               float* loss) {
  if (!w || !X || !T || !K || B < 1 || !(lr >= 0.f)) return ws_fail(w, RPCA_EINVAL, "rpca_ws_train_step: bad arguments");
  const int nblk = (B + WS_TB - 1) / WS_TB;
  if (nblk > w->part_blocks) {
    cudaStreamSynchronize(w->stream);
    cudaFree(w->part);
    cudaFree(w->loss_part);
    w->part = nullptr;
    w->loss_part = nullptr;
    w->part_blocks = 0;
    WS_CUDA(w, cudaMalloc(&w->part, sizeof(float) * (size_t)nblk * WS_NPARAM));
    WS_CUDA(w, cudaMalloc(&w->loss_part, sizeof(float) * nblk));
    w->part_blocks = nblk;
  }
  ws_train_kernel<<<nblk, 256, 0, w->stream>>>(w->theta, w->q, X, T, K, B, w->part, w->loss_part);
  w->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, w->t)), c2 = (float)(1.0 - std::pow(0.999, w->t));
  ws_adam_kernel<<<(WS_NPARAM + 255) / 256, 256, 0, w->stream>>>(w->theta, w->m, w->v, w->part, nblk, w->grad, lr, b1,
                                                                  b2, 1e-8f, c1, c2);
  rpca_status s = ws_requantize(w);
  if (s != RPCA_OK) return s;
  if (loss) {
    float lp[4096];
    const int nb = std::min(nblk, 4096);
    WS_CUDA(w, cudaMemcpyAsync(lp, w->loss_part, sizeof(float) * nb, cudaMemcpyDeviceToHost, w->stream));
    WS_CUDA(w, cudaStreamSynchronize(w->stream));
    double l = 0.0;
    for (int i = 0; i < nb; ++i) l += lp[i];
    *loss = (float)l;
  }
  return RPCA_OK;
}

const char* rpca_ws_last_error(const rpca_ws* w) { return w ? w->err.c_str() : g_ws_err; }

void rpca_ws_destroy(rpca_ws* w) {
  if (!w) return;
  if (w->stream) cudaStreamSynchronize(w->stream);
  cudaFree(w->theta);
  cudaFree(w->m);
  cudaFree(w->v);
  cudaFree(w->grad);
  cudaFree(w->q);
  cudaFree(w->part);
  cudaFree(w->loss_part);
  delete w;
}

rpca_status rpca_set_warm_start(rpca_ctx* c, const rpca_ws* w) {
  if (!c) return RPCA_EINVAL;
  c->ws_model = w;
  return RPCA_OK;
}

rpca_status rpca_sketch_spectrum(rpca_ctx* c, float* s, int* l) {
  if (!c || !s || !l) return RPCA_EINVAL;
  *l = c->sk_l;
  if (c->sk_l == 0) return RPCA_OK;
  RPCA_CUDA(c, cudaMemcpyAsync(s, c->sk_sigma, sizeof(float) * c->sk_l, cudaMemcpyDeviceToHost, c->stream));
  RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
  return RPCA_OK;
}

}  // extern "C"

namespace rpca {

rpca_status ws_features(rpca_ctx* c, float* x) {
  if (c->sk_l < 1) return set_err(c, RPCA_EINVAL, "no sketch spectrum: run the sketch initialisation first");
  ws_features_kernel<<<1, 64, 0, c->stream>>>(c->sk_sigma, c->sk_l, c->k, c->lam_L, c->lam_S, (double)c->m,
                                              (double)c->n, x);
  count_launches(c, 1);
  RPCA_CUDA(c, cudaGetLastError());
  return RPCA_OK;
}

}  // namespace rpca

extern "C" rpca_status rpca_ws_sample(rpca_ctx* c, const float* Us, const float* Vs, const float* U, const float* V,
                                      float* x, float* wstar) {
  if (!c) return RPCA_EINVAL;
  if (!x) return set_err(c, RPCA_EINVAL, "x is required");
  rpca_status s = ws_features(c, x);
  if (s != RPCA_OK || !wstar) return s;
  if (!Us || !Vs || !U || !V) return set_err(c, RPCA_EINVAL, "Us, Vs, U and V are required for the targets");
  const int k = c->k;
  double* G = nullptr;
  TsScratch ts;
  ts.grid = 2 * c->nsm;
  ts.part_n = (size_t)ts.grid * 2304;
  RPCA_CUDA(c, cudaMalloc(&G, sizeof(double) * (2 * k * k + ts.part_n)));
  ts.part = G + 2 * k * k;
  cudaError_t e = ts_gram_c(c, Us, c->m, k, U, c->m, k, c->m, G, ts, c->stream);
  if (e == cudaSuccess) e = ts_gram_c(c, Vs, c->n, k, V, c->n, k, c->n, G + k * k, ts, c->stream);
  if (e == cudaSuccess) {
    ws_targets_kernel<<<1, 32, 0, c->stream>>>(G, G + k * k, c->sk_sigma, k, wstar);
    count_launches(c, 1);
    e = cudaGetLastError();
  }
  cudaStreamSynchronize(c->stream);
  cudaFree(G);
  if (e != cudaSuccess) return cuda_err(c, e, "rpca_ws_sample");
  return RPCA_OK;
}

namespace rpca {

// The learned start: U, V hold the sketch start on entry; the network's w scales its columns,
// and the scaled start replaces it only when its objective is lower (the plain solver's
// objective is the judge).  *used = 1 when the learned start was kept.
rpca_status ws_learned_init(rpca_ctx* c, float* U, float* V, int* used) {
  *used = 0;
  const rpca_ws* w = c->ws_model;
  if (!w) return set_err(c, RPCA_EINVAL, "RPCA_INIT_LEARNED needs a model (rpca_set_warm_start)");
  const int64_t mk = (int64_t)c->m * c->k, nk = (int64_t)c->n * c->k;
  // Scratch kept by the context (a cudaFree per solve would wait for every stream).
  const size_t need = (size_t)(2 * (mk + nk) + 64);
  if (c->ws_buf_n < need) {
    if (c->ws_buf) {
      RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
      cudaFree(c->ws_buf);
      c->ws_buf = nullptr;
      c->ws_buf_n = 0;
    }
    RPCA_CUDA(c, cudaMalloc(&c->ws_buf, sizeof(float) * need));
    c->ws_buf_n = need;
  }
  float* buf = c->ws_buf;
  float* Ul = buf;
  float* Vl = Ul + mk;
  float* G = Vl + nk;  // gradient scratch, mk + nk
  float* xw = G + mk + nk;  // 40 features | 16 outputs
  rpca_status s = ws_features(c, xw);
  if (s != RPCA_OK) return s;
  ws_forward_kernel<<<1, 256, 0, c->stream>>>(w->theta, w->q, xw, 1, xw + WS_FEAT);
  ws_scale_cols_kernel<<<std::max<int64_t>(1, std::min<int64_t>(1024, (mk + 255) / 256)), 256, 0, c->stream>>>(
      U, Ul, c->m, c->k, xw + WS_FEAT);
  ws_scale_cols_kernel<<<std::max<int64_t>(1, std::min<int64_t>(1024, (nk + 255) / 256)), 256, 0, c->stream>>>(
      V, Vl, c->n, c->k, xw + WS_FEAT);
  count_launches(c, 3);
  RPCA_CUDA(c, cudaGetLastError());
  double f[2] = {0.0, 0.0};
  const float* UU[2] = {U, Ul};
  const float* VV[2] = {V, Vl};
  for (int q = 0; q < 2; ++q) {
    FgLaunch L;
    L.U = UU[q];
    L.V = VV[q];
    L.GU = G;
    L.GV = G + mk;
    if ((s = launch_fg(c, c->fg_plan, L, c->stream)) != RPCA_OK) return s;
    RPCA_CUDA(c, cudaMemcpyAsync(&f[q], c->ws.out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if (std::isfinite(f[1]) && f[1] < f[0]) {
    RPCA_CUDA(c, cudaMemcpyAsync(U, Ul, sizeof(float) * mk, cudaMemcpyDeviceToDevice, c->stream));
    RPCA_CUDA(c, cudaMemcpyAsync(V, Vl, sizeof(float) * nk, cudaMemcpyDeviceToDevice, c->stream));
    *used = 1;
  }
  return RPCA_OK;
}

}  // namespace rpca
