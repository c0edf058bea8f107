// Precision form: the library's narrow copy of X (bfloat16, or FP8 E4M3 with a per-column
// scale), read by the fused kernel in place of the caller's float32 X until the solver
// refines on float32 X.  Conversions round to nearest (ties to even); FP8 saturates at
// +-448 and stores x / s_j with s_j = max_i |x_ij| / 448 over the observed entries of column
// j (s_j = 1 for an all-zero column).  Unobserved entries are stored as 0.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "ctx.h"
#include "fg_kernel.cuh"

namespace rpca {

__device__ inline bool xq_observed(const uint32_t* bits, int wpad, int i, int j) {
  return bits == nullptr || ((bits[(int64_t)j * wpad + (i >> 5)] >> (i & 31)) & 1u);
}

// One block per column: s_j = max |x_ij| / 448 over observed i (exact maximum, then one
// float32 division).
__global__ void __launch_bounds__(256) xq_scale_kernel(const float* X, int64_t ldx, const uint32_t* bits, int wpad,
                                                       int m, int n, float* scale) {
  __shared__ float wmax[8];
  const int j = blockIdx.x;
  if (j >= n) return;
  float mx = 0.f;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    if (xq_observed(bits, wpad, i, j)) mx = fmaxf(mx, fabsf(X[i + (int64_t)j * ldx]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, wmax[w]);
    scale[j] = t > 0.f ? t / 448.0f : 1.0f;
  }
}

template <int XT>
__global__ void __launch_bounds__(256) xq_convert_kernel(const float* X, int64_t ldx, const uint32_t* bits, int wpad,
                                                         int m, int n, const float* scale, void* Xq, int64_t ldq) {
  const int64_t total = (int64_t)ldq * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / ldq), i = (int)(e - (int64_t)j * ldq);
    float x = 0.f;
    if (i < m && xq_observed(bits, wpad, i, j)) x = X[i + (int64_t)j * ldx];
    if constexpr (XT == FG_X_BF16) {
      reinterpret_cast<uint16_t*>(Xq)[e] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    } else {
      const float y = x / scale[j];
      reinterpret_cast<uint8_t*>(Xq)[e] = (uint8_t)__nv_cvt_float_to_fp8(y, __NV_SATFINITE, __NV_E4M3);
    }
  }
}

// Allocates and fills the narrow copy (ldq a multiple of 16 elements: 16-byte aligned rows
// for the tensor copies) and, for FP8, the column scales.
rpca_status make_xq(rpca_ctx* c, int xt) {
  c->xq_dt = xt;
  c->ldq = ((int64_t)c->m + 15) / 16 * 16;
  const size_t bytes = (size_t)c->ldq * c->n * fg_x_bytes(xt);
  cudaError_t e;
  if ((e = cudaMalloc(&c->Xq, bytes)) != cudaSuccess) return cuda_err(c, e, "cudaMalloc (narrow copy of X)");
  if (xt == FG_X_E4M3) {
    if ((e = cudaMalloc(&c->xscale, sizeof(float) * c->n)) != cudaSuccess) return cuda_err(c, e, "cudaMalloc");
    xq_scale_kernel<<<c->n, 256, 0, c->stream>>>(c->X, c->ldx, c->bits, c->wpad, c->m, c->n, c->xscale);
    count_launches(c, 1);
  }
  const int64_t total = (int64_t)c->ldq * c->n;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 8LL * c->nsm);
  if (xt == FG_X_BF16)
    xq_convert_kernel<FG_X_BF16><<<grid, 256, 0, c->stream>>>(c->X, c->ldx, c->bits, c->wpad, c->m, c->n, c->xscale,
                                                              c->Xq, c->ldq);
  else
    xq_convert_kernel<FG_X_E4M3><<<grid, 256, 0, c->stream>>>(c->X, c->ldx, c->bits, c->wpad, c->m, c->n, c->xscale,
                                                              c->Xq, c->ldq);
  count_launches(c, 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(c, e, "converting X");
  return RPCA_OK;
}

}  // namespace rpca
