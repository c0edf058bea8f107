// Tall-skinny Gram and multiply kernels (certificate, Lanczos re-orthogonalisation, sketch).
#include <algorithm>

#include "common.cuh"
#include "tsla.h"

namespace rpca {

constexpr int TS_TR = 32;      // rows per shared-memory tile
constexpr int TS_PAD = 33;     // padded column stride of the tile (bank-conflict free)
constexpr int TS_MAXOUT = 9;   // outputs per thread (p * q <= 9 * 256)

// Products in float32 over a 32-row tile, float64 across tiles and blocks.
__global__ void __launch_bounds__(256) ts_gram_kernel(const float* A, int64_t lda, int p, const float* B,
                                                      int64_t ldb, int q, int64_t rows, double* C, double* part,
                                                      unsigned int* counter) {
  extern __shared__ float tile[];
  float* As = tile;
  float* Bs = tile + TS_PAD * p;
  __shared__ bool is_last;
  const int nout = p * q;
  double acc[TS_MAXOUT];
#pragma unroll
  for (int s = 0; s < TS_MAXOUT; ++s) acc[s] = 0.0;
  for (int64_t t0 = (int64_t)blockIdx.x * TS_TR; t0 < rows; t0 += (int64_t)gridDim.x * TS_TR) {
    for (int idx = threadIdx.x; idx < TS_TR * (p + q); idx += blockDim.x) {
      const int r = idx % TS_TR, c = idx / TS_TR;
      const int64_t row = t0 + r;
      float v = 0.f;
      if (row < rows) v = c < p ? A[row + (int64_t)c * lda] : B[row + (int64_t)(c - p) * ldb];
      if (c < p) As[r + c * TS_PAD] = v;
      else Bs[r + (c - p) * TS_PAD] = v;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < TS_MAXOUT; ++s) {
      const int o = threadIdx.x + s * blockDim.x;
      if (o < nout) {
        const int i = o % p, j = o / p;
        float a = 0.f;
#pragma unroll 8
        for (int r = 0; r < TS_TR; ++r) a = fmaf(As[r + i * TS_PAD], Bs[r + j * TS_PAD], a);
        acc[s] += (double)a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < TS_MAXOUT; ++s) {
    const int o = threadIdx.x + s * blockDim.x;
    if (o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[s];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(&part[(int64_t)b * nout + o]);
    C[o] = t;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

cudaError_t ts_gram(const float* A, int64_t lda, int p, const float* B, int64_t ldb, int q, int64_t rows, double* C,
                    const TsScratch& s, cudaStream_t st) {
  if (p * q > TS_MAXOUT * 256 || p < 1 || q < 1) return cudaErrorInvalidValue;
  int grid = (int)std::min<int64_t>((int64_t)s.grid, (rows + TS_TR - 1) / TS_TR);
  grid = std::max(grid, 1);
  if ((size_t)grid * p * q > s.part_n) return cudaErrorInvalidValue;
  const size_t smem = (size_t)TS_PAD * (p + q) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(ts_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  ts_gram_kernel<<<grid, 256, smem, st>>>(A, lda, p, B, ldb, q, rows, C, s.part, s.counter);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) ts_mul_kernel(const float* A, int64_t lda, int p, const double* Cm, int ldc,
                                                     int q, float* Y, int64_t ldy, int64_t rows, float alpha,
                                                     float beta) {
  extern __shared__ float Cs[];  // p x q
  for (int idx = threadIdx.x; idx < p * q; idx += blockDim.x) {
    const int i = idx % p, j = idx / p;
    Cs[idx] = (float)Cm[i + (int64_t)j * ldc];
  }
  __syncthreads();
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    for (int i = 0; i < p; ++i) {
      const float a = A[row + (int64_t)i * lda];
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < q) acc[j] = fmaf(a, Cs[i + j * p], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j < q) {
        float* y = Y + row + (int64_t)j * ldy;
        *y = beta == 0.f ? alpha * acc[j] : fmaf(alpha, acc[j], beta * *y);
      }
    }
  }
}

cudaError_t ts_mul(const float* A, int64_t lda, int p, const double* Cm, int ldc, int q, float* Y, int64_t ldy,
                   int64_t rows, float alpha, float beta, cudaStream_t st) {
  if (q < 1 || q > 32 || p < 1) return cudaErrorInvalidValue;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (rows + 255) / 256));
  const size_t smem = (size_t)p * q * sizeof(float);
  ts_mul_kernel<<<grid, 256, smem, st>>>(A, lda, p, Cm, ldc, q, Y, ldy, rows, alpha, beta);
  return cudaGetLastError();
}

}  // namespace rpca
