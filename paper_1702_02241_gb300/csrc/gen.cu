// Device generator of planted low-rank + sparse + noise instances (training data of the
// learned warm start): counter-based Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC 2011), so that any entry is a pure function of
// (seed, instance, position) and instances are generated on the GPU in any order.
//
// Counters (key = the 64-bit seed as two 32-bit words, low first):
//   A[i][c] (m x rank): ctr = (i, c, 0, instance); B[j][c] (n x rank): ctr = (j, c, 1, instance);
//   X[i][j]:             ctr = (i, j, 2, instance).
// From the four output words w0..w3 of a counter:
//   uniform24(w) = (w >> 8) 2^-24 in [0, 1);  a normal is Box-Muller on (w_a, w_b):
//   sqrt(-2 ln((w_a >> 8) + 1) 2^-24) cos(2 pi uniform24(w_b)).
//   A, B entries: normal(w0, w1) * rank^(-1/4) (variance 1/sqrt(rank), so L = A B^T has
//   unit-variance entries).  X entries: outlier when uniform24(w0) < p_outlier, sign from the
//   top bit of w1 (set: negative), magnitude 1 + 4 (w1 & 0xffffff) 2^-24; noise
//   noise_std * normal(w2, w3).  X = A B^T + S + N in float32.
#include <cmath>
#include <cstdint>

#include "ctx.h"

namespace rpca {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ float uniform24(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

__device__ __forceinline__ float normal_of(uint32_t wa, uint32_t wb) {
  const float u1 = (float)((wa >> 8) + 1u) * (1.0f / 16777216.0f);  // (0, 1]
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * uniform24(wb));
}

// F[r][c] (rows x rank, column-major, ld rows) = normal * scale, stream word `which`.
__global__ void gen_factor_kernel(float* F, int64_t rows, int rank, uint32_t which, uint32_t inst, uint32_t k0,
                                  uint32_t k1, float scale) {
  const int64_t total = rows * rank;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows;
    const int c = (int)(e / rows);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)c, which, inst), k0, k1);
    F[e] = scale * normal_of(w.x, w.y);
  }
}

// X[i][j] = sum_c A[i][c] B[j][c] + outlier + noise; one thread per entry, rows fastest.
__global__ void gen_x_kernel(float* X, int64_t ldx, float* L0, int64_t m, int64_t n, int rank, const float* A,
                             const float* B, float p_out, float noise_std, uint32_t inst, uint32_t k0, uint32_t k1) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    float l = 0.f;
    for (int c = 0; c < rank; ++c) l = fmaf(A[i + c * m], B[j + c * n], l);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)j, 2u, inst), k0, k1);
    float s = 0.f;
    if (uniform24(w.x) < p_out) {
      const float mag = 1.0f + 4.0f * (float)(w.y & 0xffffffu) * (1.0f / 16777216.0f);
      s = (w.y >> 31) ? -mag : mag;
    }
    X[i + j * ldx] = l + s + noise_std * normal_of(w.z, w.w);
    if (L0) L0[e] = l;
  }
}

// Raw Philox words for counters (c0 + t, c1, c2, c3), t < count (known-answer checks).
__global__ void gen_philox_words_kernel(uint32_t* out, int64_t count, uint32_t c0, uint32_t c1, uint32_t c2,
                                        uint32_t c3, uint32_t k0, uint32_t k1) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4(c0 + (uint32_t)t, c1, c2, c3), k0, k1);
    out[4 * t + 0] = w.x;
    out[4 * t + 1] = w.y;
    out[4 * t + 2] = w.z;
    out[4 * t + 3] = w.w;
  }
}

}  // namespace rpca

using namespace rpca;

extern "C" {

rpca_status rpca_gen_planted(int64_t m, int64_t n, int rank, double p_outlier, double noise_std, uint64_t seed,
                             uint32_t instance, float* X, int64_t ldx, float* L0, void* cuda_stream) {
  if (m < 1 || n < 1 || m >= (1LL << 32) || n >= (1LL << 32) || rank < 1 || rank > 64 || !X || ldx < m ||
      !(p_outlier >= 0.0 && p_outlier <= 1.0) || !(noise_std >= 0.0))
    return set_err_noctx(RPCA_EINVAL, "rpca_gen_planted: bad sizes, rank (1..64), p_outlier or noise_std");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  float* AB = nullptr;
  if (cudaMallocAsync(&AB, sizeof(float) * (size_t)(m + n) * rank, st) != cudaSuccess)
    return set_err_noctx(RPCA_ENOMEM, "rpca_gen_planted: cudaMallocAsync");
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const float scale = (float)std::pow((double)rank, -0.25);
  auto grid = [](int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>(8192, (total + 255) / 256)); };
  gen_factor_kernel<<<grid(m * rank), 256, 0, st>>>(AB, m, rank, 0u, instance, k0, k1, scale);
  gen_factor_kernel<<<grid(n * rank), 256, 0, st>>>(AB + m * rank, n, rank, 1u, instance, k0, k1, scale);
  gen_x_kernel<<<grid(m * n), 256, 0, st>>>(X, ldx, L0, m, n, rank, AB, AB + m * rank, (float)p_outlier,
                                            (float)noise_std, instance, k0, k1);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(AB, st);
  if (e != cudaSuccess) return set_err_noctx(RPCA_ECUDA, cudaGetErrorString(e));
  return RPCA_OK;
}

rpca_status rpca_philox4x32_10(uint32_t* out, int64_t count, const uint32_t* ctr, uint64_t key, void* cuda_stream) {
  if (!out || !ctr || count < 0) return set_err_noctx(RPCA_EINVAL, "rpca_philox4x32_10: bad arguments");
  if (count == 0) return RPCA_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (count + 255) / 256));
  gen_philox_words_kernel<<<grid, 256, 0, st>>>(out, count, ctr[0], ctr[1], ctr[2], ctr[3], (uint32_t)key,
                                                (uint32_t)(key >> 32));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err_noctx(RPCA_ECUDA, cudaGetErrorString(e));
  return RPCA_OK;
}

}  // extern "C"
