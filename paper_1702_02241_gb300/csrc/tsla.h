// Tall-skinny helpers: Gram products A^T B (float64 result) and A C products.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpca {

struct TsScratch {
  double* part = nullptr;  // block partials
  size_t part_n = 0;
  int grid = 0;
};

// C (p x q, column-major, ld p, device float64) = A^T B, A rows x p (lda), B rows x q (ldb).
// p * q <= 2304 and p * round_up(q, 4) <= 3072.  Deterministic (fixed-order reduction).
// Two launches: block partials into s.part, then their sum into C.
cudaError_t ts_gram(const float* A, int64_t lda, int p, const float* B, int64_t ldb, int q, int64_t rows, double* C,
                    const TsScratch& s, cudaStream_t st);

// The first half of ts_gram: block partials of A^T B into s.part (p * q doubles per block,
// column-major within a block).  Returns the number of blocks written, or -1 on bad
// arguments or a launch error.
int ts_gram_partial(const float* A, int64_t lda, int p, const float* B, int64_t ldb, int q, int64_t rows,
                    const TsScratch& s, cudaStream_t st);

#ifdef __CUDACC__
// Sum of the ts_gram_partial blocks, run by the whole CTA.  When nout is small the threads
// form blockDim / nout groups, each summing every G-th block of one output, and the groups
// are added in a fixed order (many independent loads in flight instead of one serial chain);
// otherwise each thread sums one output over all blocks.  scratch: blockDim.x shared doubles.
__device__ inline void ts_reduce_partials_cta(const double* part, int nblocks, int nout, double* out,
                                              double* scratch) {
  const int t = threadIdx.x, groups = (int)blockDim.x / nout;
  if (groups >= 2) {
    const int o = t % nout, g = t / nout;
    double acc = 0.0;
    if (g < groups) {
#pragma unroll 16
      for (int b = g; b < nblocks; b += groups) acc += part[(int64_t)b * nout + o];
    }
    scratch[t] = acc;
    __syncthreads();
    if (t < nout) {
      double s = 0.0;
      for (int q = 0; q < groups; ++q) s += scratch[q * nout + t];
      out[t] = s;
    }
  } else {
    for (int o = t; o < nout; o += blockDim.x) {
      double s = 0.0;
#pragma unroll 16
      for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * nout + o];
      out[o] = s;
    }
  }
}
#endif

// Y (rows x q, ldy) = alpha * A (rows x p, lda) * Cm (p x q, ld ldc, float64) + beta * Y.
// q <= 32; Y may alias A when p == q.
cudaError_t ts_mul(const float* A, int64_t lda, int p, const double* Cm, int ldc, int q, float* Y, int64_t ldy,
                   int64_t rows, float alpha, float beta, cudaStream_t st);

}  // namespace rpca
