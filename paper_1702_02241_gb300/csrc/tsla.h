// Tall-skinny helpers: Gram products A^T B (float64 result) and A C products.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpca {

struct TsScratch {
  double* part = nullptr;  // block partials
  size_t part_n = 0;
  unsigned int* counter = nullptr;
  int grid = 0;
};

// C (p x q, column-major, ld p, device float64) = A^T B, A rows x p (lda), B rows x q (ldb).
// p * q <= 2304.  Deterministic (fixed-order reduction).
cudaError_t ts_gram(const float* A, int64_t lda, int p, const float* B, int64_t ldb, int q, int64_t rows, double* C,
                    const TsScratch& s, cudaStream_t st);

// Y (rows x q, ldy) = alpha * A (rows x p, lda) * Cm (p x q, ld ldc, float64) + beta * Y.
// q <= 32; Y may alias A when p == q.
cudaError_t ts_mul(const float* A, int64_t lda, int p, const double* Cm, int ldc, int q, float* Y, int64_t ldy,
                   int64_t rows, float alpha, float beta, cudaStream_t st);

}  // namespace rpca
