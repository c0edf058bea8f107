// Context-aware wrappers of the tall-skinny helpers: they also count the launch.
#pragma once
#include "ctx.h"
#include "tsla.h"

namespace rpca {

inline cudaError_t ts_gram_c(rpca_ctx* c, const float* A, int64_t lda, int p, const float* B, int64_t ldb, int q,
                             int64_t rows, double* C, const TsScratch& s, cudaStream_t st) {
  count_launches(c, 2);
  return ts_gram(A, lda, p, B, ldb, q, rows, C, s, st);
}
inline int ts_gram_partial_c(rpca_ctx* c, const float* A, int64_t lda, int p, const float* B, int64_t ldb, int q,
                             int64_t rows, const TsScratch& s, cudaStream_t st) {
  count_launches(c, 1);
  return ts_gram_partial(A, lda, p, B, ldb, q, rows, s, st);
}
inline cudaError_t ts_mul_c(rpca_ctx* c, const float* A, int64_t lda, int p, const double* Cm, int ldc, int q,
                            float* Y, int64_t ldy, int64_t rows, float alpha, float beta, cudaStream_t st) {
  count_launches(c, 1);
  return ts_mul(A, lda, p, Cm, ldc, q, Y, ldy, rows, alpha, beta, st);
}

}  // namespace rpca
