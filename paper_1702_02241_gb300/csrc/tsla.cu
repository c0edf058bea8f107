// Tall-skinny Gram and multiply kernels (certificate, Lanczos re-orthogonalisation, sketch).
#include <algorithm>

#include "common.cuh"
#include "tsla.h"

namespace rpca {

constexpr int TS_TR = 32;      // rows per shared-memory tile
constexpr int TS_PAD = 33;     // padded column stride of the A tile (bank-conflict free)
constexpr int TS_MAXIT = 3;    // output strips per thread: p * round_up(q, 4) <= 4 * 3 * 256

// Partial Gram products A^T B of one block's rows: each thread owns strips of four outputs
// (row i of C, columns 4jq..4jq+3), reads A's column i from a padded column-major tile and
// the four B values as one broadcast float4 from a row-major tile.  Sums in float32 over a
// 32-row tile, float64 across tiles; part[block][i + j p].
__global__ void __launch_bounds__(256) ts_gram_kernel(const float* A, int64_t lda, int p, const float* B,
                                                      int64_t ldb, int q, int64_t rows, double* part) {
  extern __shared__ __align__(16) float tile[];
  const int qp = (q + 3) & ~3, nq4 = qp >> 2;
  float* As = tile;
  float* Bs = tile + ((TS_PAD * p + 3) & ~3);
  const int nitem = p * nq4;
  double acc[TS_MAXIT][4];
#pragma unroll
  for (int s = 0; s < TS_MAXIT; ++s)
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[s][t] = 0.0;
  for (int64_t t0 = (int64_t)blockIdx.x * TS_TR; t0 < rows; t0 += (int64_t)gridDim.x * TS_TR) {
    for (int idx = threadIdx.x; idx < TS_TR * p; idx += blockDim.x) {
      const int r = idx % TS_TR, c = idx / TS_TR;
      const int64_t row = t0 + r;
      As[r + c * TS_PAD] = row < rows ? A[row + (int64_t)c * lda] : 0.f;
    }
    for (int idx = threadIdx.x; idx < TS_TR * qp; idx += blockDim.x) {
      const int r = idx % TS_TR, c = idx / TS_TR;
      const int64_t row = t0 + r;
      Bs[r * qp + c] = (row < rows && c < q) ? B[row + (int64_t)c * ldb] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < TS_MAXIT; ++s) {
      const int o = threadIdx.x + s * blockDim.x;
      if (o < nitem) {
        const int i = o % p, jq = o / p;
        const float* ai = As + i * TS_PAD;
        const float* bj = Bs + 4 * jq;
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll 8
        for (int r = 0; r < TS_TR; ++r) {
          const float a = ai[r];
          const float4 b4 = *reinterpret_cast<const float4*>(bj + r * qp);
          c0 = fmaf(a, b4.x, c0);
          c1 = fmaf(a, b4.y, c1);
          c2 = fmaf(a, b4.z, c2);
          c3 = fmaf(a, b4.w, c3);
        }
        acc[s][0] += (double)c0;
        acc[s][1] += (double)c1;
        acc[s][2] += (double)c2;
        acc[s][3] += (double)c3;
      }
    }
    __syncthreads();
  }
  const int64_t nout = (int64_t)p * q;
#pragma unroll
  for (int s = 0; s < TS_MAXIT; ++s) {
    const int o = threadIdx.x + s * blockDim.x;
    if (o < nitem) {
      const int i = o % p, jq = o / p;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = 4 * jq + t;
        if (j < q) part[(int64_t)blockIdx.x * nout + i + (int64_t)j * p] = acc[s][t];
      }
    }
  }
}

// C[o] = sum over the partial blocks of part[b][o]: one warp per output, lanes striding
// over the blocks, then a fixed shuffle tree (deterministic).
__global__ void __launch_bounds__(256) ts_gram_reduce_kernel(const double* part, int nblocks, int nout, double* C) {
  const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (o >= nout) return;
  double t = 0.0;
  for (int b = lane; b < nblocks; b += 32) t += part[(int64_t)b * nout + o];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if (lane == 0) C[o] = t;
}

// The 8 x 8 case (a Lanczos block against itself or another block): each thread keeps
// the 64 products of its rows in registers (float32 over at most TS_ROWS8 rows), a warp
// reduce-scatter leaves two sums per lane, and the block's warps are added in float64 in a
// fixed order.  No shared-memory staging: the loads of a row are coalesced across threads.
constexpr int TS_ROWS8 = 16;
__global__ void __launch_bounds__(256) ts_gram8_kernel(const float* A, int64_t lda, const float* B, int64_t ldb,
                                                       int64_t rows, double* part) {
  __shared__ double ws[8][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[64];
#pragma unroll
  for (int t = 0; t < 64; ++t) acc[t] = 0.f;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    float a[8], b[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      a[i] = A[row + (int64_t)i * lda];
      b[i] = B[row + (int64_t)i * ldb];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i + 8 * j] = fmaf(a[i], b[j], acc[i + 8 * j]);
  }
  int base = 0;
  ReduceScatter<64, 16>::run(acc, lane, base);
  ws[w][base] = (double)acc[0];
  ws[w][base + 1] = (double)acc[1];
  __syncthreads();
  if (threadIdx.x < 64) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += ws[q][threadIdx.x];
    part[(int64_t)blockIdx.x * 64 + threadIdx.x] = t;
  }
}

// A^T B for q = 8 and any p (projection of a block against a basis): the block owns a range
// of rb rows; warp w takes the column groups g = w, w + 8, ... of four columns of A and, per
// group, accumulates the 4 x 8 products of its rows in registers (float32 over at most rb /
// 32 rows per lane), then a warp reduce-scatter leaves one sum per lane.  A is read once; the
// block's rows of B are re-read from L1 for each group.
__global__ void __launch_bounds__(256) ts_gram_q8_kernel(const float* A, int64_t lda, int p, const float* B,
                                                         int64_t ldb, int64_t rows, int rb, double* part) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * rb;
  const int64_t r1 = r0 + rb < rows ? r0 + rb : rows;
  const int ng = (p + 3) >> 2;
  double* out = part + (int64_t)blockIdx.x * p * 8;
  for (int g = w; g < ng; g += 8) {
    float acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.f;
    const int c0 = 4 * g;
    for (int64_t row = r0 + lane; row < r1; row += 32) {
      float a[4], b[8];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) a[ii] = c0 + ii < p ? A[row + (int64_t)(c0 + ii) * lda] : 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = B[row + (int64_t)j * ldb];
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) acc[ii + 4 * j] = fmaf(a[ii], b[j], acc[ii + 4 * j]);
    }
    int base = 0;
    ReduceScatter<32, 16>::run(acc, lane, base);
    const int ii = base & 3, j = base >> 2;
    if (c0 + ii < p) out[(c0 + ii) + (int64_t)j * p] = (double)acc[0];
  }
}

int ts_gram_partial(const float* A, int64_t lda, int p, const float* B, int64_t ldb, int q, int64_t rows,
                    const TsScratch& s, cudaStream_t st) {
  if (p < 1 || q < 1 || p * q > 2304 || p * ((q + 3) & ~3) > 4 * TS_MAXIT * 256 || rows < 1) return -1;
  if (q == 8 && p > 8) {
    // Rows per block: about two blocks per SM, a multiple of 32, at least 32.
    int64_t rb = (rows + s.grid - 1) / std::max(1, s.grid);
    rb = std::max<int64_t>(32, (rb + 31) / 32 * 32);
    const int64_t g = (rows + rb - 1) / rb;
    if ((size_t)g * p * 8 > s.part_n) return -1;
    ts_gram_q8_kernel<<<(int)g, 256, 0, st>>>(A, lda, p, B, ldb, rows, (int)rb, s.part);
    return cudaGetLastError() == cudaSuccess ? (int)g : -1;
  }
  if (p == 8 && q == 8) {
    int64_t g = std::max<int64_t>(s.grid, (rows + 256LL * TS_ROWS8 - 1) / (256LL * TS_ROWS8));
    g = std::min<int64_t>(g, (rows + 255) / 256);
    g = std::min<int64_t>(g, (int64_t)(s.part_n / 64));
    const int grid = (int)std::max<int64_t>(g, 1);
    ts_gram8_kernel<<<grid, 256, 0, st>>>(A, lda, B, ldb, rows, s.part);
    return cudaGetLastError() == cudaSuccess ? grid : -1;
  }
  int grid = (int)std::min<int64_t>((int64_t)s.grid, (rows + TS_TR - 1) / TS_TR);
  grid = std::max(grid, 1);
  if ((size_t)grid * p * q > s.part_n) return -1;
  const size_t smem = sizeof(float) * (((size_t)TS_PAD * p + 3) / 4 * 4 + (size_t)TS_TR * ((q + 3) & ~3));
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(ts_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
  }
  ts_gram_kernel<<<grid, 256, smem, st>>>(A, lda, p, B, ldb, q, rows, s.part);
  return cudaGetLastError() == cudaSuccess ? grid : -1;
}

cudaError_t ts_gram(const float* A, int64_t lda, int p, const float* B, int64_t ldb, int q, int64_t rows, double* C,
                    const TsScratch& s, cudaStream_t st) {
  const int nblk = ts_gram_partial(A, lda, p, B, ldb, q, rows, s, st);
  if (nblk < 0) return cudaErrorInvalidValue;
  const int nout = p * q;
  ts_gram_reduce_kernel<<<(nout + 7) / 8, 256, 0, st>>>(s.part, nblk, nout, C);
  return cudaGetLastError();
}

// Y = alpha A C + beta Y.  A block covers 32 rows with 8 column slices: thread (lane,
// slice) accumulates the products of row lane over the columns i = slice, slice + 8, ... of
// A (a coalesced 128-byte load per column), the slices are summed through shared memory in
// a fixed order, and each thread writes the outputs j = slice, slice + 8, ... of its row.
// Every read of a block's rows precedes its writes (Y may alias A when p == q).
template <int QMAX>
__global__ void __launch_bounds__(256) ts_mul_kernel(const float* A, int64_t lda, int p, const double* Cm, int ldc,
                                                     int q, float* Y, int64_t ldy, int64_t rows, float alpha,
                                                     float beta) {
  extern __shared__ float sm[];
  float* Cs = sm;                   // p x QMAX
  float* red = sm + p * QMAX;       // 8 slices x 32 rows x (QMAX + 1), padded against bank conflicts
  for (int idx = threadIdx.x; idx < p * QMAX; idx += blockDim.x) {
    const int i = idx / QMAX, j = idx - (idx / QMAX) * QMAX;
    Cs[idx] = j < q ? (float)Cm[i + (int64_t)j * ldc] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const int64_t row = (int64_t)blockIdx.x * 32 + lane;
  float acc[QMAX];
#pragma unroll
  for (int j = 0; j < QMAX; ++j) acc[j] = 0.f;
  if (row < rows) {
#pragma unroll 4
    for (int i = slice; i < p; i += 8) {
      const float a = A[row + (int64_t)i * lda];
      const float* ci = Cs + i * QMAX;
#pragma unroll
      for (int j = 0; j < QMAX; ++j) acc[j] = fmaf(a, ci[j], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < QMAX; ++j) red[(slice * 32 + lane) * (QMAX + 1) + j] = acc[j];
  __syncthreads();
  if (row < rows) {
    for (int j = slice; j < q; j += 8) {
      float t = 0.f;
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) t += red[(sl * 32 + lane) * (QMAX + 1) + j];
      float* y = Y + row + (int64_t)j * ldy;
      *y = beta == 0.f ? alpha * t : fmaf(alpha, t, beta * *y);
    }
  }
}

cudaError_t ts_mul(const float* A, int64_t lda, int p, const double* Cm, int ldc, int q, float* Y, int64_t ldy,
                   int64_t rows, float alpha, float beta, cudaStream_t st) {
  if (q < 1 || q > 32 || p < 1) return cudaErrorInvalidValue;
  const int64_t grid = (rows + 31) / 32;
  if (grid < 1) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  auto smem = [&](int qmax) { return sizeof(float) * ((size_t)p * qmax + 8 * 32 * (size_t)(qmax + 1)); };
  if (q <= 8) {
    ts_mul_kernel<8><<<(int)grid, 256, smem(8), st>>>(A, lda, p, Cm, ldc, q, Y, ldy, rows, alpha, beta);
  } else if (q <= 16) {
    ts_mul_kernel<16><<<(int)grid, 256, smem(16), st>>>(A, lda, p, Cm, ldc, q, Y, ldy, rows, alpha, beta);
  } else {
    if (smem(32) > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(ts_mul_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem(32));
      if (e != cudaSuccess) return e;
    }
    ts_mul_kernel<32><<<(int)grid, 256, smem(32), st>>>(A, lda, p, Cm, ldc, q, Y, ldy, rows, alpha, beta);
  }
  return cudaGetLastError();
}

}  // namespace rpca
