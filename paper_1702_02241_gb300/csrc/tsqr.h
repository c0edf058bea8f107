// TSQR (Sec. 6.1): the QR factorisation of a tall-skinny float32 matrix by a reduction tree of
// small Householder QRs, one CTA per tree node.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpca {

constexpr int TQ_LMAX = 32;            // columns
constexpr int TQ_SMEM_FLOATS = 24576;  // shared-memory budget of one node (96 KB: two CTAs per SM)
constexpr int TQ_MAXLEV = 24;

struct TsqrPlan {
  int64_t rows = 0;
  int l = 0;
  int b = 0;     // leaf block rows; the last leaf also takes the remainder (< 2b rows)
  int P = 0;     // leaves
  int G = 0;     // fan-in of the reduction levels (stacked R's per node)
  int nlev = 0;  // reduction levels above the leaves
  int cnt[TQ_MAXLEV + 1] = {};  // nodes per level (cnt[0] = P, cnt[nlev] = 1)
  size_t offQt = 0;             // leaf Q's, rows x l column-major (ld rows)
  size_t offR[TQ_MAXLEV + 1] = {}, offQn[TQ_MAXLEV + 1] = {}, offE[TQ_MAXLEV + 1] = {};
  size_t ws_floats = 0;
  size_t smem_leaf = 0, smem_node = 0;
  int launches = 0;
};

// Plan for rows x l (1 <= l <= TQ_LMAX, rows >= l) on a GPU with nsm SMs.
TsqrPlan tsqr_plan(int64_t rows, int l, int nsm);

// Q R = A with A = sum over t < npart of the matrices A + t * part_stride (each rows x l,
// column-major, ld lda: the partial sums of a split product are added on load).  R: l x l
// upper triangular with a non-negative diagonal, column-major (device, may be null).
// Q: rows x l column-major with ld ldq, or, when rowmajor, row i at Q + i * ldq with ldq >= l
// entries of which those past l are zeroed.  ws: plan.ws_floats floats of device memory.
// Returns cudaSuccess or the first launch error.
cudaError_t tsqr_run(const TsqrPlan& p, const float* A, int64_t lda, int npart, int64_t part_stride, float* Q,
                     int64_t ldq, bool rowmajor, float* R, float* ws, cudaStream_t st);

// Allows the dynamic shared memory the plan's kernels need (once per process).
bool tsqr_allow_smem();

}  // namespace rpca
