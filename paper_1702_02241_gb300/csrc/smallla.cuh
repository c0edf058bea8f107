// Small dense linear algebra run by one CTA (certificate and sketch): one-sided Jacobi SVD,
// Cholesky with inverse, and the tall-skinny kernels (Gram A^T B, A C products) they feed.
#pragma once
#include "common.cuh"

namespace rpca {

// Round-robin ("circle") schedule of ne players (ne even): pair k of round r.
RPCA_DEV void rr_pair(int r, int k, int ne, int& p, int& q) {
  if (k == 0) {
    p = ne - 1;
    q = r;
  } else {
    p = (r + k) % (ne - 1);
    q = (r - k + ne - 1) % (ne - 1);
  }
}

// One-sided Jacobi (Hestenes) SVD, executed by the whole CTA (blockDim multiple of 32).
// A: rows x cols column-major (lda), overwritten by U * diag(sig) (columns in input order).
// V: cols x cols (ldv), right singular vectors.  sig[j] = ||A_j||.  Returns the sweep count.
// `flag` is one shared int.  Works in T = float or double.
template <typename T>
__device__ int cta_jacobi_svd(T* A, int rows, int cols, int lda, T* V, int ldv, T* sig, int* flag, int max_sweeps,
                              T tol) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int idx = threadIdx.x; idx < cols * cols; idx += blockDim.x) {
    const int i = idx % cols, j = idx / cols;
    V[i + (size_t)j * ldv] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  const int ne = cols + (cols & 1);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < ne - 1; ++r) {
      for (int k = w; k < ne / 2; k += nw) {
        int p, q;
        rr_pair(r, k, ne, p, q);
        if (p >= cols || q >= cols) continue;
        T* ap = A + (size_t)p * lda;
        T* aq = A + (size_t)q * lda;
        T al = 0, be = 0, ga = 0;
        for (int i = lane; i < rows; i += 32) {
          const T x = ap[i], y = aq[i];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (ga != T(0) && fabs(ga) > tol * sqrt(al * be)) {
          const T zeta = (be - al) / (T(2) * ga);
          const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T cs = T(1) / sqrt(T(1) + t * t), sn = cs * t;
          for (int i = lane; i < rows; i += 32) {
            const T x = ap[i], y = aq[i];
            ap[i] = cs * x - sn * y;
            aq[i] = sn * x + cs * y;
          }
          T* vp = V + (size_t)p * ldv;
          T* vq = V + (size_t)q * ldv;
          for (int i = lane; i < cols; i += 32) {
            const T x = vp[i], y = vq[i];
            vp[i] = cs * x - sn * y;
            vq[i] = sn * x + cs * y;
          }
          if (lane == 0) *flag = 1;
        }
        __syncwarp();
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
  for (int j = threadIdx.x; j < cols; j += blockDim.x) {
    T s = 0;
    for (int i = 0; i < rows; ++i) s += A[i + (size_t)j * lda] * A[i + (size_t)j * lda];
    sig[j] = sqrt(s);
  }
  __syncthreads();
  return sweep;
}

// order[t] = index of the t-th largest of v[0..n) (ties by index); run by the CTA.
template <typename T>
__device__ void cta_sort_desc(const T* v, int n, int* order) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int rank = 0;
    for (int i = 0; i < n; ++i) rank += (v[i] > v[j]) || (v[i] == v[j] && i < j);
    order[rank] = j;
  }
  __syncthreads();
}

// Upper Cholesky G = R^T R of an n x n SPD matrix (column-major, ld n) with a relative
// pivot floor, and R^{-1}.  Single thread.  Returns the number of pivots that hit the floor.
__device__ inline int chol_upper_inv(const double* G, int n, double* R, double* Rinv) {
  double dmax = 0.0;
  for (int i = 0; i < n; ++i) dmax = fmax(dmax, G[i + i * n]);
  const double floor_ = fmax(dmax, 1e-300) * 1e-13;
  int bad = 0;
  for (int i = 0; i < n * n; ++i) R[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i <= j; ++i) {
      double s = G[i + j * n];
      for (int p = 0; p < i; ++p) s -= R[p + i * n] * R[p + j * n];
      if (i == j) {
        if (s < floor_) {
          s = floor_;
          ++bad;
        }
        R[j + j * n] = sqrt(s);
      } else {
        R[i + j * n] = s / R[i + i * n];
      }
    }
  }
  for (int i = 0; i < n * n; ++i) Rinv[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    Rinv[j + j * n] = 1.0 / R[j + j * n];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int p = i + 1; p <= j; ++p) s += R[i + p * n] * Rinv[p + j * n];
      Rinv[i + j * n] = -s / R[i + i * n];
    }
  }
  return bad;
}

// Upper Cholesky of the n x n Gram G (column-major) that tolerates collapsed columns: a
// pivot below `rel` * max diagonal marks column j in *mask and gets R_jj = 1 with no
// coupling (R_jk = 0), so that an all-zero column j stays zero and leaves the others alone.
// When ref is non-null the floor of column j is rel * ref[j] (e.g. its squared norm before
// a projection) instead of rel * max diagonal.
__device__ inline void chol_upper_inv_masked(const double* G, int n, double rel, double* R, double* Rinv, int* mask,
                                             const double* ref = nullptr) {
  double dmax = 0.0;
  for (int i = 0; i < n; ++i) dmax = fmax(dmax, G[i + i * n]);
  const double floor_all = fmax(dmax, 1e-300) * rel;
  int bad = 0;
  for (int i = 0; i < n * n; ++i) R[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < j; ++i) {
      if ((bad >> i) & 1) continue;
      double s = G[i + j * n];
      for (int p = 0; p < i; ++p) s -= R[p + i * n] * R[p + j * n];
      R[i + j * n] = s / R[i + i * n];
    }
    double s = G[j + j * n];
    for (int p = 0; p < j; ++p) s -= R[p + j * n] * R[p + j * n];
    const double floor_ = ref ? fmax(rel * ref[j], 1e-300) : floor_all;
    if (!(s > floor_)) {
      bad |= 1 << j;
      for (int p = 0; p < j; ++p) R[p + j * n] = 0.0;
      R[j + j * n] = 1.0;
    } else {
      R[j + j * n] = sqrt(s);
    }
  }
  for (int i = 0; i < n * n; ++i) Rinv[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    Rinv[j + j * n] = 1.0 / R[j + j * n];
    for (int i = j - 1; i >= 0; --i) {
      double t = 0.0;
      for (int p = i + 1; p <= j; ++p) t += R[i + p * n] * Rinv[p + j * n];
      Rinv[i + j * n] = -t / R[i + i * n];
    }
  }
  *mask = bad;
}

}  // namespace rpca
