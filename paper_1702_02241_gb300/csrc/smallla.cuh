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
// A pair is rotated while |a_p . a_q| > tol ||a_p|| ||a_q|| and |a_p . a_q| > noise (||a_p||^2 +
// ||a_q||^2).  tol must lie above the rounding level of the inner products (about rows * eps);
// noise (about rows * eps) stops pairs whose inner product is at the rounding level of the
// larger column -- a rotation cannot reduce it further, and without this test a column much
// smaller than its partner is rotated again in every sweep up to max_sweeps.
// `flag` is one shared int.  Works in T = float or double.
template <typename T>
__device__ int cta_jacobi_svd(T* A, int rows, int cols, int lda, T* V, int ldv, T* sig, int* flag, int max_sweeps,
                              T tol, T noise = T(0)) {
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
        if (ga != T(0) && fabs(ga) > tol * sqrt(al * be) && fabs(ga) > noise * (al + be)) {
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

// 1 / sqrt(s) for s > 0: a float32 estimate refined by two Newton steps on y^-2 = s,
// y <- y (3 - s y^2) / 2, each of which squares the relative error (about 1e-7 -> 1e-14 ->
// rounding).  Avoids the float64 square root and divide, which are slow on this GPU.
RPCA_DEV double rsqrt_nr(double s) {
  if (!(s > 1e-30 && s < 1e30)) return 1.0 / sqrt(s);
  double y = (double)rsqrtf((float)s);
  y = y * (1.5 - 0.5 * s * y * y);
  y = y * (1.5 - 0.5 * s * y * y);
  return y;
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
  double rd[32];  // 1 / R_jj (one division per column; the float64 divide is slow on this GPU)
  for (int i = 0; i < n * n; ++i) R[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < j; ++i) {
      if ((bad >> i) & 1) continue;
      double s = G[i + j * n];
      for (int p = 0; p < i; ++p) s -= R[p + i * n] * R[p + j * n];
      R[i + j * n] = s * rd[i];
    }
    double s = G[j + j * n];
    for (int p = 0; p < j; ++p) s -= R[p + j * n] * R[p + j * n];
    const double floor_ = ref ? fmax(rel * ref[j], 1e-300) : floor_all;
    if (!(s > floor_)) {
      bad |= 1 << j;
      for (int p = 0; p < j; ++p) R[p + j * n] = 0.0;
      R[j + j * n] = 1.0;
      rd[j] = 1.0;
    } else {
      rd[j] = rsqrt_nr(s);
      R[j + j * n] = s * rd[j];
    }
  }
  for (int i = 0; i < n * n; ++i) Rinv[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    Rinv[j + j * n] = rd[j];
    for (int i = j - 1; i >= 0; --i) {
      double t = 0.0;
      for (int p = i + 1; p <= j; ++p) t += R[i + p * n] * Rinv[p + j * n];
      Rinv[i + j * n] = -t * rd[i];
    }
  }
  *mask = bad;
}

// chol_upper_inv_masked (same pivot rule and outputs) run by the whole CTA: right-looking,
// one pivot per step (thread 0), the row of R and the trailing update in parallel, then
// R^{-1} by back substitution with one thread per column.  n <= 32.  G, W, R, Rinv: shared
// n x n (ld n); W is scratch, G is left intact.  rd: shared n doubles; bad_s: shared int.
// All threads of the CTA must call it.  Returns the collapsed-column mask.
__device__ inline int cta_chol_masked(const double* G, int n, double rel, const double* ref, double* W, double* R,
                                      double* Rinv, double* rd, int* bad_s) {
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < n * n; e += nt) {
    W[e] = G[e];
    R[e] = 0.0;
    Rinv[e] = 0.0;
  }
  if (t == 0) *bad_s = 0;
  __syncthreads();
  double dmax = 0.0;
  for (int q = 0; q < n; ++q) dmax = fmax(dmax, W[q * (n + 1)]);
  const double floor_all = fmax(dmax, 1e-300) * rel;
  for (int k = 0; k < n; ++k) {
    if (t == 0) {
      const double s = W[k * (n + 1)];
      const double fl = ref ? fmax(rel * ref[k], 1e-300) : floor_all;
      if (!(s > fl)) {
        *bad_s |= 1 << k;
        rd[k] = 1.0;
        R[k * (n + 1)] = 1.0;
      } else {
        rd[k] = rsqrt_nr(s);
        R[k * (n + 1)] = s * rd[k];
      }
    }
    __syncthreads();
    const bool badk = (*bad_s >> k) & 1;
    for (int j = k + 1 + t; j < n; j += nt) R[k + n * j] = badk ? 0.0 : W[k + n * j] * rd[k];
    __syncthreads();
    if (!badk) {
      for (int e = t; e < n * n; e += nt) {
        const int i = e % n, j = e / n;
        if (i > k && j >= i) W[e] -= R[k + n * i] * R[k + n * j];
      }
    }
    __syncthreads();
  }
  const int bad = *bad_s;
  for (int e = t; e < n * n; e += nt) {  // collapsed columns: no coupling above the diagonal
    const int i = e % n, j = e / n;
    if (i < j && ((bad >> j) & 1)) R[e] = 0.0;
  }
  __syncthreads();
  for (int j = t; j < n; j += nt) {
    Rinv[j * (n + 1)] = rd[j];
    for (int i = j - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int p = i + 1; p <= j; ++p) acc += R[i + n * p] * Rinv[p + n * j];
      Rinv[i + n * j] = -acc * rd[i];
    }
  }
  __syncthreads();
  return bad;
}

}  // namespace rpca
