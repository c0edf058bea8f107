// Small dense linear algebra run by one CTA (certificate and sketch): one-sided Jacobi SVD,
// Cholesky with inverse, and the tall-skinny kernels (Gram A^T B, A C products) they feed.
#pragma once
#include "common.cuh"

namespace rpca {

// Round-robin ("circle") schedule of ne players (ne even): pair k of round r (0 <= r < ne - 1,
// 0 <= k < ne / 2).  Conditional subtractions instead of a modulo by a runtime value.
RPCA_DEV void rr_pair(int r, int k, int ne, int& p, int& q) {
  if (k == 0) {
    p = ne - 1;
    q = r;
  } else {
    const int m = ne - 1;
    p = r + k;
    if (p >= m) p -= m;
    q = r - k;
    if (q < 0) q += m;
  }
}

// 2^-e for x in [2^e, 2^(e+1)) when x is positive, normal and finite (from the exponent
// field; exact), else 0.
RPCA_DEV double pow2_inv_scale(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  if (!(x > 0.0) || e == 0 || e >= 0x7fe) return 0.0;
  return __longlong_as_double((long long)(2046 - e) << 52);
}
RPCA_DEV float pow2_inv_scale(float x) {
  const int e = (int)((__float_as_uint(x) >> 23) & 0xff);
  if (!(x > 0.f) || e == 0 || e >= 0xfe) return 0.f;
  return __uint_as_float((unsigned)(254 - e) << 23);
}

// Rotation (cs, sn) of one Jacobi step on columns with squared norms al, be and inner
// product ga.  The angle is formed in float32 with fast operations (its accuracy only affects
// how far the step reduces a_p . a_q) from (be - al) and ga scaled by the same power of two,
// so that tiny or huge columns neither underflow nor overflow float32 (a flushed ga would
// make the angle 0/0); then (cs, sn) is renormalised in T by one Newton step on
// 1/sqrt(cs^2 + sn^2), so that the rotation is orthogonal to T's rounding (float64 square
// roots and divides cost hundreds of cycles each on this GPU).  Returns false, and leaves
// the pair alone, when the scaled inner product is below float32 resolution or not finite.
template <typename T>
RPCA_DEV bool jacobi_rotation(T al, T be, T ga, T& cs, T& sn) {
  const T sc = pow2_inv_scale(al + be);
  const float g = (float)(ga * sc);
  if (!(fabsf(g) >= 1e-30f && fabsf(g) <= 2.f)) return false;
  // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) from the approximate reciprocal and
  // reciprocal square root (each a single instruction; the IEEE-rounded forms are call
  // sequences, and a round of the CTA form is bound by instruction issue).  Above 2^32 the
  // square root is |zeta| in float32 (and 1 + zeta^2 would overflow further up).
  const float zeta = __fdividef((float)((be - al) * sc), 2.f * g);
  const float az = fabsf(zeta);
  const float z2 = fmaf(zeta, zeta, 1.f);
  const float root = az < 4.0e9f ? z2 * rsqrtf(z2) : az;
  const float tf = copysignf(__fdividef(1.f, az + root), zeta);
  const float csf = rsqrtf(fmaf(tf, tf, 1.f));
  cs = (T)csf;
  sn = (T)(csf * tf);
  const T corr = T(1.5) - T(0.5) * (cs * cs + sn * sn);
  cs *= corr;
  sn *= corr;
  return true;
}

// One-sided Jacobi (Hestenes) SVD, executed by a group of gnw warps starting at warp gw0 that
// synchronise on named barrier `bar` (0: the whole CTA, __syncthreads), or by the whole CTA
// (cta_jacobi_svd).
// A: rows x cols column-major (lda), overwritten by U * diag(sig) (columns in input order).
// V: cols x cols (ldv), right singular vectors.  sig[j] = ||A_j||.  Returns the sweep count.
// A pair is rotated while |a_p . a_q| > tol ||a_p|| ||a_q|| and |a_p . a_q| > noise (||a_p||^2 +
// ||a_q||^2).  tol must lie above the rounding level of the inner products (about rows * eps);
// noise (about rows * eps) stops pairs whose inner product is at the rounding level of the
// larger column -- a rotation cannot reduce it further, and without this test a column much
// smaller than its partner is rotated again in every sweep up to max_sweeps.
// `flag` is one shared int.  Works in T = float or double.
template <typename T>
__device__ int group_jacobi_svd(T* A, int rows, int cols, int lda, T* V, int ldv, T* sig, int* flag, int max_sweeps,
                                T tol, T noise, int gw0, int gnw, int bar) {
  const int lane = threadIdx.x & 31, w = (int)(threadIdx.x >> 5) - gw0, nw = gnw;
  const int gt = (int)threadIdx.x - gw0 * 32, gn = gnw * 32;  // thread index and count in the group
  auto sync = [&]() {
    if (bar == 0) __syncthreads();
    else named_bar(bar, gn);
  };
  // Butterfly width: the lanes that hold data (rows of A) or apply the rotation (rows of A,
  // rows of V = cols) must all get the sums, so the tree spans max(rows, cols) lanes.
  const int nact = rows > cols ? rows : cols;
  int top = 16;
  while (top > 1 && top >= nact) top >>= 1;
  if (nact > 32) top = 16;
  for (int idx = gt; idx < cols * cols; idx += gn) {
    const int i = idx % cols, j = idx / cols;
    V[i + (size_t)j * ldv] = (i == j) ? T(1) : T(0);
  }
  sync();
  const int ne = cols + (cols & 1);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (gt == 0) *flag = 0;
    sync();
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
        // Lanes at or beyond `rows` hold zeros: the tree spans the first 2 * top lanes.
        for (int o = top; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        T cs, sn;
        if (ga != T(0) && ga * ga > tol * tol * (al * be) && fabs(ga) > noise * (al + be) &&
            jacobi_rotation(al, be, ga, cs, sn)) {
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
      sync();
    }
    if (*flag == 0) break;
    sync();
  }
  for (int j = gt; j < cols; j += gn) {
    T s = 0;
    for (int i = 0; i < rows; ++i) s += A[i + (size_t)j * lda] * A[i + (size_t)j * lda];
    sig[j] = sqrt(s);
  }
  sync();
  return sweep;
}

// The whole CTA.
template <typename T>
__device__ int cta_jacobi_svd(T* A, int rows, int cols, int lda, T* V, int ldv, T* sig, int* flag, int max_sweeps,
                              T tol, T noise = T(0)) {
  return group_jacobi_svd<T>(A, rows, cols, lda, V, ldv, sig, flag, max_sweeps, tol, noise, 0, (int)(blockDim.x >> 5),
                             0);
}

// One-sided Jacobi (Hestenes) SVD of a small matrix by one warp: cols <= CMAX <= 32,
// rows <= RMAX.  Meant for float32 (the Ritz values): its inner products are per-lane
// chains over RMAX rows, which in float64 (64-cycle dependent adds here) lose to the CTA form.
// Lane j holds column j of A and of V in registers; round r of the round-robin ("circle")
// schedule pairs lane j with (2r - j) mod (ne - 1) (ne - 1 with r), the pair exchanges columns
// with shuffles, both lanes form the same rotation from the same three inner products, and
// each updates its own column.  No barriers: a sweep is ne - 1 rounds of shuffles and FMAs.
// Rotation test and angle as in cta_jacobi_svd.  A (rows x cols, lda) is overwritten by
// U diag(sig) in shared or global memory, V (cols x cols, ldv) receives the right singular
// vectors, sig[j] = ||A_j||.  Call from all 32 lanes of one warp; returns the sweep count.
template <typename T, int RMAX, int CMAX>
__device__ int warp_jacobi_svd(T* A, int rows, int cols, int lda, T* V, int ldv, T* sig, int max_sweeps, T tol,
                               T noise) {
  static_assert(CMAX <= 32, "one lane per column");
  const int lane = threadIdx.x & 31;
  const bool mine = lane < cols;
  T a[RMAX], v[CMAX];
#pragma unroll
  for (int i = 0; i < RMAX; ++i) a[i] = (mine && i < rows) ? A[i + (size_t)lane * lda] : T(0);
#pragma unroll
  for (int i = 0; i < CMAX; ++i) v[i] = (i == lane) ? T(1) : T(0);
  const int ne = cols + (cols & 1);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    bool rotated = false;
    for (int r = 0; r < ne - 1; ++r) {
      int partner;
      if (lane == ne - 1) {
        partner = r;
      } else if (lane == r) {
        partner = ne - 1;
      } else {  // (2 r - lane) mod (ne - 1), by conditional subtractions
        const int m = ne - 1;
        partner = 2 * r - lane + 2 * m;
        if (partner >= 2 * m) partner -= 2 * m;
        if (partner >= m) partner -= m;
      }
      const bool act = mine && partner < cols && lane < ne;
      const int src = act ? partner : lane;
      T b[RMAX];
#pragma unroll
      for (int i = 0; i < RMAX; ++i) b[i] = __shfl_sync(0xffffffffu, a[i], src);
      const bool low = lane < partner;  // the lower index plays p, the higher q
      // Inner products in four interleaved partial sums (shorter dependent chains).
      T al4[4] = {0, 0, 0, 0}, be4[4] = {0, 0, 0, 0}, ga4[4] = {0, 0, 0, 0};
#pragma unroll
      for (int i = 0; i < RMAX; ++i) {
        const T ap = low ? a[i] : b[i], aq = low ? b[i] : a[i];
        al4[i & 3] += ap * ap;
        be4[i & 3] += aq * aq;
        ga4[i & 3] += ap * aq;
      }
      const T al = (al4[0] + al4[1]) + (al4[2] + al4[3]);
      const T be = (be4[0] + be4[1]) + (be4[2] + be4[3]);
      const T ga = (ga4[0] + ga4[1]) + (ga4[2] + ga4[3]);
      T cs = T(1), sn = T(0);
      const bool rot = act && ga != T(0) && ga * ga > tol * tol * (al * be) && fabs(ga) > noise * (al + be) &&
                       jacobi_rotation(al, be, ga, cs, sn);
      if (!rot) {
        cs = T(1);
        sn = T(0);
      }
      rotated |= rot;
      // p' = cs p - sn q,  q' = sn p + cs q.
      const T ca = cs, cb = low ? -sn : sn;
#pragma unroll
      for (int i = 0; i < RMAX; ++i) a[i] = ca * a[i] + cb * b[i];
#pragma unroll
      for (int i = 0; i < CMAX; ++i) {
        const T w = __shfl_sync(0xffffffffu, v[i], src);
        v[i] = ca * v[i] + cb * w;
      }
    }
    if (!__any_sync(0xffffffffu, rotated)) break;
  }
  if (mine) {
    T s2 = 0;
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
      s2 += a[i] * a[i];
      if (i < rows) A[i + (size_t)lane * lda] = a[i];
    }
    sig[lane] = sqrt(s2);
#pragma unroll
    for (int i = 0; i < CMAX; ++i)
      if (i < cols) V[i + (size_t)lane * ldv] = v[i];
  }
  __syncwarp();
  return sweep;
}

// order[t] = index of the t-th largest of v[0..n) (ties by index, NaNs last by index); run by
// the CTA.  The ranks come from a strict total order on (value, index), so `order` is a
// permutation of 0..n-1 whatever the values are: callers index memory with it.
template <typename T>
__device__ void cta_sort_desc(const T* v, int n, int* order) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const T vj = v[j];
    const bool nj = isnan(vj);
    int rank = 0;
    for (int i = 0; i < n; ++i) {
      const T vi = v[i];
      rank += isnan(vi) ? (nj && i < j) : (nj || vi > vj || (vi == vj && i < j));
    }
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
