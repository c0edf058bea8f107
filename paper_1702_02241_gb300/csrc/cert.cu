// Computable convergence certificate of Sec. 3.4 on the device.
//
// At L = U V^T the certificate is ||E||_F for an element E = lam_L Z + D of the
// subdifferential of lam_L ||L||_* + phi(L), D = P_Omega(clip(U V^T - X)) (Sec. 3.2):
//   ||E||_F^2 = t1 + t2 + t3 + t4,
//   t1 = ||lam_L I + U1^T D V1||^2,  t2 = ||U1^T D V2||^2,  t3 = ||U2^T D V1||^2,
//   t4 = sum_i (sigma_i(P_U1perp D P_V1perp) - lam_L)_+^2     (projection onto the ball)
// with U1, V1 the singular vectors of L for its r nonzero singular values.
//
// Steps (all on the device, float64 unless noted):
//  1. one pass over X: F(U, V) and the raw products DV = D V (m x k), DtU = D^T U (n x k);
//  2. Gram matrices U^T U, V^T V, U^T (D V);
//  3. one CTA: eigen-decompositions of the two Grams give orthonormal bases of range(U),
//     range(V) (the thin-QR route of the footnote in Sec. 3.4, with rank-deficient factors
//     allowed), the SVD of the small core M gives sigma(L), U1 = U T_U, V1 = V T_V, r, and
//     B = U1^T D V1 = T_U^T (U^T D V) T_V, t1 = ||lam_L I + B||^2;
//  4. t3 = ||D V1 - U1 B||^2 and t2 = ||D^T U1 - V1 B^T||^2 row by row (the same numbers as
//     the paper's ||U1^T D||^2 - ||U1^T D V1||^2, without its cancellation near optimum);
//  5. t4: block Golub-Kahan-Lanczos (block 8, full re-orthogonalisation) on
//     P_U1perp D P_V1perp, whose products D Q and D^T P each take one pass over X through
//     the fused kernel in apply mode; after every block step from the second, the Ritz values
//     of the projected matrix T = P^T A Q (float32 Householder bidiagonalisation, then
//     bisection on Sturm counts for sigma_1 and the values above lam_L); stops when the
//     leading Ritz value and t4 settle.  The leading Ritz vectors (rank increase) are formed
//     on request by a one-sided Jacobi SVD of the same T.
// Also F_bound = min(F(0), best F seen) and the gap bound cert * (||L||_F + F_bound/lam_L)
// (Sec. 3.4, "Bounding the distance to the feasible set") plus F_trunc, the cost of the
// directions of L that step 3 moves to the complement block (2 lam_L times their singular
// values), and trunc_rel = F_trunc / (lam_L ||L||_F + F_bound).
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cooperative_groups.h>

#include "common.cuh"
#include "ctx.h"
#include "smallla.cuh"
#include "tsla_ctx.h"

namespace rpca {

constexpr int CERT_KMAX = 16;
constexpr int LZ_B = 8;       // Lanczos block size
constexpr int LZ_SMAX = 32;   // maximum block steps (Krylov dimension 256)
constexpr int LZ_TMAX = LZ_B * LZ_SMAX;
constexpr int RITZ_TOPQ = 16;  // leading Ritz pairs kept for the rank increase
constexpr double RANK_TAU = 1e-8;  // numerical rank of L: sigma_i > RANK_TAU * sigma_1
constexpr double DROP_TAU = 1e-3;  // tiny-and-inactive directions go to the complement
constexpr double NEG_TAU = 1e-12;  // lam_L sigma_i <= NEG_TAU F: numerically zero direction

struct CertState {
  double AUU[CERT_KMAX * CERT_KMAX], AVV[CERT_KMAX * CERT_KMAX], MUDV[CERT_KMAX * CERT_KMAX];
  double TU[CERT_KMAX * CERT_KMAX], TV[CERT_KMAX * CERT_KMAX];  // k x r, ld KMAX
  double P2[CERT_KMAX * CERT_KMAX], P3[CERT_KMAX * CERT_KMAX];  // T_U B, T_V B^T
  double sig[CERT_KMAX];
  int r;
  double t1, t2, t3, t4, normL, sigma1;
  double sig_drop;  // sum of the singular values of L moved to the complement block
  double G[(CERT_KMAX + LZ_TMAX) * LZ_B];    // Gram scratch (p x q)
  double G2[(CERT_KMAX + LZ_TMAX + LZ_B) * LZ_B];  // projection Gram [B | Y]^T Y
  double R[LZ_B * LZ_B], Rinv[LZ_B * LZ_B];
  int bad_mask;  // columns whose Cholesky pivot collapsed in the last block QR
  double n0[LZ_B];  // squared column norms before the last projection
  double t4_prev, s1_prev;
  int converged;
  double resid[2];
  // Leading Ritz pairs of the last spectral evaluation (their coefficients in the Lanczos
  // bases P[:, 0:d], Q[:, 0:d] are in CertBuffers::ritz): values, count, d.
  double ritz_s[RITZ_TOPQ];
  int ritz_q, ritz_d;
};

struct CertBuffers {
  int Kp = 0;
  float* DV = nullptr;   // m x k
  float* DtU = nullptr;  // n x k
  float* U1 = nullptr;   // m x KMAX
  float* V1 = nullptr;   // n x KMAX
  float* P = nullptr;    // m x TMAX
  float* Q = nullptr;    // n x (TMAX + B)
  float* W = nullptr;    // m x B
  float* Z = nullptr;    // n x B
  float* Up = nullptr;   // m x Kp (zero-padded U)
  float* Vp = nullptr;   // n x Kp
  float* zm = nullptr;   // m x max(B, k) zeros
  float* zn = nullptr;   // n x max(B, k) zeros
  double* T = nullptr;   // TMAX x TMAX
  double* ritz = nullptr;  // leading Ritz pairs' coefficients: [2][RITZ_TOPQ][LZ_TMAX] (P side, Q side)
  float* Tw = nullptr;   // TMAX x TMAX float32 working copy for the Ritz SVD
  float* Tv = nullptr;   // TMAX x TMAX right vectors
  float* Wraw = nullptr; // m x B, A Q_j before orthogonalisation
  CertState* st = nullptr;
  CertState* host = nullptr;
  double* blk = nullptr;
  unsigned int* counter = nullptr;
  TsScratch ts;
  bool have_F0 = false;
  double last_F = 0.0;  // F at the point of the last evaluation (its first four steps)
};

// ---------------------------------------------------------------------------------------------
// Step 3: one CTA of 256 threads.
__global__ void __launch_bounds__(256) cert_small_kernel(CertState* st, int k, double lam_L, const double* Fp) {
  __shared__ double Au[CERT_KMAX * CERT_KMAX], Wu[CERT_KMAX * CERT_KMAX], su[CERT_KMAX];
  __shared__ double Av[CERT_KMAX * CERT_KMAX], Wv[CERT_KMAX * CERT_KMAX], sv[CERT_KMAX];
  __shared__ double M[CERT_KMAX * CERT_KMAX], Vm[CERT_KMAX * CERT_KMAX], sm[CERT_KMAX];
  __shared__ double Ru[CERT_KMAX * CERT_KMAX], Rv[CERT_KMAX * CERT_KMAX];
  __shared__ int ordu[CERT_KMAX], ordv[CERT_KMAX], ordm[CERT_KMAX];
  __shared__ int flag, flag2, ku, kv;
  const int t = threadIdx.x;
  for (int i = t; i < k * k; i += blockDim.x) {
    const int a = i % k, b = i / k;
    Au[i] = st->AUU[a + b * CERT_KMAX];
    Av[i] = st->AVV[a + b * CERT_KMAX];
  }
  __syncthreads();
  // Symmetric PSD Grams: the one-sided Jacobi SVD is their eigen-decomposition; the two run
  // at once on the two halves of the CTA (named barriers 1 and 2).
  {
    const int hw = (int)(blockDim.x >> 6);
    if ((int)(t >> 5) < hw)
      group_jacobi_svd<double>(Au, k, k, k, Wu, k, su, &flag, 60, 1e-13, 4.0 * k * 1.1e-16, 0, hw, 1);
    else
      group_jacobi_svd<double>(Av, k, k, k, Wv, k, sv, &flag2, 60, 1e-13, 4.0 * k * 1.1e-16, hw, hw, 2);
  }
  __syncthreads();
  cta_sort_desc<double>(su, k, ordu);
  cta_sort_desc<double>(sv, k, ordv);
  if (t == 0) {
    // Eigen-directions kept for the range bases (float64 floor on the Gram eigenvalues).
    ku = 0;
    kv = 0;
    for (int i = 0; i < k; ++i) ku += su[ordu[i]] > 1e-14 * su[ordu[0]] && su[ordu[i]] > 0.0;
    for (int i = 0; i < k; ++i) kv += sv[ordv[i]] > 1e-14 * sv[ordv[0]] && sv[ordv[i]] > 0.0;
  }
  __syncthreads();
  // R_U = Lambda_U^{1/2} W_U^T (ku x k) and R_V likewise; M = R_U R_V^T (ku x kv).
  for (int i = t; i < ku * k; i += blockDim.x) {
    const int a = i % ku, b = i / ku;
    Ru[a + b * CERT_KMAX] = sqrt(su[ordu[a]]) * Wu[b + ordu[a] * k];
  }
  for (int i = t; i < kv * k; i += blockDim.x) {
    const int a = i % kv, b = i / kv;
    Rv[a + b * CERT_KMAX] = sqrt(sv[ordv[a]]) * Wv[b + ordv[a] * k];
  }
  __syncthreads();
  for (int i = t; i < ku * kv; i += blockDim.x) {
    const int a = i % ku, b = i / ku;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s += Ru[a + l * CERT_KMAX] * Rv[b + l * CERT_KMAX];
    M[a + b * ku] = s;
  }
  __syncthreads();
  int r = 0;
  if (ku > 0 && kv > 0) {
    cta_jacobi_svd<double>(M, ku, kv, ku, Vm, kv, sm, &flag, 60, 1e-13, 4.0 * ku * 1.1e-16);
    cta_sort_desc<double>(sm, kv, ordm);
    const double s1 = sm[ordm[0]];
    for (int i = 0; i < std::min(ku, kv); ++i) r += (sm[ordm[i]] > RANK_TAU * s1 && s1 > 0.0);
  }
  __syncthreads();
  // T_U = W_U Lambda_U^{-1/2} U_M[:, :r], U_M[:, c] = M_c / sigma_c; T_V = W_V Lambda_V^{-1/2} V_M[:, :r].
  for (int i = t; i < k * r; i += blockDim.x) {
    const int l = i % k, c = i / k;
    const int jc = ordm[c];
    double su_ = 0.0, sv_ = 0.0;
    for (int a = 0; a < ku; ++a) su_ += Wu[l + ordu[a] * k] / sqrt(su[ordu[a]]) * (M[a + jc * ku] / sm[jc]);
    for (int b = 0; b < kv; ++b) sv_ += Wv[l + ordv[b] * k] / sqrt(sv[ordv[b]]) * Vm[b + jc * kv];
    st->TU[l + c * CERT_KMAX] = su_;
    st->TV[l + c * CERT_KMAX] = sv_;
  }
  __syncthreads();
  // B = T_U^T (U^T D V) T_V (r x r), t1, P2 = T_U B, P3 = T_V B^T.
  __shared__ double Bs[CERT_KMAX * CERT_KMAX], Tmp[CERT_KMAX * CERT_KMAX];
  for (int i = t; i < k * r; i += blockDim.x) {  // Tmp = (U^T D V) T_V   (k x r)
    const int a = i % k, c = i / k;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s += st->MUDV[a + l * CERT_KMAX] * st->TV[l + c * CERT_KMAX];
    Tmp[a + c * CERT_KMAX] = s;
  }
  __syncthreads();
  for (int i = t; i < r * r; i += blockDim.x) {
    const int a = i % r, c = i / r;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s += st->TU[l + a * CERT_KMAX] * Tmp[l + c * CERT_KMAX];
    Bs[a + c * CERT_KMAX] = s;
  }
  __syncthreads();
  // A direction that is both tiny (sigma_i <= DROP_TAU sigma_1) and inactive
  // (|lam_L + u_i^T D v_i| > lam_L / 2) is moved to the complement block: it is rounding
  // residue of a factor column that the nuclear penalty drives to zero, and the certificate
  // is then that of L with it truncated.  So is a direction whose nuclear-norm term is
  // negligible against the objective (lam_L sigma_i <= NEG_TAU F), which the relative test
  // cannot see when all of L is at the float32 rounding floor (a solution L = 0).
  // Their singular values are summed: the truncation costs at most 2 lam_L sum sigma_i in the
  // optimality gap (subgradient inequalities of phi at L and of the nuclear norm at the
  // truncated point), which the host reports beside the certificate.
  __shared__ int keep[CERT_KMAX], rk;
  if (t == 0) {
    rk = 0;
    double drop = 0.0;
    const double Fv = *Fp;
    for (int c = 0; c < r; ++c) {
      const bool tiny = sm[ordm[c]] <= DROP_TAU * sm[ordm[0]];
      const bool inactive = fabs(lam_L + Bs[c + c * CERT_KMAX]) > 0.5 * lam_L;
      const bool negligible = lam_L * sm[ordm[c]] <= NEG_TAU * Fv;
      if (!(tiny && inactive) && !negligible) keep[rk++] = c;
      else drop += sm[ordm[c]];
    }
    st->sig_drop = drop;
    if (rk < r) {
      for (int q = 0; q < rk; ++q) {
        for (int l = 0; l < k; ++l) {
          st->TU[l + q * CERT_KMAX] = st->TU[l + keep[q] * CERT_KMAX];
          st->TV[l + q * CERT_KMAX] = st->TV[l + keep[q] * CERT_KMAX];
        }
      }
      for (int q = 0; q < rk; ++q)
        for (int q2 = 0; q2 < rk; ++q2) Tmp[q + q2 * CERT_KMAX] = Bs[keep[q] + keep[q2] * CERT_KMAX];
      for (int q = 0; q < rk; ++q)
        for (int q2 = 0; q2 < rk; ++q2) Bs[q + q2 * CERT_KMAX] = Tmp[q + q2 * CERT_KMAX];
    }
  }
  __syncthreads();
  r = rk;
  for (int i = t; i < k * r; i += blockDim.x) {
    const int l = i % k, c = i / k;
    double s2 = 0.0, s3 = 0.0;
    for (int a = 0; a < r; ++a) {
      s2 += st->TU[l + a * CERT_KMAX] * Bs[a + c * CERT_KMAX];
      s3 += st->TV[l + a * CERT_KMAX] * Bs[c + a * CERT_KMAX];
    }
    st->P2[l + c * CERT_KMAX] = s2;
    st->P3[l + c * CERT_KMAX] = s3;
  }
  if (t == 0) {
    double t1 = 0.0;
    for (int a = 0; a < r; ++a)
      for (int c = 0; c < r; ++c) {
        const double e = Bs[a + c * CERT_KMAX] + (a == c ? lam_L : 0.0);
        t1 += e * e;
      }
    double nl = 0.0;
    for (int i = 0; i < std::min(ku, kv); ++i) nl += sm[ordm[i]] * sm[ordm[i]];
    st->t1 = t1;
    st->r = r;
    st->normL = sqrt(nl);
    for (int i = 0; i < CERT_KMAX; ++i) st->sig[i] = i < std::min(ku, kv) ? sm[ordm[i]] : 0.0;
  }
}

// Step 4: sum over rows of ||A_i T - C_i P||^2 (A, C rows x k; T, P k x r), float64.
__global__ void __launch_bounds__(256) cert_resid_kernel(const float* A, const float* Cm, int64_t rows, int k,
                                                         const CertState* st, int which, double* blk,
                                                         unsigned int* counter, CertState* out) {
  __shared__ double Ts[CERT_KMAX * CERT_KMAX], Ps[CERT_KMAX * CERT_KMAX];
  __shared__ double scr[32];
  __shared__ bool is_last;
  const int r = st->r;
  const double* T = which == 0 ? st->TV : st->TU;
  const double* P = which == 0 ? st->P2 : st->P3;
  for (int i = threadIdx.x; i < CERT_KMAX * CERT_KMAX; i += blockDim.x) {
    Ts[i] = T[i];
    Ps[i] = P[i];
  }
  __syncthreads();
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    double a[CERT_KMAX], cc[CERT_KMAX];
    for (int l = 0; l < k; ++l) {
      a[l] = A[i + (int64_t)l * rows];
      cc[l] = Cm[i + (int64_t)l * rows];
    }
    for (int c = 0; c < r; ++c) {
      double e = 0.0;
      for (int l = 0; l < k; ++l) e += a[l] * Ts[l + c * CERT_KMAX] - cc[l] * Ps[l + c * CERT_KMAX];
      acc += e * e;
    }
  }
  acc = block_sum_d(acc, scr);
  if (threadIdx.x == 0) {
    blk[blockIdx.x] = acc;
    __threadfence();
    is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&blk[b]);
  s = block_sum_d(s, scr);
  if (threadIdx.x == 0) {
    out->resid[which] = s;
    *counter = 0u;
  }
}

// Factors the Gram st->G of an 8-column block (masked Cholesky) and records the columns whose
// pivot collapsed (that column is numerically in the span of the earlier ones and of the bases
// projected out).  st->G was summed over the row blocks by ts_gram's multi-block reduction (one
// CTA summing every block's float64 partials was most of this step: float64 runs at a few
// operations per clock per SM on this GPU).
constexpr int CHOL_THREADS = 128;
__global__ void __launch_bounds__(CHOL_THREADS) cert_gram_chol_kernel(CertState* st, double rel, int per_column) {
  __shared__ double G[LZ_B * LZ_B], W[LZ_B * LZ_B], R[LZ_B * LZ_B], Ri[LZ_B * LZ_B], rd[LZ_B];
  __shared__ int bad;
  if (threadIdx.x < LZ_B * LZ_B) G[threadIdx.x] = st->G[threadIdx.x];
  __syncthreads();
  const int mask = cta_chol_masked(G, LZ_B, rel, per_column ? st->n0 : nullptr, W, R, Ri, rd, &bad);
  if (threadIdx.x < LZ_B * LZ_B) {
    st->R[threadIdx.x] = R[threadIdx.x];
    st->Rinv[threadIdx.x] = Ri[threadIdx.x];
  }
  if (threadIdx.x == 0) st->bad_mask = mask;
}

// Records the squared column norms (the diagonal of the Gram st->G).
__global__ void cert_gram_norms_kernel(CertState* st) {
  if (threadIdx.x < LZ_B) st->n0[threadIdx.x] = st->G[threadIdx.x * (LZ_B + 1)];
}

// Columns flagged in st->bad_mask are set to zero (the Krylov space is exhausted there).
__global__ void cert_zero_cols_kernel(float* Y, int64_t rows, const CertState* st) {
  const int mask = st->bad_mask;
  if (mask == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * LZ_B; i += (int64_t)gridDim.x * blockDim.x)
    if ((mask >> (int)(i / rows)) & 1) Y[i] = 0.f;
}

// Collapsed columns of Y (rows x 8) are replaced by fresh Gaussian columns.
__global__ void cert_refill_kernel(float* Y, int64_t rows, const CertState* st, uint64_t seed) {
  const int mask = st->bad_mask;
  if (mask == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * LZ_B; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / rows);
    if ((mask >> c) & 1) {
      uint64_t z = seed * 0x9E3779B97F4A7C15ull + (uint64_t)i;
      z += 0x9e3779b97f4a7c15ull;
      z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
      z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
      z ^= z >> 31;
      Y[i] = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
  }
}

// T[0:p, col:col+8] = st->G (p x 8): the block P^T (A Q_j) of the projected matrix.
__global__ void cert_store_T_kernel(const CertState* st, double* T, int p, int col) {
  for (int i = threadIdx.x; i < p * LZ_B; i += blockDim.x) {
    const int a = i % p, b = i / p;
    T[a + (int64_t)(col + b) * LZ_TMAX] = st->G[i];
  }
}

// Start of a spectral step: T = 0 and the Lanczos loop's stopping state cleared.
__global__ void cert_zero_T_kernel(double* T, CertState* st) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < LZ_TMAX * LZ_TMAX; i += gridDim.x * blockDim.x) T[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->t4_prev = -1.0;
    st->s1_prev = -1.0;
    st->converged = 0;
    st->ritz_d = 0;
    st->ritz_q = 0;
  }
}

__global__ void cert_reset_kernel(CertState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->bad_mask = 0;
  st->t4_prev = -1.0;
  st->s1_prev = -1.0;
  st->converged = 0;
  st->t4 = 0.0;
  st->sigma1 = 0.0;
  st->ritz_d = 0;
  st->ritz_q = 0;
}

// Stopping tests of the Lanczos loop from the Ritz values of T[0:d, 0:d]: s1 the largest, t4
// the sum of (sigma - lam_L)^2 over those above lam_L, `above` their count (one thread).
__device__ void ritz_update(CertState* st, double s1, double t4, int above, int d, double lam_L, int final_step) {
  // Settled: sigma_1 and t4 stopped moving, and the Ritz values above lam_L leave at least
  // two blocks of the Krylov space to spare (otherwise more of them may be missing).
  const bool settled = st->s1_prev >= 0.0 && fabs(s1 - st->s1_prev) <= 1e-5 * s1 &&
                       fabs(t4 - st->t4_prev) <= 1e-4 * t4 + 1e-12 * lam_L * lam_L && above + 2 * LZ_B <= d;
  // When the leading Ritz value has settled (to 1e-3) at half of lam_L or less, no singular
  // value of the projected residual reaches lam_L: t4 = 0.
  const bool clear = st->s1_prev >= 0.0 && fabs(s1 - st->s1_prev) <= 1e-3 * s1 && s1 <= 0.5 * lam_L;
  st->converged = settled || clear || final_step;
  st->t4_prev = t4;
  st->s1_prev = s1;
  st->t4 = t4;
  st->sigma1 = s1;
}

// Ritz values of T[0:d, 0:d] (float32 one-sided Jacobi in global memory) -> t4 estimate,
// sigma_1, and whether both have settled since the previous check.
// Ritz values of the projected matrix, sorted: t4 and the stopping tests of the Lanczos loop.
// Called by the whole CTA (the sort is CTA-wide); thread 0 updates the state.
__device__ void ritz_finish(CertState* st, const float* s, int* ord, int d, double lam_L, int final_step,
                            const float* A, const float* V, double* ritz) {
  cta_sort_desc<float>(s, d, ord);
  {  // the leading pairs: left vector A[:, j] / s_j (A holds U diag(s)), right vector V[:, j]
    const int q = d < RITZ_TOPQ ? d : RITZ_TOPQ;
    for (int e = threadIdx.x; e < q * d; e += blockDim.x) {
      const int t = e / d, c = e - t * d;
      const int j = ord[t];
      const float sj = s[j];
      ritz[t * LZ_TMAX + c] = sj > 0.f ? (double)A[c + (size_t)j * d] / (double)sj : 0.0;
      ritz[(RITZ_TOPQ + t) * LZ_TMAX + c] = (double)V[c + (size_t)j * d];
    }
    for (int t = threadIdx.x; t < q; t += blockDim.x) st->ritz_s[t] = s[ord[t]];
    if (threadIdx.x == 0) {
      st->ritz_d = d;
      st->ritz_q = q;
    }
  }
  if (threadIdx.x == 0) {
    double t4 = 0.0;
    for (int i = 0; i < d; ++i) {
      const double e = (double)s[i] - lam_L;
      if (e > 0.0) t4 += e * e;
    }
    int above = 0;
    for (int i = 0; i < d; ++i) above += (double)s[i] > lam_L;
    ritz_update(st, s[ord[0]], t4, above, d, lam_L, final_step);
  }
}

// Rotation threshold of the Ritz SVDs: above the float32 rounding of the column inner
// products (about d * eps relative); below it every sweep would rotate every pair until the
// sweep limit.
__device__ inline float ritz_tol(int d) { return fmaxf(1e-6f, 4.0f * d * 1.2e-7f); }
__device__ inline float ritz_noise(int d) { return 2.0f * d * 6e-8f; }

// d <= 32: one warp, the matrix in registers (warp_jacobi_svd).
__global__ void __launch_bounds__(32) cert_ritz_warp_kernel(CertState* st, const double* T, int d, double lam_L,
                                                            int final_step, double* ritz) {
  __shared__ float A[32 * 32], V[32 * 32], s[32];
  __shared__ int ord[32];
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) {
    const int a = i % d, b = i / d;
    A[i] = (float)T[a + (int64_t)b * LZ_TMAX];
  }
  __syncwarp();
  warp_jacobi_svd<float, 32, 32>(A, d, d, d, V, d, s, 40, ritz_tol(d), ritz_noise(d));
  ritz_finish(st, s, ord, d, lam_L, final_step, A, V, ritz);
}

// Larger d: the CTA form, in shared memory up to d = 96, else in global memory.
// Projected matrices up to RITZ_SMEM_D on a side are rotated in shared memory (A and V, 200 KB
// at 160); larger ones in global memory (measured 3.7 ms for d in [128, 160) there).
constexpr int RITZ_SMEM_D = 160;
__global__ void __launch_bounds__(1024) cert_ritz_kernel(CertState* st, const double* T, float* Ag, float* Vg, int d,
                                                          double lam_L, int final_step, double* ritz) {
  __shared__ float s[LZ_TMAX];
  __shared__ int ord[LZ_TMAX];
  __shared__ int flag;
  extern __shared__ float dyn[];
  const bool in_smem = d <= RITZ_SMEM_D;
  float* A = in_smem ? dyn : Ag;
  float* V = in_smem ? dyn + d * d : Vg;
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) {
    const int a = i % d, b = i / d;
    A[i] = (float)T[a + (int64_t)b * LZ_TMAX];
  }
  __syncthreads();
  cta_jacobi_svd<float>(A, d, d, d, V, d, s, &flag, 40, ritz_tol(d), ritz_noise(d));
  ritz_finish(st, s, ord, d, lam_L, final_step, A, V, ritz);
}

// ---- Ritz values alone (the stopping tests after every Lanczos step) ----------------------
// T (d x d, d <= RITZV_DMAX) is reduced to upper bidiagonal form B = H^T T G by Householder
// reflections from the left (columns) and the right (rows) in float32 in shared memory (B has
// T's singular values); those of B are located by bisection on Sturm counts of its
// Golub-Kahan form, the symmetric tridiagonal of order 2d with zero diagonal and off-diagonal
// (a_0, b_0, a_1, b_1, ..., a_{d-1}), whose eigenvalues are +-sigma_i.  Only sigma_1 and the
// values above lam_L are located; the Ritz vectors are formed on request (ritz_vectors).
constexpr int RITZV_DMAX = 128;
constexpr int RITZV_THREADS = 128;

// Number of singular values of the bidiagonal (a, b) that are >= s (s > 0): 2d minus the
// negative pivots of the LDL^T factorisation of (Golub-Kahan form - s I).  Pivots smaller
// than pivmin in magnitude are replaced by -pivmin (Kahan's safeguard).
__device__ int gk_count_ge(const float* a, const float* b, int d, float s, float pivmin) {
  float q = -s;
  int neg = 1;
  for (int i = 0; i < 2 * d - 1; ++i) {
    const float e = (i & 1) ? b[i >> 1] : a[i >> 1];
    if (fabsf(q) < pivmin) q = -pivmin;
    q = -s - __fdividef(e * e, q);
    neg += q < 0.f;
  }
  return 2 * d - neg;
}

// The (idx+1)-th largest singular value of the bidiagonal, bracketed in (lo, hi): 32-point
// multisection by one warp (every lane counts at its own shift), until the bracket is a few
// float32 units wide.
__device__ float gk_kth_largest(const float* a, const float* b, int d, int idx, float lo, float hi, float pivmin) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < 12 && hi - lo > 2.5e-7f * hi; ++round) {
    const float w = (hi - lo) * (1.f / 33.f);
    const float s = lo + w * (float)(lane + 1);
    const unsigned msk = __ballot_sync(0xffffffffu, gk_count_ge(a, b, d, s, pivmin) >= idx + 1);
    const int top = 32 - __clz(msk);  // shifts 1..top are at or below the value
    const float nlo = top > 0 ? lo + w * (float)top : lo;
    hi = top < 32 ? lo + w * (float)(top + 1) : hi;
    lo = nlo;
  }
  return 0.5f * (lo + hi);
}

__global__ void __launch_bounds__(RITZV_THREADS) cert_ritz_values_kernel(CertState* st, const double* T, int d,
                                                                         double lam_L, int final_step) {
  extern __shared__ float A[];  // d x d, column-major, ld = d + 1 (odd: a row or a column
                                // read by consecutive threads hits distinct banks)
  __shared__ float ad[RITZV_DMAX], bd[RITZV_DMAX], sv[RITZV_DMAX];
  __shared__ float hh[4];  // alpha, v_0, beta of the current reflection, and a skip flag
  __shared__ int n_above;
  __shared__ float s1_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int ld = d + 1;
  for (int i = tid; i < d * d; i += blockDim.x) {
    const int r = i % d, c = i / d;
    A[r + c * ld] = (float)T[r + (int64_t)c * LZ_TMAX];
  }
  __syncthreads();
  // Reflection data from a vector x of length h with squared norm nrm2 and first entry x0:
  // alpha = -sign(x0) ||x||, v = x - alpha e_1, beta = 2 / ||v||^2 (warp 0, lane 0).
  auto reflector = [&](float nrm2, float x0, float* out_alpha) {
    if (nrm2 > 0.f) {
      const float alpha = -copysignf(sqrtf(nrm2), x0);
      const float v0 = x0 - alpha;
      hh[0] = alpha;
      hh[1] = v0;
      hh[2] = 2.f / (nrm2 - x0 * x0 + v0 * v0);
      hh[3] = 0.f;
      *out_alpha = alpha;
    } else {
      hh[3] = 1.f;
      *out_alpha = 0.f;
    }
  };
  for (int k = 0; k < d; ++k) {
    // Left reflection I - beta v v^T on rows k.. (v = A[k:, k] - alpha e_1, v_0 in hh[1]):
    // thread j forms w_j = beta v^T A[k:, j] and updates its column j > k.
    if (warp == 0) {
      float part = 0.f;
      for (int i = k + lane; i < d; i += 32) part += A[i + k * ld] * A[i + k * ld];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) reflector(part, A[k + k * ld], &ad[k]);
    }
    __syncthreads();
    if (hh[3] == 0.f) {
      const float v0 = hh[1], beta = hh[2];
      for (int j = k + 1 + tid; j < d; j += blockDim.x) {
        float* col = A + j * ld;
        const float* vk = A + k * ld;
        float w = v0 * col[k];
        for (int i = k + 1; i < d; ++i) w = fmaf(vk[i], col[i], w);
        w *= beta;
        col[k] -= v0 * w;
        for (int i = k + 1; i < d; ++i) col[i] = fmaf(-vk[i], w, col[i]);
      }
    }
    __syncthreads();
    if (k + 1 == d) break;
    // Right reflection on columns k+1.. (v = A[k, k+1:] - alpha e_1): thread i forms
    // w_i = beta A[i, k+1:] v and updates its row i > k.
    if (warp == 0) {
      float part = 0.f;
      for (int j = k + 1 + lane; j < d; j += 32) part += A[k + j * ld] * A[k + j * ld];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) reflector(part, A[k + (k + 1) * ld], &bd[k]);
    }
    __syncthreads();
    if (hh[3] == 0.f) {
      const float v0 = hh[1], beta = hh[2];
      for (int i = k + 1 + tid; i < d; i += blockDim.x) {
        float w = A[i + (k + 1) * ld] * v0;
        for (int j = k + 2; j < d; ++j) w = fmaf(A[i + j * ld], A[k + j * ld], w);
        w *= beta;
        A[i + (k + 1) * ld] -= w * v0;
        for (int j = k + 2; j < d; ++j) A[i + j * ld] = fmaf(-w, A[k + j * ld], A[i + j * ld]);
      }
    }
    __syncthreads();
  }
  if (tid == 0) bd[d - 1] = 0.f;
  __syncthreads();
  // Bracket: every eigenvalue of the Golub-Kahan form lies within its largest absolute row
  // sum (Gershgorin); pivmin scales with its largest squared entry.
  float hi = 0.f, e2 = 0.f;
  for (int i = 0; i < d; ++i) {
    const float bl = i > 0 ? fabsf(bd[i - 1]) : 0.f;
    hi = fmaxf(hi, fmaxf(fabsf(ad[i]) + bl, fabsf(ad[i]) + fabsf(bd[i])));
    e2 = fmaxf(e2, fmaxf(ad[i] * ad[i], bd[i] * bd[i]));
  }
  hi = hi * 1.0001f + 1e-30f;
  const float pivmin = 1e-30f * fmaxf(1.f, e2);
  if (tid == 0) n_above = (float)lam_L < hi ? gk_count_ge(ad, bd, d, (float)lam_L, pivmin) : 0;
  __syncthreads();
  const int na = n_above;
  // The values above lam_L (one warp each), then sigma_1 if none is.
  for (int idx = warp; idx < na; idx += nw) {
    const float v = gk_kth_largest(ad, bd, d, idx, 0.f, hi, pivmin);
    if (lane == 0) sv[idx] = v;
  }
  if (na == 0 && warp == 0) {
    const float v = gk_kth_largest(ad, bd, d, 0, 0.f, hi, pivmin);
    if (lane == 0) s1_sh = v;
  }
  __syncthreads();
  if (tid == 0) {
    double t4 = 0.0;
    for (int i = 0; i < na; ++i) {
      const double e = (double)sv[i] - lam_L;
      if (e > 0.0) t4 += e * e;
    }
    const double s1 = na > 0 ? (double)sv[0] : (double)s1_sh;
    ritz_update(st, s1, t4, na, d, lam_L, final_step);
    st->ritz_d = d;
    st->ritz_q = 0;  // Ritz vectors of this T not formed yet
  }
}

__global__ void pad_copy_kernel(const float* src, int64_t rows, int k, float* dst, int kp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * kp; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / rows;
    dst[i] = c < k ? src[i] : 0.f;
  }
}

void fill_normal(float* out, int64_t count, uint64_t seed, float scale, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
void free_cert(rpca_ctx* c) {
  CertBuffers* b = c->cert;
  if (!b) return;
  dev_free(b->DV);
  dev_free(b->T);
  dev_free(b->ritz);
  dev_free(b->st);
  dev_free(b->blk);
  dev_free(b->counter);
  dev_free(b->ts.part);
  host_pinned_free(b->host);
  delete b;
  c->cert = nullptr;
}

#define CERT_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(c, e_, #call); \
  } while (0)

static rpca_status ensure_cert(rpca_ctx* c) {
  if (c->cert) return RPCA_OK;
  CertBuffers* b = new CertBuffers();
  c->cert = b;
  const int64_t m = c->m, n = c->n, k = c->k;
  b->Kp = k <= 8 ? 8 : 16;
  const int zc = std::max<int>(LZ_B, (int)k);
  const int64_t nf = m * k + n * k + m * (CERT_KMAX + LZ_TMAX) + n * (CERT_KMAX + LZ_TMAX + LZ_B) + m * LZ_B +
                     n * LZ_B + m * b->Kp + n * b->Kp + m * zc + n * zc + m * LZ_B + 2 * LZ_TMAX * LZ_TMAX;
  CERT_CUDA(dev_alloc(&b->DV, sizeof(float) * nf));
  float* p = b->DV;
  p += m * k;
  b->DtU = p;
  p += n * k;
  // [U1 | P_0 | P_1 | ...] and [V1 | Q_0 | Q_1 | ...] are contiguous: U1 (r columns) sits
  // right before P_0, so one projection covers both bases.
  b->P = p + m * CERT_KMAX;
  p += m * (CERT_KMAX + LZ_TMAX);
  b->Q = p + n * CERT_KMAX;
  p += n * (CERT_KMAX + LZ_TMAX + LZ_B);
  b->W = p;
  p += m * LZ_B;
  b->Z = p;
  p += n * LZ_B;
  b->Up = p;
  p += m * b->Kp;
  b->Vp = p;
  p += n * b->Kp;
  b->zm = p;
  p += m * zc;
  b->zn = p;
  p += n * zc;
  b->Wraw = p;
  p += m * LZ_B;
  b->Tw = p;
  p += LZ_TMAX * LZ_TMAX;
  b->Tv = p;
  CERT_CUDA(cudaMemsetAsync(b->zm, 0, sizeof(float) * (m + n) * zc, c->stream));
  CERT_CUDA(dev_alloc(&b->T, sizeof(double) * LZ_TMAX * LZ_TMAX));
  CERT_CUDA(dev_alloc(&b->ritz, sizeof(double) * 2 * RITZ_TOPQ * LZ_TMAX));
  CERT_CUDA(dev_alloc(&b->st, sizeof(CertState)));
  CERT_CUDA(cudaMemsetAsync(b->st, 0, sizeof(CertState), c->stream));
  CERT_CUDA(host_pinned_alloc(&b->host, sizeof(CertState)));
  CERT_CUDA(dev_alloc(&b->blk, sizeof(double) * 4 * c->nsm));
  CERT_CUDA(dev_alloc(&b->counter, 64));
  CERT_CUDA(cudaMemsetAsync(b->counter, 0, 64, c->stream));
  b->ts.grid = 2 * c->nsm;
  b->ts.part_n = (size_t)b->ts.grid * 2304;
  CERT_CUDA(dev_alloc(&b->ts.part, sizeof(double) * b->ts.part_n));
  return RPCA_OK;
}

// Sums the partials of [B | Y]^T Y ((p + 8) x 8, one warp per output) into st->G2 and records
// the squared column norms of Y (the diagonal of its trailing 8 x 8 block) in st->n0.
__global__ void __launch_bounds__(256) cert_proj_reduce_kernel(const double* part, int nblk, int p, CertState* st) {
  const int ld = p + LZ_B, nout = ld * LZ_B;
  const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (o >= nout) return;
  double t = 0.0;
  for (int b = lane; b < nblk; b += 32) t += part[(int64_t)b * nout + o];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if (lane == 0) {
    st->G2[o] = t;
    const int i = o % ld, j = o / ld;
    if (i - p == j) st->n0[j] = t;
  }
}

// Y (rows x 8) <- Y - B (B^T Y) for a basis B (rows x p, orthonormal columns).
static rpca_status project_out(rpca_ctx* c, const float* Bm, int p, float* Y, int64_t rows) {
  CertBuffers* b = c->cert;
  if (p == 0) return RPCA_OK;
  CERT_CUDA(ts_gram_c(c, Bm, rows, p, Y, rows, LZ_B, rows, b->st->G2, b->ts, c->stream));
  CERT_CUDA(ts_mul_c(c, Bm, rows, p, b->st->G2, p, LZ_B, Y, rows, rows, -1.f, 1.f, c->stream));
  return RPCA_OK;
}

// Gram of Y and its masked Cholesky.  per_column: a pivot below rel * (squared norm of
// that column recorded by record_norms) marks it collapsed; otherwise the floor is
// rel * (largest squared column norm).
static rpca_status gram_chol(rpca_ctx* c, float* Y, int64_t rows, double rel, int per_column) {
  CertBuffers* b = c->cert;
  CERT_CUDA(ts_gram_c(c, Y, rows, LZ_B, Y, rows, LZ_B, rows, b->st->G, b->ts, c->stream));
  cert_gram_chol_kernel<<<1, CHOL_THREADS, 0, c->stream>>>(b->st, rel, per_column);
  count_launches(c, 1);
  CERT_CUDA(cudaGetLastError());
  return RPCA_OK;
}

static rpca_status record_norms(rpca_ctx* c, float* Y, int64_t rows) {
  CertBuffers* b = c->cert;
  CERT_CUDA(ts_gram_c(c, Y, rows, LZ_B, Y, rows, LZ_B, rows, b->st->G, b->ts, c->stream));
  cert_gram_norms_kernel<<<1, 32, 0, c->stream>>>(b->st);
  count_launches(c, 1);
  CERT_CUDA(cudaGetLastError());
  return RPCA_OK;
}

// Two passes of classical Gram-Schmidt against the basis B (rows x p, orthonormal columns).
static rpca_status project_twice(rpca_ctx* c, float* Y, int64_t rows, const float* Bm, int p) {
  rpca_status s;
  for (int pass = 0; pass < 2; ++pass)
    if ((s = project_out(c, Bm, p, Y, rows)) != RPCA_OK) return s;
  return RPCA_OK;
}

static rpca_status normalise(rpca_ctx* c, float* Y, int64_t rows) {
  rpca_status s = gram_chol(c, Y, rows, 1e-12, 0);
  if (s != RPCA_OK) return s;
  CERT_CUDA(ts_mul_c(c, Y, rows, LZ_B, c->cert->st->Rinv, LZ_B, LZ_B, Y, rows, rows, 1.f, 0.f, c->stream));
  return RPCA_OK;
}

// ---------------------------------------------------------------------------------------------
// The orthonormalisation of orth_block in one launch: a thread-block cluster of up to OC_MAXC
// CTAs, each owning a contiguous range of rows of Y (kept in its shared memory for the whole
// launch, written back at the end).  A Gram product ([B | Y]^T Y, B^T Y or Y^T Y) is formed per
// CTA with one warp per column of the left factor, each lane summing its rows in float32 with
// sixteen loads in flight, the lanes added in float-float; the CTAs' partials are exchanged
// through distributed shared memory and summed by every CTA in rank order (every CTA holds the
// same Gram matrix), and each CTA updates its own rows, one thread per row.  The steps, pivot
// rules and collapse handling are those of orth_block; nothing is read back by the host.  Used
// while the rows fit OC_MAXC x OC_ROWS and p <= OC_PMAX.
constexpr int OC_THREADS = 512;
constexpr int OC_WARPS = OC_THREADS / 32;
constexpr int OC_MAXC = 8;                           // CTAs per cluster (the portable limit)
constexpr int OC_ROWS = 2560;                        // rows per CTA at most
constexpr int OC_PMAX = CERT_KMAX + LZ_B * LZ_SMAX;  // basis columns at most
constexpr int OC_NA = OC_PMAX + LZ_B;                // Gram rows at most ([B | Y])
constexpr int OC_UNROLL = 16;                        // loads in flight per lane

struct OrthArgs {
  const float* B;    // rows x p basis (orthonormal columns), ld rows
  int p;
  float* Y;          // rows x LZ_B block, ld rows: in place
  const float* src;  // Y starts as a copy of src (rows x LZ_B, ld rows; may be Y)
  int64_t rows;
  int rows_per;      // rows per CTA
  uint64_t seed;     // refill of collapsed columns
};

struct OcSmem {
  double* G;     // [OC_NA * LZ_B] the summed Gram, G[i * LZ_B + c]
  float2* part;  // [2][OC_NA * LZ_B] this CTA's Gram partials (float-float)
  float* Gf;     // [OC_PMAX * LZ_B] G rows < p as float32 for the update
  float* Ys;     // [OC_ROWS][LZ_B] this CTA's rows of Y, row-major
};
inline size_t oc_smem_bytes() {
  return sizeof(double) * OC_NA * LZ_B + sizeof(float2) * 2 * OC_NA * LZ_B + sizeof(float) * OC_PMAX * LZ_B +
         sizeof(float) * (size_t)OC_ROWS * LZ_B;
}
__device__ inline OcSmem oc_layout(unsigned char* base) {
  OcSmem L;
  L.G = reinterpret_cast<double*>(base);
  L.part = reinterpret_cast<float2*>(L.G + OC_NA * LZ_B);
  L.Gf = reinterpret_cast<float*>(L.part + 2 * OC_NA * LZ_B);
  L.Ys = L.Gf + OC_PMAX * LZ_B;
  return L;
}

// Warp reduce-scatter of eight float-float sums: afterwards lane l with (l & 3) == 0 holds the
// warp's total of sum number l >> 2.
__device__ inline ff2 oc_warp_sum8(ff2 v[8], int lane) {
  // xor 16: keep four of the eight (upper half of the lanes the upper four).
  const bool h16 = lane & 16;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const ff2 send = h16 ? v[q] : v[q + 4];
    const ff2 recv = ff_shfl_xor(send, 16);
    v[q] = ff_add(h16 ? v[q + 4] : v[q], recv);
  }
  const bool h8 = lane & 8;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const ff2 send = h8 ? v[q] : v[q + 2];
    const ff2 recv = ff_shfl_xor(send, 8);
    v[q] = ff_add(h8 ? v[q + 2] : v[q], recv);
  }
  const bool h4 = lane & 4;
  {
    const ff2 send = h4 ? v[0] : v[1];
    const ff2 recv = ff_shfl_xor(send, 4);
    v[0] = ff_add(h4 ? v[1] : v[0], recv);
  }
  v[0] = ff_add(v[0], ff_shfl_xor(v[0], 2));
  v[0] = ff_add(v[0], ff_shfl_xor(v[0], 1));
  return v[0];  // sum number (lane >> 4) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1) = lane >> 2
}

// Gram rows [nb columns of B | ny (0 or LZ_B) columns of Y]^T Y over this CTA's nr rows (from
// row r0), summed over the cluster into L.G[i * LZ_B + c] (i < nb + ny).  buf alternates
// between calls, so that one cluster barrier per call orders every CTA's reads of a buffer
// before its next write.
__device__ void oc_gram(const OrthArgs& a, const OcSmem& L, int nb, int ny, int64_t r0, int nr, int buf,
                        cooperative_groups::cluster_group& cl) {
  const int nA = nb + ny;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* mine = L.part + (size_t)buf * OC_NA * LZ_B;
  for (int i = warp; i < nA; i += OC_WARPS) {
    float acc[LZ_B];
#pragma unroll
    for (int c = 0; c < LZ_B; ++c) acc[c] = 0.f;
    const float* col = i < nb ? a.B + (int64_t)i * a.rows + r0 : nullptr;
    const int yc = i - nb;
    for (int base = 0; base < nr; base += 32 * OC_UNROLL) {
      float x[OC_UNROLL];
#pragma unroll
      for (int u = 0; u < OC_UNROLL; ++u) {
        const int rl = base + u * 32 + lane;
        x[u] = rl < nr ? (col ? __ldg(col + rl) : L.Ys[rl * LZ_B + yc]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < OC_UNROLL; ++u) {
        const int rl = base + u * 32 + lane;
        if (rl < nr) {
          const float4 y0 = *reinterpret_cast<const float4*>(L.Ys + rl * LZ_B);
          const float4 y1 = *reinterpret_cast<const float4*>(L.Ys + rl * LZ_B + 4);
          acc[0] = fmaf(x[u], y0.x, acc[0]);
          acc[1] = fmaf(x[u], y0.y, acc[1]);
          acc[2] = fmaf(x[u], y0.z, acc[2]);
          acc[3] = fmaf(x[u], y0.w, acc[3]);
          acc[4] = fmaf(x[u], y1.x, acc[4]);
          acc[5] = fmaf(x[u], y1.y, acc[5]);
          acc[6] = fmaf(x[u], y1.z, acc[6]);
          acc[7] = fmaf(x[u], y1.w, acc[7]);
        }
      }
    }
    ff2 v[LZ_B];
#pragma unroll
    for (int c = 0; c < LZ_B; ++c) v[c] = ff_make(acc[c]);
    const ff2 t = oc_warp_sum8(v, lane);
    if ((lane & 3) == 0) mine[i * LZ_B + (lane >> 2)] = make_float2(t.hi, t.lo);
  }
  cl.sync();
  const int nc = (int)cl.num_blocks();
  for (int e = threadIdx.x; e < nA * LZ_B; e += OC_THREADS) {
    ff2 t = ff_make(0.f);
    for (int q = 0; q < nc; ++q) {
      const float2 v = cl.map_shared_rank(mine, q)[e];
      t = ff_add(t, ff2{v.x, v.y});
    }
    L.G[e] = ff_to_d(t);
    if (e < nb * LZ_B) L.Gf[e] = (float)L.G[e];  // B^T Y for oc_sub_basis
  }
  __syncthreads();
}

// Y -= B G[0:p] over this CTA's rows, one thread per row (G from the last oc_gram).
__device__ void oc_sub_basis(const OrthArgs& a, const OcSmem& L, int64_t r0, int nr) {
  for (int rl = threadIdx.x; rl < nr; rl += OC_THREADS) {
    const float* brow = a.B + r0 + rl;
    float s[LZ_B];
#pragma unroll
    for (int c = 0; c < LZ_B; ++c) s[c] = 0.f;
    for (int i0 = 0; i0 < a.p; i0 += OC_UNROLL) {
      float x[OC_UNROLL];
#pragma unroll
      for (int u = 0; u < OC_UNROLL; ++u) x[u] = i0 + u < a.p ? __ldg(brow + (int64_t)(i0 + u) * a.rows) : 0.f;
#pragma unroll
      for (int u = 0; u < OC_UNROLL; ++u) {
        if (i0 + u < a.p) {
          const float4 g0 = *reinterpret_cast<const float4*>(L.Gf + (i0 + u) * LZ_B);
          const float4 g1 = *reinterpret_cast<const float4*>(L.Gf + (i0 + u) * LZ_B + 4);
          s[0] = fmaf(x[u], g0.x, s[0]);
          s[1] = fmaf(x[u], g0.y, s[1]);
          s[2] = fmaf(x[u], g0.z, s[2]);
          s[3] = fmaf(x[u], g0.w, s[3]);
          s[4] = fmaf(x[u], g1.x, s[4]);
          s[5] = fmaf(x[u], g1.y, s[5]);
          s[6] = fmaf(x[u], g1.z, s[6]);
          s[7] = fmaf(x[u], g1.w, s[7]);
        }
      }
    }
    float* y = L.Ys + rl * LZ_B;
#pragma unroll
    for (int c = 0; c < LZ_B; ++c) y[c] -= s[c];
  }
  __syncthreads();
}

// Y <- Y M over this CTA's rows, M an 8 x 8 matrix (column-major doubles in shared memory).
__device__ void oc_mul_small(const OcSmem& L, const double* M, int nr) {
  __shared__ float Mf[LZ_B * LZ_B];
  if (threadIdx.x < LZ_B * LZ_B) Mf[threadIdx.x] = (float)M[threadIdx.x];
  __syncthreads();
  for (int rl = threadIdx.x; rl < nr; rl += OC_THREADS) {
    float* y = L.Ys + rl * LZ_B;
    float v[LZ_B], o[LZ_B];
#pragma unroll
    for (int j = 0; j < LZ_B; ++j) v[j] = y[j];
#pragma unroll
    for (int c = 0; c < LZ_B; ++c) {
      float t = 0.f;
#pragma unroll
      for (int j = 0; j < LZ_B; ++j) t = fmaf(v[j], Mf[j + c * LZ_B], t);
      o[c] = t;
    }
#pragma unroll
    for (int c = 0; c < LZ_B; ++c) y[c] = o[c];
  }
  __syncthreads();
}

// Columns in `mask` of this CTA's rows: replaced by the counter-based values of
// cert_refill_kernel (refill) or zeroed.
__device__ void oc_fix_cols(const OrthArgs& a, const OcSmem& L, int mask, bool refill, int64_t r0, int nr) {
  for (int e = threadIdx.x; e < nr * LZ_B; e += OC_THREADS) {
    const int rl = e >> 3, c = e & 7;
    if (!((mask >> c) & 1)) continue;
    float v = 0.f;
    if (refill) {
      const int64_t i = r0 + rl + (int64_t)c * a.rows;
      uint64_t z = a.seed * 0x9E3779B97F4A7C15ull + (uint64_t)i;
      z += 0x9e3779b97f4a7c15ull;
      z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
      z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
      z ^= z >> 31;
      v = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
    L.Ys[e] = v;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(OC_THREADS, 1) cert_orth_cluster_kernel(OrthArgs a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char oc_raw[];
  const OcSmem L = oc_layout(oc_raw);
  __shared__ double H[LZ_B * LZ_B], W[LZ_B * LZ_B], R[LZ_B * LZ_B], Ri[LZ_B * LZ_B], rd[LZ_B], n0[LZ_B];
  __shared__ int bad_s;
  const int64_t r0 = (int64_t)cl.block_rank() * a.rows_per;
  const int nr = (int)(r0 < a.rows ? (a.rows - r0 < a.rows_per ? a.rows - r0 : a.rows_per) : 0);
  for (int e = threadIdx.x; e < nr * LZ_B; e += OC_THREADS) {  // this CTA's rows of Y (from src)
    const int c = e / nr, rl = e - c * nr;
    L.Ys[rl * LZ_B + c] = a.src[r0 + rl + (int64_t)c * a.rows];
  }
  __syncthreads();
  int buf = 0;
  const int p = a.p;
  auto gram = [&](int nb, int ny) {
    oc_gram(a, L, nb, ny, r0, nr, buf, cl);
    buf ^= 1;
  };
  auto yty = [&]() {  // H = Y^T Y
    gram(0, LZ_B);
    if (threadIdx.x < LZ_B * LZ_B) H[threadIdx.x] = L.G[threadIdx.x];
    __syncthreads();
  };
  auto project = [&]() {  // Y -= B (B^T Y)
    if (p == 0) return;
    gram(p, 0);
    oc_sub_basis(a, L, r0, nr);
  };
  auto normalise = [&]() {  // Y <- Y R^{-1}, floor 1e-12 of the largest pivot
    yty();
    cta_chol_masked(H, LZ_B, 1e-12, nullptr, W, R, Ri, rd, &bad_s);
    oc_mul_small(L, Ri, nr);
  };
  const double collapse = 1e-6;
  // First projection with the column norms from the same pass ([B | Y]^T Y).
  gram(p, LZ_B);
  if (threadIdx.x < LZ_B) n0[threadIdx.x] = L.G[(p + threadIdx.x) * LZ_B + threadIdx.x];
  __syncthreads();
  if (p > 0) oc_sub_basis(a, L, r0, nr);
  project();
  yty();
  int bad = cta_chol_masked(H, LZ_B, collapse, n0, W, R, Ri, rd, &bad_s);
  if (bad != 0) {
    // Collapsed columns: refilled with random values, projected again and zeroed if they
    // collapse once more.
    oc_fix_cols(a, L, bad, true, r0, nr);
    yty();
    if (threadIdx.x < LZ_B) n0[threadIdx.x] = H[threadIdx.x * (LZ_B + 1)];
    __syncthreads();
    project();
    project();
    yty();
    bad = cta_chol_masked(H, LZ_B, collapse, n0, W, R, Ri, rd, &bad_s);
    if (bad != 0) oc_fix_cols(a, L, bad, false, r0, nr);
    normalise();
  } else {
    oc_mul_small(L, Ri, nr);
  }
  project();
  normalise();
  for (int e = threadIdx.x; e < nr * LZ_B; e += OC_THREADS) {
    const int c = e / nr, rl = e - c * nr;
    a.Y[r0 + rl + (int64_t)c * a.rows] = L.Ys[rl * LZ_B + c];
  }
  cl.sync();  // no CTA leaves while another may still read its partials
}

// Whether orth_block can run as one cluster launch for these sizes.
static bool orth_cluster_fits(int64_t rows, int p) {
  return rows >= 1 && rows <= (int64_t)OC_MAXC * OC_ROWS && p >= 0 && p <= OC_PMAX;
}

static rpca_status orth_block_cluster(rpca_ctx* c, const float* src, float* Y, int64_t rows, const float* Bm, int p,
                                      uint64_t seed) {
  static const bool attr_ok = [] {
    return cudaFuncSetAttribute(cert_orth_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)oc_smem_bytes()) == cudaSuccess;
  }();
  if (!attr_ok) return set_err(c, RPCA_ECUDA, "shared memory of the cluster orthonormalisation");
  // About 128 rows per CTA: the basis Grams are latency-bound per CTA, so a block of up to a
  // thousand rows spreads over up to eight SMs of one cluster (measured on the 1000-row side
  // of the video workload: 1, 2, 4, 8 CTAs took the certificate from 3.24 to 3.13, 3.11, 3.08 ms).
  const int nc = (int)std::min<int64_t>(OC_MAXC, std::max<int64_t>(1, (rows + 127) / 128));
  OrthArgs a;
  a.B = Bm;
  a.p = p;
  a.Y = Y;
  a.src = src ? src : Y;
  a.rows = rows;
  a.rows_per = (int)((rows + nc - 1) / nc);
  a.seed = seed;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(OC_THREADS);
  cfg.dynamicSmemBytes = oc_smem_bytes();
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CERT_CUDA(cudaLaunchKernelEx(&cfg, cert_orth_cluster_kernel, a));
  count_launches(c, 1);
  return RPCA_OK;
}

// Orthonormalises the block Y (rows x 8) against the basis B (rows x p; the fixed range
// basis followed by the Krylov blocks, contiguous), by two passes of classical Gram-Schmidt
// and CholeskyQR.  A column that loses all but 1e-3 of its norm to the projection and to the
// earlier columns of its block is treated as collapsed (in float32 its remainder is mostly
// rounding along B, which normalising would amplify): it is replaced by a random column,
// projected again, and zeroed if it collapses once more (the complement of B is exhausted).
// Then: normalise, project again, normalise again; zero columns stay zero.  The host reads
// the collapse mask once per block; when nothing collapsed, the factor of the collapse test
// is the first CholeskyQR pass.
static rpca_status orth_block(rpca_ctx* c, float* Y, int64_t rows, const float* Bm, int p, uint64_t seed) {
  rpca_status s;
  CertBuffers* b = c->cert;
  const double collapse = 1e-6;  // squared-norm ratio
  if (p > 0 && Bm + (int64_t)p * rows == Y) {
    // First projection with the column norms of Y from the same pass: [B | Y]^T Y.
    const int nblk = ts_gram_partial_c(c, Bm, rows, p + LZ_B, Y, rows, LZ_B, rows, b->ts, c->stream);
    if (nblk < 0) return set_err(c, RPCA_ECUDA, "ts_gram_partial");
    cert_proj_reduce_kernel<<<((p + LZ_B) * LZ_B + 7) / 8, 256, 0, c->stream>>>(b->ts.part, nblk, p, b->st);
    count_launches(c, 1);
    CERT_CUDA(ts_mul_c(c, Bm, rows, p, b->st->G2, p + LZ_B, LZ_B, Y, rows, rows, -1.f, 1.f, c->stream));
    if ((s = project_out(c, Bm, p, Y, rows)) != RPCA_OK) return s;
  } else {
    if ((s = record_norms(c, Y, rows)) != RPCA_OK) return s;
    if ((s = project_twice(c, Y, rows, Bm, p)) != RPCA_OK) return s;
  }
  if ((s = gram_chol(c, Y, rows, collapse, 1)) != RPCA_OK) return s;
  CERT_CUDA(cudaMemcpyAsync(&b->host->bad_mask, &b->st->bad_mask, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CERT_CUDA(cudaStreamSynchronize(c->stream));
  if (b->host->bad_mask != 0) {
    cert_refill_kernel<<<256, 256, 0, c->stream>>>(Y, rows, b->st, seed);
    count_launches(c, 1);
    if ((s = record_norms(c, Y, rows)) != RPCA_OK) return s;
    if ((s = project_twice(c, Y, rows, Bm, p)) != RPCA_OK) return s;
    if ((s = gram_chol(c, Y, rows, collapse, 1)) != RPCA_OK) return s;
    cert_zero_cols_kernel<<<256, 256, 0, c->stream>>>(Y, rows, b->st);
    count_launches(c, 1);
    if ((s = normalise(c, Y, rows)) != RPCA_OK) return s;
  } else {
    CERT_CUDA(ts_mul_c(c, Y, rows, LZ_B, b->st->Rinv, LZ_B, LZ_B, Y, rows, rows, 1.f, 0.f, c->stream));
  }
  if ((s = project_out(c, Bm, p, Y, rows)) != RPCA_OK) return s;
  return normalise(c, Y, rows);
}

// orth_block of Y (first a copy of src when src is not null): one cluster launch (up to eight
// CTAs of about 128 rows) for up to OC_SINGLE rows, else the multi-launch form.  RPCA_CERT_CLUSTER=1 takes the cluster
// launch wherever it fits (up to OC_MAXC x OC_ROWS rows), =0 never.  Measured on the
// 256-instance batch (m up to 20000), the eight-CTA cluster kept the m-side blocks 2.5x longer
// on the device than the multi-launch form (eight SMs stream the basis at a fraction of the
// GPU's rate), although it made a quarter of the launches; the cluster takes the small side.
constexpr int64_t OC_SINGLE = 1024;
static rpca_status orth_any(rpca_ctx* c, const float* src, float* Y, int64_t rows, const float* Bm, int p,
                            uint64_t seed) {
  const char* env = getenv("RPCA_CERT_CLUSTER");
  const int mode = env ? (env[0] == '0' ? 0 : 2) : 1;  // 0 never, 1 small side only, 2 wherever it fits
  if (mode > 0 && orth_cluster_fits(rows, p) && (mode == 2 || rows <= OC_SINGLE))
    return orth_block_cluster(c, src, Y, rows, Bm, p, seed);
  if (src && src != Y) CERT_CUDA(cudaMemcpyAsync(Y, src, sizeof(float) * rows * LZ_B, cudaMemcpyDeviceToDevice, c->stream));
  return orth_block(c, Y, rows, Bm, p, seed);
}

// Leading Ritz pairs of the projected matrix T[0:d, 0:d] of the last spectral step (one-sided
// Jacobi SVD: one warp up to d = 32, else one CTA), into CertBuffers::ritz and the state.
static rpca_status ritz_vectors(rpca_ctx* c, int d) {
  CertBuffers* b = c->cert;
  if (d <= 32) {
    cert_ritz_warp_kernel<<<1, 32, 0, c->stream>>>(b->st, b->T, d, c->lam_L, 1, b->ritz);
  } else {
    const size_t rsm = d <= RITZ_SMEM_D ? (size_t)2 * d * d * sizeof(float) : 0;
    CERT_CUDA(cudaFuncSetAttribute(cert_ritz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   2 * RITZ_SMEM_D * RITZ_SMEM_D * (int)sizeof(float)));
    cert_ritz_kernel<<<1, 1024, rsm, c->stream>>>(b->st, b->T, b->Tw, b->Tv, d, c->lam_L, 1, b->ritz);
  }
  count_launches(c, 1);
  CERT_CUDA(cudaGetLastError());
  return RPCA_OK;
}

// side 1: Y1 = D BV;  side 2: Y2 = D^T BU  (one pass over X each).
static rpca_status apply_D(rpca_ctx* c, int side, const float* BV, const float* BU, float* Y1, float* Y2) {
  CertBuffers* b = c->cert;
  const FgPlan* P = apply_plan(c, c->k, side);
  if (!P) return RPCA_EUNSUPPORTED;
  FgLaunch L;
  L.U = b->Up;
  L.V = b->Vp;
  L.BU = BU;
  L.BV = BV;
  L.fin_mode = FIN_APPLY;
  L.GU = Y1;
  L.GV = Y2;
  return launch_fg(c, *P, L, c->stream);
}

// reuse: the last call on this context evaluated the first four steps (F, Grams, t1, t2, t3 and
// the range bases) at this same point and nothing has changed them since: go straight to the
// spectral step (a solve that just found the cheap terms within the tolerance).
// D V and D^T U from a gradient at the same point: G = D (V, U) + lam_L (U, V) (g, x: the
// solver's vectors [U | V], the V part from offset mk).
__global__ void cert_raw_from_grad_kernel(const float* g, const float* x, float lam, int64_t mk, int64_t nk, float* DV,
                                          float* DtU) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mk + nk; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = fmaf(-lam, x[i], g[i]);
    if (i < mk) DV[i] = v;
    else DtU[i - mk] = v;
  }
}

rpca_status cert_compute(rpca_ctx* c, const float* U, const float* V, rpca_cert* out, bool full, bool reuse,
                         const float* grad, const double* f_dev, double f_host) {
  rpca_status s = ensure_cert(c);
  if (s != RPCA_OK) return s;
  CertBuffers* b = c->cert;
  const int64_t m = c->m, n = c->n;
  const int k = c->k;
  CertState* st = b->st;
  double F = 0;
  if (reuse) {
    F = b->last_F;
  } else {
    cert_reset_kernel<<<1, 1, 0, c->stream>>>(st);
    count_launches(c, 1);
    // F(0) = phi(0) once per context (distance bound).
    if (!b->have_F0) {
      FgLaunch L0;
      L0.U = b->zm;
      L0.V = b->zn;
      L0.GU = b->DV;
      L0.GV = b->DtU;
      L0.fin_mode = FIN_FG_RAW;
      L0.out = c->ws.out + 4;
      if ((s = launch_fg(c, c->fg_plan, L0, c->stream)) != RPCA_OK) return s;
      double f0 = 0;
      CERT_CUDA(cudaMemcpyAsync(&f0, c->ws.out + 4, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      CERT_CUDA(cudaStreamSynchronize(c->stream));
      c->F0 = f0;
      b->have_F0 = true;
    }
    // 1. F and the raw products: one pass over X, or, given the gradient at this point (a
    // solve's current iterate, [U | V] contiguous), D V = G_U - lam_L U and D^T U = G_V - lam_L V.
    const double* Fp = grad ? f_dev : c->ws.out;
    if (grad) {
      const int64_t mk = m * k, nk = n * k;
      cert_raw_from_grad_kernel<<<(int)std::min<int64_t>(4 * c->nsm, (mk + nk + 255) / 256), 256, 0, c->stream>>>(
          grad, U, (float)c->lam_L, mk, nk, b->DV, b->DtU);
      count_launches(c, 1);
      CERT_CUDA(cudaGetLastError());
    } else {
      FgLaunch L;
      L.U = U;
      L.V = V;
      L.GU = b->DV;
      L.GV = b->DtU;
      L.fin_mode = FIN_FG_RAW;
      L.out = c->ws.out;
      if ((s = launch_fg(c, c->fg_plan, L, c->stream)) != RPCA_OK) return s;
    }
    // 2. Grams.
    CERT_CUDA(ts_gram_c(c, U, m, k, U, m, k, m, st->G, b->ts, c->stream));
    CERT_CUDA(cudaMemcpy2DAsync(st->AUU, CERT_KMAX * 8, st->G, k * 8, k * 8, k, cudaMemcpyDeviceToDevice, c->stream));
    CERT_CUDA(ts_gram_c(c, V, n, k, V, n, k, n, st->G, b->ts, c->stream));
    CERT_CUDA(cudaMemcpy2DAsync(st->AVV, CERT_KMAX * 8, st->G, k * 8, k * 8, k, cudaMemcpyDeviceToDevice, c->stream));
    CERT_CUDA(ts_gram_c(c, U, m, k, b->DV, m, k, m, st->G, b->ts, c->stream));
    CERT_CUDA(cudaMemcpy2DAsync(st->MUDV, CERT_KMAX * 8, st->G, k * 8, k * 8, k, cudaMemcpyDeviceToDevice, c->stream));
    // 3. Small factorisations, t1.
    cert_small_kernel<<<1, 256, 0, c->stream>>>(st, k, c->lam_L, Fp);
    count_launches(c, 1);
    CERT_CUDA(cudaGetLastError());
    // 4. t3 = ||DV T_V - U P2||^2, t2 = ||DtU T_U - V P3||^2.
    const int rg = (int)std::min<int64_t>(2 * c->nsm, (std::max(m, n) + 255) / 256);
    cert_resid_kernel<<<std::max(1, (int)std::min<int64_t>(rg, (m + 255) / 256)), 256, 0, c->stream>>>(
        b->DV, U, m, k, st, 0, b->blk, b->counter, st);
    count_launches(c, 1);
    cert_resid_kernel<<<std::max(1, (int)std::min<int64_t>(rg, (n + 255) / 256)), 256, 0, c->stream>>>(
        b->DtU, V, n, k, st, 1, b->blk, b->counter, st);
    count_launches(c, 1);
    CERT_CUDA(cudaGetLastError());
    CERT_CUDA(cudaMemcpyAsync(b->host, st, sizeof(CertState), cudaMemcpyDeviceToHost, c->stream));
    if (!grad) CERT_CUDA(cudaMemcpyAsync(&F, c->ws.out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CERT_CUDA(cudaStreamSynchronize(c->stream));
    if (grad) F = f_host;
    b->last_F = F;
  }
  const int r = b->host->r;
  int steps = 0;
  if (full) {
    // 5. t4 by block Golub-Kahan-Lanczos on A = P_U1perp D P_V1perp.
    b->U1 = b->P - m * r;
    b->V1 = b->Q - n * r;
    if (r > 0) {
      CERT_CUDA(ts_mul_c(c, U, m, k, st->TU, CERT_KMAX, r, b->U1, m, m, 1.f, 0.f, c->stream));
      CERT_CUDA(ts_mul_c(c, V, n, k, st->TV, CERT_KMAX, r, b->V1, n, n, 1.f, 0.f, c->stream));
    }
    pad_copy_kernel<<<256, 256, 0, c->stream>>>(U, m, k, b->Up, b->Kp);
    count_launches(c, 1);
    pad_copy_kernel<<<256, 256, 0, c->stream>>>(V, n, k, b->Vp, b->Kp);
    count_launches(c, 1);
    cert_zero_T_kernel<<<64, 256, 0, c->stream>>>(b->T, st);
    count_launches(c, 1);
    fill_normal(b->Q, n * LZ_B, 0x5eedULL + (uint64_t)c->opt.seed, 1.f, c->stream);
    count_launches(c, 1);
    if ((s = orth_any(c, nullptr, b->Q, n, b->V1, r, 11)) != RPCA_OK) return s;
    // Krylov dimension cap: 256, or the dimension of the complement of range(V1).
    const int64_t room = std::max<int64_t>(1, std::min(m, n) - r);
    const int smax = (int)std::min<int64_t>(LZ_SMAX, (room + LZ_B - 1) / LZ_B);
    for (int j = 0; j < smax; ++j) {
      float* Qj = b->Q + (int64_t)j * LZ_B * n;
      float* Pj = b->P + (int64_t)j * LZ_B * m;
      // D Q_j (Q_j is orthogonal to V1 by construction).  A Q_j = P_U1perp D Q_j; its
      // projection on U1 is removed by orth_block, and T = P^T A Q_j = P^T D Q_j because the
      // columns of P are orthogonal to U1.
      if ((s = apply_D(c, 1, Qj, b->zm, b->Wraw, b->Z)) != RPCA_OK) return s;
      if ((s = orth_any(c, b->Wraw, Pj, m, b->U1, r + j * LZ_B, 1000 + 2 * j)) != RPCA_OK) return s;
      // Column block j of T = P^T A Q.
      CERT_CUDA(ts_gram_c(c, b->P, m, (j + 1) * LZ_B, b->Wraw, m, LZ_B, m, st->G, b->ts, c->stream));
      cert_store_T_kernel<<<1, 256, 0, c->stream>>>(st, b->T, (j + 1) * LZ_B, j * LZ_B);
      count_launches(c, 1);
      steps = j + 1;
      const bool last = (j == smax - 1);
      const int d = steps * LZ_B;
      // Up to RITZV_DMAX the Ritz values alone are located after every step from the second
      // on (the vectors are formed on request, ritz_vectors); beyond it the Jacobi SVD (values
      // and vectors) runs every fourth step.
      if (d <= RITZV_DMAX && (steps >= 2 || last)) {
        static const bool attr_ok = [] {
          return cudaFuncSetAttribute(cert_ritz_values_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      RITZV_DMAX * (RITZV_DMAX + 1) * (int)sizeof(float)) == cudaSuccess;
        }();
        if (!attr_ok) return set_err(c, RPCA_ECUDA, "shared memory of the Ritz-value kernel");
        cert_ritz_values_kernel<<<1, RITZV_THREADS, (size_t)d * (d + 1) * sizeof(float), c->stream>>>(
            st, b->T, d, c->lam_L, last ? 1 : 0);
        count_launches(c, 1);
        CERT_CUDA(cudaGetLastError());
        int conv = 0;
        CERT_CUDA(cudaMemcpyAsync(&conv, &st->converged, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CERT_CUDA(cudaStreamSynchronize(c->stream));
        if (conv) break;
      } else if (d > RITZV_DMAX && ((steps % 4) == 0 || last)) {
        if (d <= 32) {
          cert_ritz_warp_kernel<<<1, 32, 0, c->stream>>>(st, b->T, d, c->lam_L, last ? 1 : 0, b->ritz);
        } else {
          const size_t rsm = d <= RITZ_SMEM_D ? (size_t)2 * d * d * sizeof(float) : 0;
          CERT_CUDA(cudaFuncSetAttribute(cert_ritz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * RITZ_SMEM_D * RITZ_SMEM_D * (int)sizeof(float)));
          cert_ritz_kernel<<<1, 1024, rsm, c->stream>>>(st, b->T, b->Tw, b->Tv, d, c->lam_L, last ? 1 : 0, b->ritz);
        }
        count_launches(c, 1);
        CERT_CUDA(cudaGetLastError());
        int conv = 0;
        CERT_CUDA(cudaMemcpyAsync(&conv, &st->converged, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CERT_CUDA(cudaStreamSynchronize(c->stream));
        if (conv) break;
      }
      // Q_{j+1} from A^T P_j = P_V1perp D^T P_j, orthogonal to V1 and Q_0..Q_j.
      float* Qn = b->Q + (int64_t)(j + 1) * LZ_B * n;
      if ((s = apply_D(c, 2, b->zn, Pj, b->W, Qn)) != RPCA_OK) return s;
      if ((s = orth_any(c, nullptr, Qn, n, b->V1, r + (j + 1) * LZ_B, 1001 + 2 * j)) != RPCA_OK) return s;
    }
  }
  CERT_CUDA(cudaMemcpyAsync(b->host, st, sizeof(CertState), cudaMemcpyDeviceToHost, c->stream));
  CERT_CUDA(cudaStreamSynchronize(c->stream));
  if ((s = check_dev_err(c)) != RPCA_OK) return s;
  const CertState& h = *b->host;
  rpca_cert o;
  memset(&o, 0, sizeof o);
  o.t1 = h.t1;
  o.t2 = h.resid[1];
  o.t3 = h.resid[0];
  o.t4 = full ? h.t4 : 0.0;
  o.cert = std::sqrt(std::max(0.0, o.t1 + o.t2 + o.t3 + o.t4));
  o.cert_rel = o.cert / c->lam_L;
  o.normL_F = h.normL;
  o.F = F;
  if (F < c->F_best) c->F_best = F;
  o.F_bound = std::min(c->F0, c->F_best);
  o.F_trunc = 2.0 * c->lam_L * h.sig_drop;
  {
    const double scale = c->lam_L * o.normL_F + o.F_bound;
    o.trunc_rel = scale > 0.0 ? o.F_trunc / scale : (o.F_trunc > 0.0 ? INFINITY : 0.0);
  }
  o.gap_bound = o.cert * (o.normL_F + o.F_bound / c->lam_L) + o.F_trunc;
  o.rank_r = h.r;
  o.krylov_steps = steps;
  o.sigma1_perp = full ? h.sigma1 : 0.0;
  *out = o;
  return RPCA_OK;
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_certificate(rpca_ctx* c, const float* U, const float* V, rpca_cert* out) {
  if (!c) return RPCA_EINVAL;
  if (c->lk) return set_err(c, RPCA_EUNSUPPORTED, "the certificate is built for k <= 16");
  if (!U || !V || !out) return set_err(c, RPCA_EINVAL, "U, V and out are required");
  return cert_compute(c, U, V, out, true, false, nullptr, nullptr, 0.0);
}

extern "C" rpca_status rpca_perp_directions(rpca_ctx* c, int qmax, float* U, int64_t ldu, float* V, int64_t ldv,
                                            double* sig, int* q_out) {
  if (!c) return RPCA_EINVAL;
  if (!U || !V || !q_out || qmax < 1 || ldu < c->m || ldv < c->n)
    return set_err(c, RPCA_EINVAL, "U, V, q_out are required, qmax >= 1, ldu >= m, ldv >= n");
  *q_out = 0;
  CertBuffers* b = c->cert;
  if (!b) return set_err(c, RPCA_EINVAL, "no certificate has been computed on this context");
  int dq[2] = {0, 0};
  double s[RITZ_TOPQ];
  CERT_CUDA(cudaMemcpyAsync(dq, &b->st->ritz_q, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CERT_CUDA(cudaStreamSynchronize(c->stream));
  if (dq[1] >= 1 && dq[0] < 1) {
    // The last spectral step located the Ritz values alone: form the leading pairs of its
    // projected matrix now (Jacobi SVD of T, which the step left in place).
    rpca_status rs = ritz_vectors(c, dq[1]);
    if (rs != RPCA_OK) return rs;
    CERT_CUDA(cudaMemcpyAsync(dq, &b->st->ritz_q, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  }
  CERT_CUDA(cudaMemcpyAsync(s, b->st->ritz_s, sizeof s, cudaMemcpyDeviceToHost, c->stream));
  CERT_CUDA(cudaStreamSynchronize(c->stream));
  const int q = std::min(std::min(qmax, dq[0]), RITZ_TOPQ), d = dq[1];
  if (d < 1 || q < 1) return set_err(c, RPCA_EINVAL, "the last certificate had no spectral step (rpca_certificate first)");
  const int64_t m = c->m, n = c->n;
  CERT_CUDA(ts_mul_c(c, b->P, m, d, b->ritz, LZ_TMAX, q, U, ldu, m, 1.f, 0.f, c->stream));
  CERT_CUDA(ts_mul_c(c, b->Q, n, d, b->ritz + RITZ_TOPQ * LZ_TMAX, LZ_TMAX, q, V, ldv, n, 1.f, 0.f, c->stream));
  CERT_CUDA(cudaStreamSynchronize(c->stream));
  if (sig)
    for (int t = 0; t < q; ++t) sig[t] = s[t];
  *q_out = q;
  return RPCA_OK;
}

extern "C" rpca_status rpca_perp_direction(rpca_ctx* c, float* u, float* v, double* sigma1) {
  int q = 0;
  double s1 = 0.0;
  rpca_status st = rpca_perp_directions(c, 1, u, c ? c->m : 0, v, c ? c->n : 0, &s1, &q);
  if (st == RPCA_OK && sigma1) *sigma1 = s1;
  return st;
}
