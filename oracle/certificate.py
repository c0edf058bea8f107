"""Computable convergence certificate of Sec. 3.4, float64.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

Given a factored point L = U V^T, Sec. 3.4 builds an element E of the subdifferential of
lam_L ||L||_* + phi(L) of smallest Frobenius norm reachable from the SVD of L:

  L = [U1 U2] diag(Sigma1, 0) [V1 V2]^T        (U1, V1: the r directions with sigma > 0)
  U1, V1 from thin QR of U and V and an SVD of the small k x k R_U R_V^T (footnote of Sec. 3.4)
  D = P_Omega(clip(U V^T - X, +-lam_S))        (gradient of phi, Sec. 3.2)
  ||E||_F^2 = t1 + t2 + t3 + t4 with
    t1 = || lam_L I + U1^T D V1 ||_F^2
    t2 = || U1^T D V2 ||_F^2   (the paper evaluates it as ||U1^T D||^2 - ||U1^T D V1||^2)
    t3 = || U2^T D V1 ||_F^2   (likewise ||D V1||^2 - ||U1^T D V1||^2)
    t4 = min_{||W'|| <= lam_L} || U2^T D V2 + W' ||_F^2 = sum_i (sigma_i(P_U1perp D P_V1perp) - lam_L)_+^2

Readings of the paper taken here (each is pinned by a test):
* The printed first block is "I - U1^T D V1"; expanding U~^T (Z + D) V~ with Z in the
  nuclear-norm subdifferential gives "I + U1^T D V1" (at the optimum D = -U1 V1^T on the
  range of L).  The sign of the W' block does not matter (the ball is symmetric).
* The paper sets lam_L = 1 "for convenience"; for general lam_L the nuclear-norm
  subgradient is scaled by lam_L (t1 uses lam_L I, t4 thresholds at lam_L), and
  cert_rel = cert / lam_L is the scale-free number that is compared against 1e-4.
* The numerical rank r counts singular values of L above tau * sigma_1 (tau = 1e-8); in
  addition a direction that is both tiny (sigma_i <= 1e-3 sigma_1) and inactive
  (|lam_L + u_i^T D v_i| > lam_L / 2) is placed in the complement block: it is rounding
  residue of a factor column that the nuclear penalty drives to zero, and the certificate is
  then the one of L with that direction truncated (a valid subgradient of the truncated
  point, as the W' block of Eq. subdiff allows).
* A direction whose whole nuclear-norm term is negligible against the objective,
  lam_L sigma_i <= 1e-12 F(L), is numerically zero and goes to the complement block as
  well, active or not (the relative test above cannot see it when every singular value of
  L is at that level, e.g. factors at the rounding floor of float32 when the solution is
  L = 0).  Truncating it changes F by at most (lam_L + ||D||_2) sigma_i.
* Distance bound: ||L - L*||_F <= ||L||_F + F_bound / lam_L with
  F_bound = min(F(0) = phi(0), best objective seen), and the optimality-gap bound
  G(L) - G* <= cert * (||L||_F + F_bound / lam_L) + F_trunc, G(L) = lam_L ||L||_* + phi(L).
* Cost of the truncation (not in the paper, which assumes exact ranks).  With T the directions
  moved to the complement, L^ = L - sum_T sigma_i u_i v_i^T, E = lam_L Z + D, Z in the
  subdifferential of ||.||_* at L^ and D = grad phi(L) (phi convex), every L' satisfies
    G(L') >= G(L) + <E, L' - L> - lam_L sum_T sigma_i (1 - u_i^T W v_i),  ||W||_2 <= 1,
  so G(L) - G* <= cert ||L - L*||_F + F_trunc with F_trunc = 2 lam_L sum_T sigma_i.  The
  certificate reports F_trunc and trunc_rel = F_trunc / (lam_L ||L||_F + F_bound), the same
  quantity in the units of cert_rel (gap_bound = (cert_rel + trunc_rel)(lam_L ||L||_F +
  F_bound)); a point counts as certified at tolerance tol only when both are <= tol.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import core

TAU = 1e-8
DROP_TAU = 1e-3
NEG_TAU = 1e-12


@dataclasses.dataclass
class Cert:
    cert: float
    cert_rel: float
    t1: float
    t2: float
    t3: float
    t4: float
    rank_r: int
    normL_F: float
    F: float
    F_bound: float
    gap_bound: float
    sigma_perp: np.ndarray  # leading singular values of P_U1perp D P_V1perp that were computed
    F_trunc: float = 0.0    # 2 lam_L sum of the truncated singular values (bound on their cost)
    trunc_rel: float = 0.0  # F_trunc / (lam_L ||L||_F + F_bound)

    def certified(self, tol):
        """Both the certificate and the truncation's cost within tol (relative units)."""
        return self.cert_rel <= tol and self.trunc_rel <= tol


def range_bases(U, V, tau=TAU):
    """U1, V1, Sigma1 of L = U V^T via thin QR and the SVD of R_U R_V^T (footnote, Sec. 3.4)."""
    U = np.asarray(U, np.float64)
    V = np.asarray(V, np.float64)
    QU, RU = np.linalg.qr(U)
    QV, RV = np.linalg.qr(V)
    Ur, s, Vrt = np.linalg.svd(RU @ RV.T)
    r = int(np.sum(s > tau * s[0])) if s.size and s[0] > 0 else 0
    return QU @ Ur[:, :r], QV @ Vrt[:r].T, s[:r]


def perp_singular_values(D, U1, V1, lam_L, method="auto", k_s=32):
    """Singular values of P_U1perp D P_V1perp that can exceed lam_L, largest first.

    Small problems: all of them, from a dense SVD of the explicit projected matrix.
    Large problems: the leading k_s from scipy's svds on a LinearOperator, doubling k_s
    until the smallest one returned is below lam_L.
    """
    m, n = D.shape
    if method == "auto":
        method = "dense" if m * n <= 4_000_000 else "svds"
    if method == "dense":
        M = D - U1 @ (U1.T @ D)
        M = M - (M @ V1) @ V1.T
        return np.linalg.svd(M, compute_uv=False)
    from scipy.sparse.linalg import LinearOperator, svds

    def mv(x):
        x = x - V1 @ (V1.T @ x)
        y = D @ x
        return y - U1 @ (U1.T @ y)

    def rmv(y):
        y = y - U1 @ (U1.T @ y)
        x = D.T @ y
        return x - V1 @ (V1.T @ x)

    op = LinearOperator((m, n), matvec=mv, rmatvec=rmv, matmat=mv, rmatmat=rmv, dtype=np.float64)
    while True:
        kk = min(k_s, min(m, n) - 1)
        s = svds(op, k=kk, return_singular_vectors=False, tol=1e-10,
                 random_state=np.random.default_rng(0))
        s = np.sort(s)[::-1]
        if s[-1] < lam_L or kk >= min(m, n) - 1:
            return s
        k_s *= 2


def certificate(X, mask, U, V, lam_L, lam_S, F_best=None, tau=TAU, t4_method="auto"):
    """The Sec. 3.4 certificate at L = U V^T, with the paper's term formulas."""
    U = np.asarray(U, np.float64)
    V = np.asarray(V, np.float64)
    R = core.residual(X, U, V)
    D = core.D_of_R(R, mask, lam_S)
    F = 0.5 * lam_L * (np.sum(U * U) + np.sum(V * V)) + core.phi_of_R(R, mask, lam_S)
    U1, V1, s1 = range_bases(U, V, tau)
    if s1.size:
        b_diag = np.einsum("ij,ij->j", U1, D @ V1)
        keep = ~((s1 <= DROP_TAU * s1[0]) & (np.abs(lam_L + b_diag) > 0.5 * lam_L))
        keep &= ~(lam_L * s1 <= NEG_TAU * F)
        U1, V1, s1_kept = U1[:, keep], V1[:, keep], s1[keep]
        sig_dropped = float(np.sum(s1[~keep]))
    else:
        s1_kept = s1
        sig_dropped = 0.0
    r = s1_kept.size
    DV1 = D @ V1
    UtD = U1.T @ D
    B = U1.T @ DV1
    t1 = float(np.sum((lam_L * np.eye(r) + B) ** 2))
    # ||U1^T D V2||^2 and ||U2^T D V1||^2 as the norms of the projected blocks (the paper's
    # "||U1^T D||^2 - ||U1^T D V1||^2" is the same number but cancels near the optimum).
    E2 = UtD - B @ V1.T
    E3 = DV1 - U1 @ B
    t2 = float(np.sum(E2 * E2))
    t3 = float(np.sum(E3 * E3))
    sp = perp_singular_values(D, U1, V1, lam_L, t4_method)
    t4 = float(np.sum(np.maximum(sp - lam_L, 0.0) ** 2))
    cert = float(np.sqrt(max(t1 + t2 + t3 + t4, 0.0)))
    F0 = core.phi_of_R(-np.asarray(X, np.float64), mask, lam_S)
    F_bound = min(F0, F if F_best is None else min(F, F_best))
    normL = float(np.sqrt(np.sum(s1 ** 2)))
    F_trunc = 2.0 * lam_L * sig_dropped
    scale = lam_L * normL + F_bound
    trunc_rel = F_trunc / scale if scale > 0 else (0.0 if F_trunc == 0 else np.inf)
    gap = cert * (normL + F_bound / lam_L) + F_trunc
    return Cert(cert=cert, cert_rel=cert / lam_L, t1=t1, t2=t2, t3=t3, t4=t4, rank_r=r,
                normL_F=normL, F=float(F), F_bound=float(F_bound), gap_bound=float(gap),
                sigma_perp=sp, F_trunc=float(F_trunc), trunc_rel=float(trunc_rel))


def perp_matrix(X, mask, U, V, lam_L, lam_S, tau=TAU):
    """The explicit projected matrix P_U1perp D P_V1perp at L = U V^T (U1, V1 as the
    certificate takes them: negligible and tiny-inactive directions in the complement)."""
    U = np.asarray(U, np.float64)
    V = np.asarray(V, np.float64)
    R = core.residual(X, U, V)
    D = core.D_of_R(R, mask, lam_S)
    F = 0.5 * lam_L * (np.sum(U * U) + np.sum(V * V)) + core.phi_of_R(R, mask, lam_S)
    U1, V1, s1 = range_bases(U, V, tau)
    if s1.size:
        b_diag = np.einsum("ij,ij->j", U1, D @ V1)
        keep = ~((s1 <= DROP_TAU * s1[0]) & (np.abs(lam_L + b_diag) > 0.5 * lam_L))
        keep &= ~(lam_L * s1 <= NEG_TAU * F)
        U1, V1 = U1[:, keep], V1[:, keep]
    M = D - U1 @ (U1.T @ D)
    return M - (M @ V1) @ V1.T


def perp_top_pairs(X, mask, U, V, lam_L, lam_S, q, tau=TAU):
    """The q largest singular values of P_U1perp D P_V1perp (descending) and their unit
    singular vectors (columns of Uq, Vq, u_i^T D v_i = sigma_i)."""
    M = perp_matrix(X, mask, U, V, lam_L, lam_S, tau)
    Uu, ss, Vt = np.linalg.svd(M, full_matrices=False)
    return ss[:q], Uu[:, :q], Vt[:q].T


def perp_top_pair(X, mask, U, V, lam_L, lam_S, tau=TAU):
    """Largest singular value sigma_1 of P_U1perp D P_V1perp at L = U V^T and its unit singular
    vectors (u_1, v_1) with u_1^T D v_1 = sigma_1 (dense SVD of the explicit projected matrix)."""
    ss, Uq, Vq = perp_top_pairs(X, mask, U, V, lam_L, lam_S, 1, tau)
    return float(ss[0]), Uq[:, 0], Vq[:, 0]


def grow_column(X, mask, U, V, lam_L, lam_S):
    """Dynamic rank increase (Sec. 4.1): one more column for (U, V).  Reading of the paper,
    which leaves u, v open: the top singular pair of P_U1perp D P_V1perp, scaled so that the
    new rank-one term is -t u_1 v_1^T with t = sigma_1 - lam_L (the minimiser of the quadratic
    upper bound F(L) - t (sigma_1 - lam_L) + t^2 / 2 that psi'' <= 1 gives); no column (t = 0)
    when sigma_1 <= lam_L.  Returns (U', V', sigma_1)."""
    s1, u1, v1 = perp_top_pair(X, mask, U, V, lam_L, lam_S)
    t = max(s1 - lam_L, 0.0)
    r = np.sqrt(t)
    U2 = np.concatenate([np.asarray(U, np.float64), (r * u1)[:, None]], axis=1)
    V2 = np.concatenate([np.asarray(V, np.float64), (-r * v1)[:, None]], axis=1)
    return U2, V2, s1


def grow_columns(X, mask, U, V, lam_L, lam_S, qmax):
    """Dynamic rank increase by several columns at once (Sec. 4.1 allows growing k
    "aggressively"): every singular pair of P_U1perp D P_V1perp with sigma_i > lam_L, at most
    qmax of them, each scaled like grow_column's (t_i = sigma_i - lam_L).  The pairs are
    orthonormal, so the nuclear norms and the quadratic terms add: F drops by at least
    sum_i (sigma_i - lam_L)^2 / 2.  Returns (U', V', sigmas added)."""
    ss, Uq, Vq = perp_top_pairs(X, mask, U, V, lam_L, lam_S, qmax)
    keep = ss > lam_L
    t = np.sqrt(ss[keep] - lam_L)
    U2 = np.concatenate([np.asarray(U, np.float64), Uq[:, keep] * t], axis=1)
    V2 = np.concatenate([np.asarray(V, np.float64), -Vq[:, keep] * t], axis=1)
    return U2, V2, ss[keep]
