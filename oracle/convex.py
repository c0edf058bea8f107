"""Convex solvers of the Lagrangian SPCP program with S marginalised: FISTA with exact
singular-value thresholding (reference solutions on tiny instances), and the convex baseline
of Sec. 6.1 -- the same iteration with the thresholding done through a randomized SVD whose
orthogonalisations are TSQR.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

Solves min_L lam_L ||L||_* + phi(L) (Eq. 4 with S marginalised, Eq. genConvex).  Sec. 1
notes that proximal-gradient methods apply but need an SVD every iteration; that is fine on
20 x 15 matrices.  grad phi(L) = P_Omega(clip(L - X, +-lam_S)) is 1-Lipschitz (Sec. 3.2,
Moreau envelope), so the step is 1.  The prox of lam_L ||.||_* is singular-value soft
thresholding.

Readings for the Sec. 6.1 baseline (the paper names LagQN with a TSQR-based rSVD and gives no
iteration): the convex solver is FISTA on the marginalised Lagrangian form (the form LagQN
minimises, the same one Sec. 6.2 marginalises); the prox is the singular-value thresholding of
the rank-l randomized SVD of the gradient point Z (Halko, Martinsson, Tropp 2011, the paper's
rSVD reference) with q power iterations; every QR of the rSVD is a TSQR; the test matrix of
iteration k + 1 is the right singular basis found at iteration k (the first one, Omega_0, is
an input).  The prox is exact when fewer than l singular values of Z exceed lam_L and the
sketch captures them.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import core
from .tsqr import tsqr


def svt(Z, tau):
    """Singular-value soft thresholding: argmin_L tau ||L||_* + 1/2 ||L - Z||_F^2."""
    Uz, s, Vzt = np.linalg.svd(Z, full_matrices=False)
    return (Uz * np.maximum(s - tau, 0.0)) @ Vzt


def fista(X, mask, lam_L, lam_S, iters=20000, tol=1e-14):
    """FISTA (Beck & Teboulle) with unit step; stops when ||L_{t+1} - L_t||_F <= tol * max(1, ||L||)."""
    X = np.asarray(X, np.float64)
    L = np.zeros_like(X)
    Y = L.copy()
    t = 1.0
    for _ in range(iters):
        G = core.D_of_R(Y - X, mask, lam_S)
        Ln = svt(Y - G, lam_L)
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        Y = Ln + ((t - 1.0) / tn) * (Ln - L)
        step = np.linalg.norm(Ln - L)
        L, t = Ln, tn
        if step <= tol * max(1.0, np.linalg.norm(L)):
            break
    return L


def balanced_factors(L, k, tau=1e-12):
    """U = U_k S^1/2, V = V_k S^1/2 from the SVD of L (zero-padded to k columns)."""
    Uz, s, Vzt = np.linalg.svd(np.asarray(L, np.float64), full_matrices=False)
    r = min(k, int(np.sum(s > tau * max(s[0], 1e-300))))
    U = np.zeros((L.shape[0], k))
    V = np.zeros((L.shape[1], k))
    U[:, :r] = Uz[:, :r] * np.sqrt(s[:r])
    V[:, :r] = Vzt[:r].T * np.sqrt(s[:r])
    return U, V


def rsvd_svt(Z, Omega, lam_L, q=1):
    """Rank-l randomized SVD of Z with test matrix Omega (n x l) and q power iterations, each
    QR a TSQR; returns (left m x l, s descending, right n x l, s_thr = max(s - lam_L, 0)) with
    Z ~ left diag(s) right^T and the thresholded prox left diag(s_thr) right^T.

    Steps: A = Z Omega, Q = qr(A); q times: Q_w = qr(Z^T Q), Q = qr(Z Q_w); then
    W = Z^T Q (= B^T with B = Q^T Z), W = Q_w R_w, R_w = U_r diag(s) V_r^T, so that
    B = V_r diag(s) (Q_w U_r)^T: left = Q V_r, right = Q_w U_r."""
    Z = np.asarray(Z, np.float64)
    Q, _ = tsqr(Z @ np.asarray(Omega, np.float64))
    for _ in range(q):
        Qw, _ = tsqr(Z.T @ Q)
        Q, _ = tsqr(Z @ Qw)
    Qw, Rw = tsqr(Z.T @ Q)
    Ur, s, Vrt = np.linalg.svd(Rw)
    return Q @ Vrt.T, s, Qw @ Ur, np.maximum(s - lam_L, 0.0)


@dataclasses.dataclass
class ConvexStep:
    L: np.ndarray      # the iterate L_k entering iteration k
    F: float           # lam_L ||L_k||_* + phi(L_k)
    rel: float         # ||L_k - L_{k-1}||_F / max(1, ||L_k||_F)
    s: np.ndarray      # singular values of the rSVD at iteration k (before thresholding)
    rank: int          # rank of the prox result L_{k+1}


def fista_rsvd(X, mask, lam_L, lam_S, Omega0, q=1, iters=50, L0=None):
    """The Sec. 6.1 convex baseline: FISTA (unit step) whose prox is ``rsvd_svt``.

    Iteration k, from (L_k, L_{k-1}, t_k), t_0 = 1, L_{-1} = L_0:
      Y = L_k + beta_k (L_k - L_{k-1}),  beta_0 = 0,  beta_k = (t_{k-1} - 1) / t_k
      Z = Y - P_Omega(clip(Y - X, +-lam_S))           (gradient step, step 1)
      L_{k+1} = rsvd_svt(Z, Omega_k, lam_L, q)        (Omega_{k+1} = its right basis)
      t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    Returns the list of ConvexStep, one per iteration, each describing L_k (the iterate
    entering the iteration) and the rSVD computed in it."""
    X = np.asarray(X, np.float64)
    L = np.zeros_like(X) if L0 is None else np.asarray(L0, np.float64).copy()
    Lp = L.copy()
    Om = np.asarray(Omega0, np.float64)
    t_prev, t = 1.0, 1.0
    nuc = np.linalg.svd(L, compute_uv=False).sum() if L0 is not None else 0.0
    out = []
    for k in range(iters):
        beta = 0.0 if k == 0 else (t_prev - 1.0) / t
        Y = L + beta * (L - Lp)
        Z = Y - core.D_of_R(Y - X, mask, lam_S)
        left, s, right, st = rsvd_svt(Z, Om, lam_L, q)
        F = lam_L * nuc + core.phi_of_R(L - X, mask, lam_S)
        rel = float(np.linalg.norm(L - Lp) / max(1.0, np.linalg.norm(L)))
        out.append(ConvexStep(L=L, F=float(F), rel=rel, s=s, rank=int(np.count_nonzero(st))))
        Lp, L = L, (left * st) @ right.T
        nuc = float(st.sum())
        Om = right
        t_prev, t = t, 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
    return out
