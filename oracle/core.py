"""Huber marginal, factored Split-SPCP objective and gradient, in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

Notation (paper, Sec. 1 and Sec. 5): X is m x n, Omega the observed set (``mask``; None
means every entry is observed), U is m x k, V is n x k, R = U V^T - X.
"""
from __future__ import annotations

import numpy as np


def psi(r, lam):
    """Huber value psi_lam(r): the per-entry value of min_s 1/2 (r + s)^2 + lam |s|.

    Sec. 1 ("Marginalization in S") states that minimising the l1-penalised least-squares
    SPCP objective over S leaves the Huber function of the residual.  Closed form:
    r^2/2 for |r| <= lam, lam |r| - lam^2/2 otherwise.  lam = +inf gives r^2/2.
    """
    r = np.asarray(r, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    a = np.abs(r)
    with np.errstate(invalid="ignore"):
        lin = lam * a - 0.5 * lam * lam
    return np.where(a <= lam, 0.5 * r * r, lin)


def dpsi(r, lam):
    """Derivative of psi_lam: r clipped to [-lam, lam] (Sec. 3.2: the gradient of the
    Moreau envelope, A*(A(L) + S* - b) with S* the soft-thresholded residual)."""
    r = np.asarray(r, dtype=np.float64)
    return np.clip(r, -np.asarray(lam, np.float64), lam)


def residual(X, U, V):
    """R = U V^T - X in float64."""
    return np.asarray(U, np.float64) @ np.asarray(V, np.float64).T - np.asarray(X, np.float64)


def phi_of_R(R, mask, lam_S):
    """phi(L) = sum over observed entries of psi(R_ij) (Eq. after Thm5; masked form Sec. 6.2).
    Unobserved entries contribute nothing."""
    P = psi(R, lam_S)
    if mask is not None:
        P = np.where(np.asarray(mask) != 0, P, 0.0)
    return float(P.sum())


def D_of_R(R, mask, lam_S):
    """D = P_Omega(clip(R, -lam_S, lam_S)): the gradient of phi at L (Sec. 3.2)."""
    D = dpsi(R, lam_S)
    if mask is not None:
        D = np.where(np.asarray(mask) != 0, D, 0.0)
    return D


def objective(X, mask, U, V, lam_L, lam_S):
    """F(U, V) = lam_L/2 (||U||_F^2 + ||V||_F^2) + phi(U V^T)   (Eq. Thm5 / Eq. 7)."""
    U = np.asarray(U, np.float64)
    V = np.asarray(V, np.float64)
    R = residual(X, U, V)
    return 0.5 * lam_L * (np.sum(U * U) + np.sum(V * V)) + phi_of_R(R, mask, lam_S)


def fg(X, mask, U, V, lam_L, lam_S):
    """Objective and gradient of the factored problem.

    f   = lam_L/2 (||U||^2 + ||V||^2) + sum_Omega psi(R)
    G_U = D V + lam_L U,   G_V = D^T U + lam_L V,   D = P_Omega(clip(R, +-lam_S))
    (chain rule through L = U V^T applied to the gradient of phi given in Sec. 3.2).
    Returns (f, G_U, G_V) in float64.
    """
    U = np.asarray(U, np.float64)
    V = np.asarray(V, np.float64)
    R = residual(X, U, V)
    D = D_of_R(R, mask, lam_S)
    f = 0.5 * lam_L * (np.sum(U * U) + np.sum(V * V)) + phi_of_R(R, mask, lam_S)
    return f, D @ V + lam_L * U, D.T @ U + lam_L * V


def apply_D(X, mask, U, V, lam_S, BV, BU):
    """D B_V (m x b) and D^T B_U (n x b) for D = P_Omega(clip(U V^T - X)).

    The products the certificate's spectral step and the sketch initialisation need; with
    U = V = 0 and lam_S = inf, D = -X and these are -X B_V and -X^T B_U.
    """
    D = D_of_R(residual(X, U, V), mask, lam_S)
    return D @ np.asarray(BV, np.float64), D.T @ np.asarray(BU, np.float64)


def sparse_part(X, mask, L, lam_S):
    """S = soft(X - L, lam_S) on Omega and 0 off Omega, so that X ~ L + S.

    Sec. 3.2 writes S* = prox(A(L) - b); with the sign convention of the marginalised
    objective min_S 1/2 ||L + S - X||^2 + lam_S ||S||_1 the minimiser is soft(X - L).
    """
    Z = np.asarray(X, np.float64) - np.asarray(L, np.float64)
    S = np.sign(Z) * np.maximum(np.abs(Z) - lam_S, 0.0)
    if mask is not None:
        S = np.where(np.asarray(mask) != 0, S, 0.0)
    return S


def convex_objective(X, mask, L, lam_L, lam_S):
    """Marginalised convex objective lam_L ||L||_* + phi(L)   (Eq. genConvex with Eq. 4)."""
    L = np.asarray(L, np.float64)
    nuc = np.linalg.svd(L, compute_uv=False).sum()
    return lam_L * nuc + phi_of_R(L - np.asarray(X, np.float64), mask, lam_S)
