"""Convex reference solver for tiny instances: FISTA with singular-value thresholding.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

Solves min_L lam_L ||L||_* + phi(L) (Eq. 4 with S marginalised, Eq. genConvex).  Sec. 1
notes that proximal-gradient methods apply but need an SVD every iteration; that is fine on
20 x 15 matrices.  grad phi(L) = P_Omega(clip(L - X, +-lam_S)) is 1-Lipschitz (Sec. 3.2,
Moreau envelope), so the step is 1.  The prox of lam_L ||.||_* is singular-value soft
thresholding.
"""
from __future__ import annotations

import numpy as np

from . import core


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
