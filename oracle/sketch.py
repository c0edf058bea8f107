"""Randomized-SVD initialisation (Sec. 4.2), float64.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

Sec. 4.2: U0 = U_k Sigma^1/2, V0 = V_k Sigma^1/2 from the SVD of A*(X), computed with a
randomized SVD (Halko, Martinsson, Tropp 2011, which the paper cites for the rSVD).  The
paper is silent on oversampling, power iterations and masked data; the readings used:
oversampling p = 10, q = 2 power iterations, and for a mask the sampled matrix is rescaled
by 1/p_hat with p_hat = |Omega| / (m n).  The Gaussian test matrix ``Omega`` is an input
(n x (k + p)), so the oracle and the GPU path see the same draw.
"""
from __future__ import annotations

import numpy as np


def sampled(X, mask):
    """A*(X): the observed entries of X (zero elsewhere), rescaled by 1/p_hat."""
    X = np.asarray(X, np.float64)
    if mask is None:
        return X
    M = np.asarray(mask) != 0
    p = M.mean()
    return np.where(M, X, 0.0) / max(p, 1e-300)


def rsvd_parts(X, mask, Omega, q=2):
    """Q U_B, the singular values s (descending, one per column of Omega) and V_B of the
    randomized SVD of A*(X) with test matrix Omega."""
    Xs = sampled(X, mask)
    Om = np.asarray(Omega, np.float64)
    Q, _ = np.linalg.qr(Xs @ Om)
    for _ in range(q):
        Z, _ = np.linalg.qr(Xs.T @ Q)
        Q, _ = np.linalg.qr(Xs @ Z)
    B = Q.T @ Xs
    Ub, s, Vbt = np.linalg.svd(B, full_matrices=False)
    return Q @ Ub, s, Vbt.T


def rsvd_init(X, mask, k, Omega, q=2):
    """Return (U0, V0) float64 from the randomized SVD of A*(X) with test matrix Omega."""
    Uq, s, Vq = rsvd_parts(X, mask, Omega, q)
    sq = np.sqrt(s[:k])
    return Uq[:, :k] * sq, Vq[:, :k] * sq
