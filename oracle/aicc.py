"""Corrected Akaike information criterion of an SPCP solution (Sec. 5.2), float64 host.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

For a solution L = U V^T, S = shrink(X - L, lam_S) on the observed set (the marginalised
sparse part), Z = L + S - X, the paper's statistical model gives (as printed):

  sigma^2 = ||X||_F^2 / (m n),  b = ||S||_1 / (m n)
  ell = -(m n / 2) log(2 pi sigma^2) - ||Z||_F^2 / (2 sigma^2) - (m n) log(2 b) - ||S||_1 / (2 b)
        - rank(L) log(2 b_*) - ||L||_* / (2 b_*)
  p   = r (m + n - r) + nnz(S) + (||Z||_F^2 / ||X||_F^2) (m n),   r = rank(L)
  AIC_c = 2 (p - ell) + 2 p (p + 1) / (m n - p - 1)

Readings (where the paper is silent or loose): "log(ell_max)" in the printed AIC_c is the
maximised log-likelihood itself (ell above); b_* = ||L||_* / rank(L) (the Laplace scale of the
singular values, as b is that of S's entries); rank(L) counts singular values above 1e-6 of
the largest (float32 factors); with a mask, m n counts the observed entries.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RANK_TOL = 1e-6


@dataclasses.dataclass
class AICc:
    aicc: float
    loglik: float
    dof: float
    rank: int
    nuclear: float
    s_l1: float
    nnz_s: int
    resid2: float
    x2: float
    count: int


def parts(X, mask, U, V, lam_S):
    X = np.asarray(X, np.float64)
    obs = np.ones(X.shape, bool) if mask is None else np.asarray(mask) != 0
    L = np.asarray(U, np.float64) @ np.asarray(V, np.float64).T
    E = X - L
    S = np.where(obs, np.sign(E) * np.maximum(np.abs(E) - lam_S, 0.0), 0.0)
    Z = np.where(obs, L + S - X, 0.0)
    sv = np.linalg.svd(L, compute_uv=False)
    r = int(np.sum(sv > RANK_TOL * sv[0])) if sv.size and sv[0] > 0 else 0
    return dict(Z=Z, S=S, obs=obs, r=r, nuclear=float(sv[:r].sum()),
                x2=float(np.sum(np.where(obs, X, 0.0) ** 2)))


def aicc(X, mask, U, V, lam_S):
    X = np.asarray(X, np.float64)
    m, n = X.shape
    P = parts(X, mask, U, V, lam_S)
    N = int(P["obs"].sum())
    resid2 = float(np.sum(P["Z"] ** 2))
    s_l1 = float(np.sum(np.abs(P["S"])))
    nnz = int(np.count_nonzero(P["S"]))
    r, nuc, x2 = P["r"], P["nuclear"], P["x2"]
    sigma2 = x2 / N
    b = s_l1 / N
    ell = -(N / 2.0) * math.log(2.0 * math.pi * sigma2) - resid2 / (2.0 * sigma2)
    if b > 0:
        ell += -N * math.log(2.0 * b) - s_l1 / (2.0 * b)
    if r > 0:
        bstar = nuc / r
        ell += -r * math.log(2.0 * bstar) - nuc / (2.0 * bstar)
    p = r * (m + n - r) + nnz + (resid2 / x2) * N
    a = 2.0 * (p - ell) + 2.0 * p * (p + 1.0) / (N - p - 1.0)
    return AICc(aicc=a, loglik=ell, dof=p, rank=r, nuclear=nuc, s_l1=s_l1, nnz_s=nnz, resid2=resid2, x2=x2, count=N)
