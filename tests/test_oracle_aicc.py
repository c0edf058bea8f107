"""Pins of the AIC_c oracle (oracle/aicc.py, Sec. 5.2) against independent routes:

* the Gaussian part of the log-likelihood equals a sum of scipy.stats.norm.logpdf, the printed
  Laplace parts equal sums of scipy.stats.laplace.logpdf at scale 2b plus m n log 2 (the
  printed term divides ||S||_1 by 2b), and likewise for the singular values with b_*;
* a 3 x 2 worked example: rank, nnz(S), degrees of freedom and AIC_c by hand.
"""
import math

import numpy as np
import pytest

from oracle import aicc

scipy_stats = pytest.importorskip("scipy.stats")


def _case(seed=0, m=30, n=20, k=3):
    g = np.random.default_rng(seed)
    U = g.normal(size=(m, k))
    V = g.normal(size=(n, k))
    X = U @ V.T + np.where(g.random((m, n)) < 0.2, 3 * g.normal(size=(m, n)), 0.0) + 0.05 * g.normal(size=(m, n))
    return X, U, V


def test_loglik_terms_match_scipy():
    X, U, V = _case()
    lam_S = 0.3
    r = aicc.aicc(X, None, U, V, lam_S)
    P = aicc.parts(X, None, U, V, lam_S)
    m, n = X.shape
    N = m * n
    sigma = math.sqrt(r.x2 / N)
    b = r.s_l1 / N
    gauss = scipy_stats.norm.logpdf(P["Z"], scale=sigma).sum()
    lap = scipy_stats.laplace.logpdf(P["S"], scale=2 * b).sum() + N * math.log(2.0)
    sv = np.linalg.svd(U @ V.T, compute_uv=False)[: r.rank]
    bstar = sv.sum() / r.rank
    lap_L = scipy_stats.laplace.logpdf(sv, scale=2 * bstar).sum() + r.rank * math.log(2.0)
    assert r.loglik == pytest.approx(gauss + lap + lap_L, rel=1e-12)
    assert r.rank == 3


def test_worked_example_3x2():
    X = np.array([[2.0, 1.0], [1.0, 5.0], [0.0, -1.0]])
    U = np.array([[1.0], [0.5], [0.0]])
    V = np.array([[2.0], [1.0]])        # L = [[2, 1], [1, 0.5], [0, 0]]
    lam_S = 1.0
    r = aicc.aicc(X, None, U, V, lam_S)
    # X - L = [[0, 0], [0, 4.5], [0, -1]]: S = shrink(., 1) = [[0, 0], [0, 3.5], [0, 0]]
    assert r.rank == 1 and r.nnz_s == 1 and r.s_l1 == pytest.approx(3.5)
    # Z = L + S - X = [[0, 0], [0, -1], [0, 1]]: ||Z||^2 = 2; ||X||^2 = 4 + 1 + 1 + 25 + 0 + 1 = 32
    assert r.resid2 == pytest.approx(2.0) and r.x2 == pytest.approx(32.0)
    p = 1 * (3 + 2 - 1) + 1 + (2.0 / 32.0) * 6
    assert r.dof == pytest.approx(p)
    nuc = math.sqrt(5.0) * math.sqrt(1.25)  # sigma_1 of L = ||u|| ||v||
    ell = (-(6 / 2) * math.log(2 * math.pi * 32 / 6) - 2.0 / (2 * 32 / 6)
           - 6 * math.log(2 * 3.5 / 6) - 3.5 / (2 * 3.5 / 6) - math.log(2 * nuc) - nuc / (2 * nuc))
    assert r.loglik == pytest.approx(ell, rel=1e-12)
    assert r.aicc == pytest.approx(2 * (p - ell) + 2 * p * (p + 1) / (6 - p - 1), rel=1e-12)
