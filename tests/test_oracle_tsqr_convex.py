"""Pins of the TSQR oracle (oracle/tsqr.py) and of the Sec. 6.1 convex baseline
(oracle/convex.py: rsvd_svt, fista_rsvd), each against something other than the oracle's own
formula:

* TSQR equals the library QR normalised to a non-negative diagonal (the unique QR of a full-rank
  matrix), whatever the tree shape; R^T R = A^T A (the Cholesky factor of the Gram matrix);
  Q R = A and Q^T Q = I also for rank-deficient inputs;
* the rSVD thresholding of a matrix of exact rank r < l equals the exact singular-value
  thresholding (a full SVD), and its singular values are the matrix's;
* the FISTA-rSVD iteration reaches the optimum of the exact-SVD FISTA reference and of the
  factored problem solved by L-BFGS (the two programs share their optimum when k >= rank L*,
  by the factored form of the nuclear norm, Sec. 2), and its iterates converge.
"""
import numpy as np
import pytest

from oracle import convex, core, lbfgs
from oracle.tsqr import tsqr


def _qr_pos(A):
    q, r = np.linalg.qr(A)
    d = np.where(np.diag(r) < 0, -1.0, 1.0)
    return q * d, d[:, None] * r


@pytest.mark.parametrize("rows,l,block,fan", [(300, 7, 20, 3), (300, 7, 1000, 4), (97, 5, 9, 2), (64, 16, 16, 8),
                                              (16, 16, 64, 4), (1000, 1, 30, 5)])
def test_tsqr_is_the_positive_diagonal_qr(rows, l, block, fan):
    g = np.random.default_rng(rows + l)
    A = g.normal(size=(rows, l)) * np.logspace(0, -3, l)
    Q, R = tsqr(A, block_rows=block, fan_in=fan)
    q2, r2 = _qr_pos(A)
    assert np.abs(Q - q2).max() <= 1e-10
    assert np.abs(R - r2).max() <= 1e-12 * np.abs(A).max() * rows
    assert np.all(np.diag(R) >= 0) and np.allclose(np.tril(R, -1), 0)
    assert np.abs(R.T @ R - A.T @ A).max() <= 1e-12 * np.abs(A.T @ A).max()


def test_tsqr_tree_shapes_agree():
    g = np.random.default_rng(5)
    A = g.normal(size=(777, 9))
    ref = tsqr(A, block_rows=777)
    for block, fan in [(9, 2), (13, 3), (50, 7), (100, 16)]:
        Q, R = tsqr(A, block_rows=block, fan_in=fan)
        assert np.abs(Q - ref[0]).max() <= 1e-12
        assert np.abs(R - ref[1]).max() <= 1e-12


def test_tsqr_rank_deficient_input():
    g = np.random.default_rng(6)
    A = g.normal(size=(200, 6))
    A[:, 2] = 0.0
    A[:, 4] = A[:, 1]
    Q, R = tsqr(A, block_rows=17, fan_in=3)
    assert np.abs(Q @ R - A).max() <= 1e-12
    assert np.abs(Q.T @ Q - np.eye(6)).max() <= 1e-12
    assert abs(R[2, 2]) <= 1e-12 and abs(R[4, 4]) <= 1e-12


def test_rsvd_svt_is_exact_on_low_rank_matrices():
    g = np.random.default_rng(7)
    m, n, r, l = 120, 80, 4, 7
    Z = g.normal(size=(m, r)) @ np.diag([9.0, 5.0, 2.5, 1.2]) @ g.normal(size=(r, n))
    Om = g.normal(size=(n, l))
    lam = 1.0
    left, s, right, st = convex.rsvd_svt(Z, Om, lam, q=0)
    sv = np.linalg.svd(Z, compute_uv=False)
    assert np.abs(s[:r] - sv[:r]).max() <= 1e-10 * sv[0]
    assert np.abs(s[r:]).max() <= 1e-10 * sv[0]
    assert np.abs((left * st) @ right.T - convex.svt(Z, lam)).max() <= 1e-10 * sv[0]
    assert np.abs(left.T @ left - np.eye(l)).max() <= 1e-10
    assert np.abs(right.T @ right - np.eye(l)).max() <= 1e-10


def test_rsvd_power_iterations_find_the_top_singular_values():
    g = np.random.default_rng(8)
    m, n, l = 150, 90, 6
    U, _ = np.linalg.qr(g.normal(size=(m, n)))
    V, _ = np.linalg.qr(g.normal(size=(n, n)))
    sv = 2.0 ** -np.arange(n, dtype=float) * 40.0
    Z = (U * sv) @ V.T
    _, s, _, _ = convex.rsvd_svt(Z, g.normal(size=(n, l)), 0.0, q=12)
    assert np.abs(s[:4] - sv[:4]).max() <= 1e-8 * sv[0]


def _case(seed=0, m=40, n=30, rank=2, p=0.08):
    g = np.random.default_rng(seed)
    L0 = g.normal(size=(m, rank)) @ g.normal(size=(rank, n))
    S0 = np.where(g.random((m, n)) < p, g.uniform(1, 5, (m, n)) * np.sign(g.normal(size=(m, n))), 0.0)
    return L0 + S0 + 0.01 * g.normal(size=(m, n))


@pytest.mark.parametrize("masked", [False, True])
def test_fista_rsvd_reaches_the_convex_and_factored_optimum(masked):
    X = _case(1)
    m, n = X.shape
    g = np.random.default_rng(3)
    mask = (g.random((m, n)) < 0.8).astype(np.uint8) if masked else None
    lam_L, lam_S = 2.0, 0.3
    steps = convex.fista_rsvd(X, mask, lam_L, lam_S, g.normal(size=(n, 6)), q=1, iters=600)
    F_end = steps[-1].F
    L_ref = convex.fista(X, mask, lam_L, lam_S, iters=20000, tol=1e-13)
    F_ref = core.convex_objective(X, mask, L_ref, lam_L, lam_S)
    assert abs(F_end - F_ref) <= 1e-8 * abs(F_ref)
    assert np.abs(steps[-1].L - L_ref).max() <= 1e-5 * np.abs(L_ref).max()
    assert steps[-1].rel <= 1e-8
    # The factored problem at k = 5 >= rank L*: the same optimum value (Sec. 2).
    k = 5
    r = lbfgs.solve(X, mask, g.normal(size=(m, k)) * 0.1, g.normal(size=(n, k)) * 0.1, lam_L, lam_S,
                    gtol=1e-12, max_iter=5000)
    F_fact = core.objective(X, mask, r.U, r.V, lam_L, lam_S)
    assert abs(F_end - F_fact) <= 1e-7 * abs(F_fact)
    # The first step from L = 0, with enough power iterations for the sketch to converge, is
    # the exact prox of the gradient point Z = 0 - grad phi(0) = P_Omega clip(X).
    Z0 = -core.D_of_R(-X, mask, lam_S)
    first = convex.fista_rsvd(X, mask, lam_L, lam_S, g.normal(size=(n, 6)), q=30, iters=2)
    assert np.abs(first[1].L - convex.svt(Z0, lam_L)).max() <= 1e-9 * np.abs(Z0).max()
