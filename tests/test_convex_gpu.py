"""GPU TSQR and the Sec. 6.1 convex baseline (FISTA with a TSQR-based rSVD prox) against the
FP64 oracle (oracle/tsqr.py, oracle/convex.py).

* TSQR: Q and R equal the oracle's positive-diagonal QR of the same float32 input to float32
  accuracy, over shapes that give one leaf, many leaves, several reduction levels and ragged
  last leaves; a rank-deficient input still gives an orthonormal Q with Q R = A.
* Trajectory parity: the objective, relative change and rank of every iterate, and the final
  iterate, follow the oracle's fista_rsvd on the same Omega_0, with and without a mask, for sketch
  widths on both sides of the float64 / float32 switch of the small SVD.
* Convergence: the convex solver reaches the optimum of the factored problem certified by the
  Split-SPCP solver on the same data (the two programs share their optimum, Sec. 2).
* Edge cases: max_iter = 0, a lam_L above sigma_1 (L = 0 is optimal), l = 1, l = min(m, n),
  and the argument checks.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import convex as ocv  # noqa: E402
from oracle import core  # noqa: E402
from oracle.tsqr import tsqr as otsqr  # noqa: E402
from paper_1702_02241_gb300 import rpca  # noqa: E402
from paper_1702_02241_gb300.engine import ld_for  # noqa: E402

from gpu_util import dev, host, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def _case(m, n, seed, mask_p=None, scales=(3.0, 2.0, 1.2), p=0.08):
    g = np.random.default_rng(seed)
    r = len(scales)
    A = g.normal(size=(m, r)) * np.array(scales)
    L0 = A @ g.normal(size=(r, n))
    S0 = np.where(g.random((m, n)) < p, g.uniform(1, 5, (m, n)) * np.sign(g.normal(size=(m, n))), 0.0)
    X = np.asfortranarray((L0 + S0 + 0.01 * g.normal(size=(m, n))).astype(np.float32))
    mask = None if mask_p is None else np.asfortranarray((g.random((m, n)) < mask_p).astype(np.uint8))
    return X, mask


def _omega(n, l, seed):
    return np.random.default_rng(seed).standard_normal((n, l)).astype(np.float32)


@pytest.mark.parametrize("rows,l", [(37, 5), (40, 32), (1000, 8), (5000, 1), (20011, 20), (77123, 16),
                                    (150000, 32)])
def test_tsqr_matches_oracle(rows, l):
    g = np.random.default_rng(rows + l)
    A = (g.normal(size=(rows, l)) * np.logspace(0, -2, l)).astype(np.float32)
    P = make_problem(np.ones((8, 8), np.float32), None, 1, 1.0, 1.0)
    Ad = dev(A)
    Qd = torch.zeros((l, rows), dtype=torch.float32, device="cuda")
    Rd = torch.zeros((l, l), dtype=torch.float32, device="cuda")
    rpca.rpca_tsqr(P.ctx, Ad, rows, rows, l, Qd, rows, Rd)
    Q = host(Qd, rows)
    R = Rd.double().cpu().numpy().T
    Qo, Ro = otsqr(A.astype(np.float64))
    assert np.abs(Q - Qo).max() <= 1e-4
    assert np.abs(R - Ro).max() <= 2e-5 * np.abs(Ro).max()
    assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)
    assert np.abs(Q.T @ Q - np.eye(l)).max() <= 2e-5
    assert np.abs(Q @ R - A).max() <= 2e-5 * np.abs(A).max()
    P.close()


def test_tsqr_rank_deficient():
    g = np.random.default_rng(3)
    rows, l = 3001, 7
    A = g.normal(size=(rows, l)).astype(np.float32)
    A[:, 2] = 0.0
    A[:, 5] = A[:, 1]
    P = make_problem(np.ones((8, 8), np.float32), None, 1, 1.0, 1.0)
    Qd = torch.zeros((l, rows), dtype=torch.float32, device="cuda")
    Rd = torch.zeros((l, l), dtype=torch.float32, device="cuda")
    rpca.rpca_tsqr(P.ctx, dev(A), rows, rows, l, Qd, rows, Rd)
    Q, R = host(Qd, rows), Rd.double().cpu().numpy().T
    assert np.abs(Q.T @ Q - np.eye(l)).max() <= 2e-5
    assert np.abs(Q @ R - A).max() <= 2e-5 * np.abs(A).max()
    assert abs(R[2, 2]) <= 1e-5 and abs(R[5, 5]) <= 1e-4
    P.close()


def _run(X, mask, lam_L, lam_S, l, Om, iters, q=1, tol=0.0):
    m, n = X.shape
    P = make_problem(X, mask, 1, lam_L, lam_S)
    ld = ld_for(m)
    L = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    r, log = rpca.rpca_convex_solve(P.ctx, L, ld, l, dev(Om), iters, tol, q)
    Ld = L[:, :m].double().cpu().numpy().T
    P.close()
    return r, log, Ld


@pytest.mark.parametrize("m,n,mask_p,l", [(301, 123, None, 6), (257, 190, 0.6, 8), (513, 77, None, 20),
                                          (130, 64, 0.8, 12)])
def test_trajectory_matches_oracle(m, n, mask_p, l):
    X, mask = _case(m, n, m + n, mask_p)
    lam_L, lam_S = 2.5, 0.3
    Om = _omega(n, l, 7)
    iters = 25
    r, log, Ld = _run(X, mask, lam_L, lam_S, l, Om, iters)
    steps = ocv.fista_rsvd(X.astype(np.float64), mask, lam_L, lam_S, Om.astype(np.float64), q=1, iters=iters + 1)
    assert r.iters == iters and len(log) == iters + 1
    for k, (row, so) in enumerate(zip(log, steps)):
        F, rel, rank, _ = row
        assert F == pytest.approx(so.F, rel=2e-5), k
        if k >= 1:
            assert rel == pytest.approx(so.rel, rel=2e-3, abs=1e-6), k
            assert int(rank) == steps[k - 1].rank, k
    Lo = steps[iters].L
    assert np.linalg.norm(Ld - Lo) <= 1e-4 * np.linalg.norm(Lo)
    assert r.F == pytest.approx(steps[iters].F, rel=2e-5)
    assert r.nuclear == pytest.approx(np.linalg.svd(Lo, compute_uv=False).sum(), rel=1e-4)


@pytest.mark.parametrize("mask_p", [None, 0.7])
def test_converges_to_the_certified_factored_optimum(mask_p):
    m, n = 4000, 300
    X, mask = _case(m, n, 11, mask_p)
    lam_S = 1.0 / np.sqrt(max(m, n))
    lam_L = lam_S * (np.sqrt(m) + np.sqrt(n))  # the solution has the planted rank 3 < l
    # Stop at a relative change of 1e-6: float32 iterates settle at a few 1e-7.
    r, log, Ld = _run(X, mask, lam_L, lam_S, 8, _omega(n, 8, 1), 2000, q=1, tol=1e-6)
    assert r.rel_change <= 1e-6 and r.truncated == 0
    P = make_problem(X, mask, 4, lam_L, lam_S, init=rpca.RPCA_INIT_SKETCH, max_iter=5000, cert_tol=1e-4)
    U = torch.zeros((4, m), dtype=torch.float32, device="cuda")
    V = torch.zeros((4, n), dtype=torch.float32, device="cuda")
    res = P.solve(U, V)
    assert res.status == rpca.RPCA_OK
    F_star = res.F
    assert r.F == pytest.approx(F_star, rel=1e-5)
    # The returned L and its reported objective agree with the oracle's objective of it.
    assert r.F == pytest.approx(core.convex_objective(X.astype(np.float64), mask, Ld, lam_L, lam_S), rel=1e-5)
    P.close()


def test_edge_cases():
    m, n = 203, 57
    X, _ = _case(m, n, 4)
    lam_S = 0.3
    # max_iter = 0: F = phi(0), nothing else done.
    r, log, Ld = _run(X, None, 2.0, lam_S, 4, _omega(n, 4, 2), 0)
    assert r.iters == 0 and np.all(Ld == 0)
    assert r.F == pytest.approx(core.phi_of_R(-X.astype(np.float64), None, lam_S), rel=1e-6)
    # lam_L above sigma_1 of P_Omega clip(X): L = 0 is optimal; one step, rank 0, stop.
    s1 = np.linalg.svd(np.clip(X.astype(np.float64), -lam_S, lam_S), compute_uv=False)[0]
    r, log, Ld = _run(X, None, 1.5 * s1, lam_S, 4, _omega(n, 4, 2), 50, tol=1e-9)
    assert r.iters == 1 and r.rank == 0 and np.all(Ld == 0)
    # l = 1 and l = min(m, n) follow the oracle.
    for l in (1, 32):
        mm, nn = (203, 57) if l == 1 else (48, 32)
        Xs, _ = _case(mm, nn, l)
        Om = _omega(nn, l, 5)
        r, log, Ld = _run(Xs, None, 2.0, lam_S, l, Om, 8)
        steps = ocv.fista_rsvd(Xs.astype(np.float64), None, 2.0, lam_S, Om.astype(np.float64), q=1, iters=9)
        assert np.linalg.norm(Ld - steps[8].L) <= 2e-4 * max(1.0, np.linalg.norm(steps[8].L))
    # Argument checks.
    P = make_problem(X, None, 1, 2.0, lam_S)
    ld = ld_for(m)
    L = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    Om = dev(_omega(n, 4, 1))
    for l in (0, 33, n + 1):
        with pytest.raises(rpca.RpcaError):
            rpca.rpca_convex_solve(P.ctx, L, ld, l, Om, 5)
    with pytest.raises(rpca.RpcaError):
        rpca.rpca_convex_solve(P.ctx, L, m - 1, 4, Om, 5)
    with pytest.raises(rpca.RpcaError):
        rpca.rpca_tsqr(P.ctx, Om, n, 3, 4, Om, n)
    P.close()
