"""Device L-BFGS solve against the FP64 oracle solve.

Parity is on the converged result (the method is an iteration, trajectories differ):
F within 1e-6 relative, ||L - L_oracle||_F / ||L_oracle||_F <= 1e-4, both certificates
<= 1e-4, and the S-support symmetric difference <= 1e-4 of |Omega| counting only entries
whose | |X - L| - lam_S | > 1e-6.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import certificate as ocert  # noqa: E402
from oracle import convex, core, lbfgs, sketch  # noqa: E402
from paper_1702_02241_gb300 import gen, rpca  # noqa: E402

from gpu_util import dev, empty_factors, host, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def oracle_solution(X, mask, k, lam_L, lam_S, seed=11):
    Om = gen.gaussian(X.shape[1], k + 10, seed=seed)
    U0, V0 = sketch.rsvd_init(X, mask, k, Om)
    return lbfgs.solve(X, mask, U0, V0, lam_L, lam_S, gtol=1e-11, max_iter=5000), U0, V0


def check_solution(X, mask, lam_L, lam_S, res, U, V, ref):
    L = U @ V.T
    Lr = ref.U @ ref.V.T
    assert res.F == pytest.approx(ref.f, rel=1e-6)
    assert core.objective(X, mask, U, V, lam_L, lam_S) == pytest.approx(ref.f, rel=1e-6)
    assert np.linalg.norm(L - Lr) <= 1e-4 * np.linalg.norm(Lr)
    assert res.cert.cert_rel <= 1e-4
    assert ocert.certificate(X, mask, U, V, lam_L, lam_S).cert_rel <= 1e-4
    Xd = X.astype(np.float64)
    Rg, Rr = np.abs(Xd - L), np.abs(Xd - Lr)
    M = np.ones(X.shape, bool) if mask is None else mask != 0
    clear = M & (np.abs(Rr - lam_S) > 1e-6)
    diff = np.sum(((Rg > lam_S) != (Rr > lam_S)) & clear)
    assert diff <= 1e-4 * M.sum()


@pytest.mark.parametrize("init", ["user", "sketch", "random"])
def test_solve_planted_500x400(init):
    inst = gen.planted_500x400(0)
    ref, U0, V0 = oracle_solution(inst.X, None, inst.k, inst.lam_L, inst.lam_S)
    kind = {"user": rpca.RPCA_INIT_USER, "sketch": rpca.RPCA_INIT_SKETCH, "random": rpca.RPCA_INIT_RANDOM}[init]
    P = make_problem(inst.X, None, inst.k, inst.lam_L, inst.lam_S, init=kind, max_iter=3000, cert_every=10)
    if init == "user":
        Ud, Vd = dev(U0), dev(V0)
    else:
        Ud, Vd = empty_factors(inst.m, inst.n, inst.k)
    res = P.solve(Ud, Vd)
    assert res.status == rpca.RPCA_OK, (rpca.rpca_last_error(P.ctx), res.cert.asdict())
    check_solution(inst.X, None, inst.lam_L, inst.lam_S, res, host(Ud, inst.m), host(Vd, inst.n), ref)
    P.close()


def test_solve_masked():
    inst = gen.planted(600, 300, rank=4, k=8, seed=3, mask_p=0.7)
    ref, U0, V0 = oracle_solution(inst.X, inst.mask, inst.k, inst.lam_L, inst.lam_S)
    P = make_problem(inst.X, inst.mask, inst.k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_USER, max_iter=4000,
                     cert_every=10)
    Ud, Vd = dev(U0), dev(V0)
    res = P.solve(Ud, Vd)
    assert res.status == rpca.RPCA_OK, (rpca.rpca_last_error(P.ctx), res.cert.asdict())
    check_solution(inst.X, inst.mask, inst.lam_L, inst.lam_S, res, host(Ud, inst.m), host(Vd, inst.n), ref)
    P.close()


def test_solve_least_squares_matches_svt_closed_form():
    g = np.random.default_rng(0)
    m, n = 220, 160
    X = np.asfortranarray((g.normal(size=(m, 3)) @ g.normal(size=(3, n)) + 0.05 * g.normal(size=(m, n)))
                          .astype(np.float32))
    lam_L = 3.0
    Ls = convex.svt(X.astype(np.float64), lam_L)
    Fc = core.convex_objective(X, None, Ls, lam_L, math.inf)
    P = make_problem(X, None, 6, lam_L, math.inf, init=rpca.RPCA_INIT_SKETCH, max_iter=3000, cert_every=10)
    Ud, Vd = empty_factors(m, n, 6)
    res = P.solve(Ud, Vd)
    assert res.status == rpca.RPCA_OK, (rpca.rpca_last_error(P.ctx), res.cert.asdict())
    U, V = host(Ud, m), host(Vd, n)
    assert res.F == pytest.approx(Fc, rel=1e-6)
    assert np.linalg.norm(U @ V.T - Ls) <= 1e-4 * np.linalg.norm(Ls)
    P.close()


def test_solve_k1():
    g = np.random.default_rng(2)
    m, n = 150, 100
    X = np.asfortranarray((np.outer(g.normal(size=m), g.normal(size=n)) * 2 + 0.01 * g.normal(size=(m, n)))
                          .astype(np.float32))
    ref, U0, V0 = oracle_solution(X, None, 1, 1.0, 0.1)
    P = make_problem(X, None, 1, 1.0, 0.1, init=rpca.RPCA_INIT_USER, max_iter=2000, cert_every=10)
    Ud, Vd = dev(U0), dev(V0)
    res = P.solve(Ud, Vd)
    assert res.status == rpca.RPCA_OK, (rpca.rpca_last_error(P.ctx), res.cert.asdict())
    check_solution(X, None, 1.0, 0.1, res, host(Ud, m), host(Vd, n), ref)
    P.close()


def test_solve_reports_not_converged_when_capped():
    inst = gen.planted_500x400(0)
    P = make_problem(inst.X, None, inst.k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_RANDOM, max_iter=3,
                     cert_every=0)
    Ud, Vd = empty_factors(inst.m, inst.n, inst.k)
    res = P.solve(Ud, Vd)
    assert res.status == rpca.RPCA_ENOTCONV and res.iters == 3
    P.close()


def test_host_driven_solver_matches_graph(monkeypatch):
    """RPCA_SOLVER_GRAPH=0 runs the same kernels from a host loop: identical iterates."""
    inst = gen.planted_500x400(1)
    out = []
    for flag in (None, "0"):
        if flag is None:
            monkeypatch.delenv("RPCA_SOLVER_GRAPH", raising=False)
        else:
            monkeypatch.setenv("RPCA_SOLVER_GRAPH", flag)
        P = make_problem(inst.X, None, inst.k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH,
                         max_iter=3000, cert_every=10)
        Ud, Vd = empty_factors(inst.m, inst.n, inst.k)
        res = P.solve(Ud, Vd)
        out.append((res.status, res.iters, res.evals, res.F, host(Ud, inst.m)))
        P.close()
    (s0, i0, e0, f0, U0), (s1, i1, e1, f1, U1) = out
    assert s0 == s1 == rpca.RPCA_OK
    assert (i0, e0) == (i1, e1)
    assert f0 == f1
    assert np.array_equal(U0, U1)
