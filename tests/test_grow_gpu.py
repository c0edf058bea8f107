"""Dynamic rank increase (Sec. 4.1) on the GPU.

* The top singular pair of P_U1perp D P_V1perp from the certificate's Lanczos bases against
  the oracle's dense SVD (sigma_1 to the certificate's 1e-3, the pair up to a common sign).
* A solve started with k below the rank of the solution grows k until the certificate holds
  and reaches the objective of a solve with enough rank from the start.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import certificate as ocert  # noqa: E402
from paper_1702_02241_gb300 import gen, rpca  # noqa: E402

from gpu_util import dev, empty_factors, host, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def _planted(m, n, rank, seed):
    lam_S = 1.0 / math.sqrt(max(m, n))
    return gen.planted(m, n, rank=rank, k=rank, p_outlier=0.05, noise=1e-3,
                       lam_L=lam_S * (math.sqrt(m) + math.sqrt(n)), lam_S=lam_S, seed=seed)


def test_perp_direction_matches_oracle():
    inst = _planted(900, 150, 4, 3)
    m, n = inst.m, inst.n
    U, V = gen.factors(m, n, 2, seed=5, scale=0.5)
    P = make_problem(inst.X, None, 2, inst.lam_L, inst.lam_S)
    c = P.certificate(dev(U), dev(V))
    u = torch.zeros(m, dtype=torch.float32, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    s1 = rpca.rpca_perp_direction(P.ctx, u, v)
    so, uo, vo = ocert.perp_top_pair(inst.X, None, U, V, inst.lam_L, inst.lam_S)
    assert s1 == pytest.approx(so, rel=1e-3) and c.sigma1_perp == pytest.approx(so, rel=1e-3)
    ud, vd = u.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    cu, cv = ud @ uo, vd @ vo
    assert abs(abs(cu) - 1) < 1e-3 and abs(abs(cv) - 1) < 1e-3 and cu * cv > 0
    P.close()


def test_solve_grows_rank_to_the_certificate():
    inst = _planted(2000, 220, 4, 7)
    m, n = inst.m, inst.n
    kmax = 8
    P = make_problem(inst.X, None, 1, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH, max_iter=3000,
                     cert_every=10)
    U = torch.zeros((kmax, m), dtype=torch.float32, device="cuda")
    V = torch.zeros((kmax, n), dtype=torch.float32, device="cuda")
    r, k = rpca.rpca_solve_grow(P.ctx, U, V, kmax)
    assert r.status == rpca.RPCA_OK and 4 <= k <= kmax
    ref = make_problem(inst.X, None, kmax, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH, max_iter=3000,
                       cert_every=10)
    U8, V8 = empty_factors(m, n, kmax)
    r8 = ref.solve(U8, V8)
    assert r8.status == rpca.RPCA_OK
    assert r.F == pytest.approx(r8.F, rel=1e-6)
    L = host(U, m)[:, :k] @ host(V, n)[:, :k].T
    L8 = host(U8, m) @ host(V8, n).T
    assert np.linalg.norm(L - L8) <= 1e-3 * np.linalg.norm(L8)
    ref.close()
    P.close()


def test_grow_does_nothing_when_certified():
    inst = _planted(800, 120, 3, 9)
    m, n = inst.m, inst.n
    P = make_problem(inst.X, None, 5, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH, max_iter=3000,
                     cert_every=10)
    U = torch.zeros((8, m), dtype=torch.float32, device="cuda")
    V = torch.zeros((8, n), dtype=torch.float32, device="cuda")
    r, k = rpca.rpca_solve_grow(P.ctx, U, V, 8)
    assert r.status == rpca.RPCA_OK and k == 5
    assert torch.all(U[5:] == 0) and torch.all(V[5:] == 0)
    P.close()


def test_perp_directions_match_oracle():
    """The leading pairs (values and subspace) from the certificate's Lanczos bases."""
    inst = _planted(1200, 200, 6, 8)
    m, n = inst.m, inst.n
    U, V = gen.factors(m, n, 1, seed=6, scale=0.5)
    P = make_problem(inst.X, None, 1, inst.lam_L, inst.lam_S)
    P.certificate(dev(U), dev(V))
    Ud = torch.zeros((4, m), dtype=torch.float32, device="cuda")
    Vd = torch.zeros((4, n), dtype=torch.float32, device="cuda")
    sig = rpca.rpca_perp_directions(P.ctx, 4, Ud, m, Vd, n)
    so, uo, vo = ocert.perp_top_pairs(inst.X, None, U, V, inst.lam_L, inst.lam_S, 4)
    assert len(sig) == 4
    assert np.allclose(sig, so, rtol=2e-3)
    ud = host(Ud, m)
    vd = host(Vd, n)
    M = ocert.perp_matrix(inst.X, None, U, V, inst.lam_L, inst.lam_S)
    for i in range(4):  # each device pair is a singular pair of M (whatever the value spacing)
        assert np.linalg.norm(M @ vd[:, i] - sig[i] * ud[:, i]) <= 2e-2 * sig[i]
        assert np.linalg.norm(M.T @ ud[:, i] - sig[i] * vd[:, i]) <= 2e-2 * sig[i]
    P.close()
