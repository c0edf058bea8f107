"""GPU AIC_c (Sec. 5.2) against the FP64 oracle on the same factors: the sums, the rank and
nuclear norm of L, the degrees of freedom and the criterion, for the fused-kernel ranks and a
large rank, with and without a mask."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import aicc as oaicc  # noqa: E402
from paper_1702_02241_gb300 import gen, rpca  # noqa: E402

from gpu_util import dev, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


@pytest.mark.parametrize("m,n,rank,k,mask_p", [(700, 300, 4, 6, None), (500, 350, 3, 5, 0.7), (600, 400, 30, 40, None)])
def test_aicc_matches_oracle(m, n, rank, k, mask_p):
    lam_S = 1.0 / math.sqrt(max(m, n))
    inst = gen.planted(m, n, rank=rank, k=k, p_outlier=0.05, noise=1e-3, lam_L=1.0, lam_S=lam_S, seed=m + k,
                       mask_p=mask_p)
    g = np.random.default_rng(k)
    # Factors of a rank-`rank` L (the surplus columns exactly zero), as a solver would return.
    A = np.linalg.qr(g.normal(size=(m, rank)))[0] * np.linspace(30, 3, rank)
    B = np.linalg.qr(g.normal(size=(n, rank)))[0]
    U = np.zeros((m, k)); U[:, :rank] = A
    V = np.zeros((n, k)); V[:, :rank] = B
    U = U.astype(np.float32); V = V.astype(np.float32)
    P = make_problem(inst.X, inst.mask, k, inst.lam_L, inst.lam_S)
    r = rpca.rpca_aicc(P.ctx, dev(U), dev(V))
    o = oaicc.aicc(inst.X, inst.mask, U, V, inst.lam_S)
    assert r.rank == o.rank == rank
    assert r.count == o.count
    assert abs(r.nnz_s - o.nnz_s) <= 2
    for f in ("resid2", "s_l1", "x2", "nuclear"):
        assert getattr(r, f) == pytest.approx(getattr(o, f), rel=1e-5), f
    assert r.dof == pytest.approx(o.dof, rel=1e-6, abs=2.5)
    assert r.aicc == pytest.approx(o.aicc, rel=1e-5)
    P.close()
