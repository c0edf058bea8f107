"""GPU Frank-Wolfe with marginalization (Sec. 6.2, Algorithm 1) against the FP64 oracle.

* Trajectory parity: with enough power iterations for the top singular pair, the device's
  objective sequence, t and final L follow the oracle's (which takes the pair from a dense
  SVD) to float32 accuracy, with and without a mask.
* With the default 2 warm-started power iterations: F never increases, ||L||_* <= t, F stays
  above the certified optimum of the same program and moves toward it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import frank_wolfe as ofw  # noqa: E402
from paper_1702_02241_gb300 import rpca  # noqa: E402
from paper_1702_02241_gb300.engine import ld_for  # noqa: E402

from gpu_util import make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def _case(m, n, seed, mask_p=None, scales=(3.0, 2.0, 1.2)):
    g = np.random.default_rng(seed)
    r = len(scales)
    A = g.normal(size=(m, r)) * np.array(scales)
    L0 = A @ g.normal(size=(r, n))
    S0 = np.where(g.random((m, n)) < 0.08, g.uniform(1, 5, (m, n)) * np.sign(g.normal(size=(m, n))), 0.0)
    X = np.asfortranarray((L0 + S0 + 0.01 * g.normal(size=(m, n))).astype(np.float32))
    mask = None if mask_p is None else np.asfortranarray((g.random((m, n)) < mask_p).astype(np.uint8))
    return X, mask


def _dense(m, n):
    ld = ld_for(m)
    return torch.zeros((n, ld), dtype=torch.float32, device="cuda"), ld


@pytest.mark.parametrize("m,n,mask_p", [(301, 123, None), (257, 190, 0.6)])
def test_trajectory_matches_oracle(m, n, mask_p):
    # A planted rank-1 part keeps the gradient's two leading singular values apart (ratio
    # <= 0.89 over these iterations), so the warm-started power iteration reaches the top pair
    # the oracle takes from a dense SVD.
    X, mask = _case(m, n, m + n, mask_p, scales=(3.0,))
    lam_L, lam_S = 3.0, 0.3
    P = make_problem(X, mask, 1, lam_L, lam_S)
    L, ld = _dense(m, n)
    iters = 12
    r, log = rpca.rpca_fw_solve(P.ctx, L, ld, iters, 0.0, 80)
    steps = ofw.solve(X, mask, lam_L, lam_S, iters)
    assert r.iters == iters
    F_or = [ofw.objective(X, mask, np.zeros((m, n)), 0.0, lam_L, lam_S)] + [s.F for s in steps[:-1]]
    for (Fd, gap, s1, eta), Fo, so in zip(log, F_or, steps):
        assert Fd == pytest.approx(Fo, rel=2e-5)
        assert s1 == pytest.approx(so.sigma1, rel=1e-4)
        assert eta == pytest.approx(so.eta, rel=2e-3, abs=1e-5)
    Ld = L.cpu().numpy()[:, :m].T.astype(np.float64)
    assert np.linalg.norm(Ld - steps[-1].L) <= 2e-3 * np.linalg.norm(steps[-1].L)
    assert r.t == pytest.approx(steps[-1].t, rel=2e-3)
    assert r.F == pytest.approx(steps[-1].F, rel=1e-4)
    P.close()


def test_default_power_iterations_monotone_and_gap_shrinks():
    m, n = 3000, 400
    X, _ = _case(m, n, 5)
    lam_L, lam_S = 3.0, 0.05
    P = make_problem(X, None, 1, lam_L, lam_S)
    L, ld = _dense(m, n)
    r, log = rpca.rpca_fw_solve(P.ctx, L, ld, 300, 0.0, 2)
    Fs = [row[0] for row in log] + [r.F]
    assert all(b <= a * (1 + 1e-6) for a, b in zip(Fs, Fs[1:]))
    nuc = np.linalg.svd(L.cpu().numpy()[:, :m].astype(np.float64), compute_uv=False).sum()
    assert nuc <= r.t * (1 + 1e-4)
    # Progress toward the optimum of the same convex program, F* from a certified Split-SPCP
    # solve (its factored objective equals lam_L ||L||_* + phi(L) at a balanced solution).
    S = make_problem(X, None, 8, lam_L, lam_S, init=rpca.RPCA_INIT_SKETCH, max_iter=3000, cert_every=10)
    U = torch.zeros((8, m), dtype=torch.float32, device="cuda")
    V = torch.zeros((8, n), dtype=torch.float32, device="cuda")
    rs = S.solve(U, V)
    assert rs.status == rpca.RPCA_OK
    F0 = log[0][0]
    assert r.F >= rs.F * (1 - 1e-6)
    assert F0 - r.F >= 0.3 * (F0 - rs.F)
    S.close()
    P.close()
