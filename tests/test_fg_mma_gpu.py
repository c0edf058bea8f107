"""GPU parity of the tensor-core form of the fused objective/gradient pass.

The tensor-core kernel (float32 X, fg mode, k <= 8, no mask) forms R^T = X - V U^T and D^T U
as tf32 MMAs with every operand split into a tf32 part and a float32 remainder (three MMAs
per product), and D V on the fp32x2 FMA pipe.  Its results must meet the float32 path's
tolerances against the FP64 oracle: objective <= 1e-6 relative, gradient <= 1e-5 relative
in Frobenius norm.  The planner uses this form only when RPCA_FG_KERNEL=mma is set (it is
slower than the CUDA-core form on the workloads measured); each case checks that the plan
really uses it.  Cases span row passes, column splits, the 16-column
groups' ragged tail, tiny shapes (fewer rows than one warp's 32), k = 1 .. 8, lam_S = inf,
and the full 76800 x 1000 video workload.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_1702_02241_gb300 import gen  # noqa: E402

F_TOL, G_TOL = 1e-6, 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


@pytest.fixture
def mma_only(monkeypatch):
    monkeypatch.setenv("RPCA_FG_KERNEL", "mma")


def run(X, U, V, lam_L, lam_S, expect_mma=True):
    from paper_1702_02241_gb300 import rpca
    from paper_1702_02241_gb300.engine import Problem, from_device_colmajor, to_device_colmajor
    k = U.shape[1]
    P = Problem(X, None, k, lam_L, lam_S)
    kind = rpca.rpca_plan_kernel(P.ctx)["kernel"]
    if expect_mma:
        assert kind == "tensor-core", kind
    f, gU, gV = P.fg(to_device_colmajor(U), to_device_colmajor(V))
    torch.cuda.synchronize()
    out = f, from_device_colmajor(gU, X.shape[0]), from_device_colmajor(gV, X.shape[1])
    P.close()
    return out


def check(res, X, U, V, lam_L, lam_S):
    f, gU, gV = res
    fo, GUo, GVo = core.fg(X, None, U, V, lam_L, lam_S)
    assert abs(f - fo) <= F_TOL * abs(fo), (f, fo, abs(f - fo) / abs(fo))
    G = np.concatenate([gU.ravel(), gV.ravel()])
    Go = np.concatenate([GUo.ravel(), GVo.ravel()])
    assert np.linalg.norm(G - Go) <= G_TOL * np.linalg.norm(Go), np.linalg.norm(G - Go) / np.linalg.norm(Go)


def case(m, n, k, seed, lam_S=0.3, scale=0.5):
    g = np.random.default_rng(seed)
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    U, V = gen.factors(m, n, k, seed + 100, scale=scale)
    return X, U, V, 0.7, lam_S


@pytest.mark.parametrize("m,n,k", [(500, 400, 5), (37, 29, 3), (1001, 77, 1), (3000, 260, 5), (2100, 130, 8),
                                   (64, 8, 2), (9, 5, 4), (4099, 1027, 6), (200, 17, 7), (20000, 300, 4),
                                   (257, 1000, 5), (12345, 33, 8)])
def test_mma_fg_matches_oracle(mma_only, m, n, k):
    X, U, V, lam_L, lam_S = case(m, n, k, seed=m + 3 * n + k)
    check(run(X, U, V, lam_L, lam_S), X, U, V, lam_L, lam_S)


def test_mma_least_squares_limit(mma_only):
    X, U, V, lam_L, _ = case(900, 120, 6, seed=5)
    check(run(X, U, V, lam_L, math.inf), X, U, V, lam_L, math.inf)


def test_mma_residual_near_zero(mma_only):
    """X = U V^T + small noise: the residual is small against u.v, the case where the tf32
    split's rounding matters most (the objective is a sum of squares of small numbers)."""
    m, n, k = 3000, 400, 5
    U, V = gen.factors(m, n, k, seed=8, scale=1.0)
    g = np.random.default_rng(9)
    X = np.asfortranarray((U.astype(np.float64) @ V.astype(np.float64).T
                           + 1e-2 * g.normal(size=(m, n))).astype(np.float32))
    check(run(X, U, V, 1.0, 0.05), X, U, V, 1.0, 0.05)


def test_mma_bitwise_deterministic(mma_only):
    from paper_1702_02241_gb300.engine import Problem, to_device_colmajor
    X, U, V, lam_L, lam_S = case(4000, 500, 5, seed=11)
    P = Problem(X, None, 5, lam_L, lam_S)
    Ud, Vd = to_device_colmajor(U), to_device_colmajor(V)
    a = P.fg(Ud, Vd)
    b = P.fg(Ud, Vd)
    assert a[0] == b[0] and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    P.close()


def test_mma_and_cuda_core_forms_agree(monkeypatch):
    X, U, V, lam_L, lam_S = case(5000, 700, 5, seed=21)
    monkeypatch.setenv("RPCA_FG_KERNEL", "mma")
    a = run(X, U, V, lam_L, lam_S)
    monkeypatch.setenv("RPCA_FG_KERNEL", "cuda")
    b = run(X, U, V, lam_L, lam_S, expect_mma=False)
    assert abs(a[0] - b[0]) <= 1e-6 * abs(b[0])
    Ga = np.concatenate([a[1].ravel(), a[2].ravel()])
    Gb = np.concatenate([b[1].ravel(), b[2].ravel()])
    assert np.linalg.norm(Ga - Gb) <= 1e-5 * np.linalg.norm(Gb)


@pytest.mark.slow
def test_mma_full_video_76800x1000(mma_only):
    inst = gen.video_76800x1000(0)
    U, V = gen.factors(inst.m, inst.n, inst.k, seed=2, scale=0.2)
    check(run(inst.X, U, V, inst.lam_L, inst.lam_S), inst.X, U, V, inst.lam_L, inst.lam_S)
