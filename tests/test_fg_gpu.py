"""GPU parity of the fused objective/gradient kernel against the FP64 oracle.

Tolerances (FP32 path): objective <= 1e-6 relative, gradient <= 1e-5 relative in Frobenius
norm, on the same seeded inputs.  Cases span several row blocks and column splits, ragged
tails, k = 1 .. 16, masked / fully-masked rows and columns / empty mask, lam_S = inf, and the
full 76800 x 1000 video workload in the launch configuration the benchmark uses.
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


def run_case(X, mask, U, V, lam_L, lam_S):
    from paper_1702_02241_gb300.engine import Problem, from_device_colmajor, to_device_colmajor
    k = U.shape[1]
    P = Problem(X, mask, k, lam_L, lam_S)
    Ud, Vd = to_device_colmajor(U), to_device_colmajor(V)
    f, gU, gV = P.fg(Ud, Vd)
    torch.cuda.synchronize()
    fo, GUo, GVo = core.fg(X, mask, U, V, lam_L, lam_S)
    gUh = from_device_colmajor(gU, X.shape[0])
    gVh = from_device_colmajor(gV, X.shape[1])
    P.close()
    return f, gUh, gVh, fo, GUo, GVo


def check(f, gU, gV, fo, GUo, GVo):
    assert abs(f - fo) <= F_TOL * abs(fo), (f, fo)
    G = np.concatenate([gU.ravel(), gV.ravel()])
    Go = np.concatenate([GUo.ravel(), GVo.ravel()])
    assert np.linalg.norm(G - Go) <= G_TOL * np.linalg.norm(Go), np.linalg.norm(G - Go) / np.linalg.norm(Go)
    # Each block on its own: on a tall X the m x k block dominates the joint norm, so an
    # error confined to the n x k block (D^T U, the cross-lane reduction) could hide there.
    for a, b, name in ((gU, GUo, "gU"), (gV, GVo, "gV")):
        nb = np.linalg.norm(b)
        if nb > 0:
            assert np.linalg.norm(a - b) <= G_TOL * nb, (name, np.linalg.norm(a - b) / nb)
        else:
            assert np.linalg.norm(a) == 0.0, name


def random_case(m, n, k, seed, mask_p=None, lam_S=0.3, scale=0.5):
    g = np.random.default_rng(seed)
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    mask = None if mask_p is None else np.asfortranarray((g.random((m, n)) < mask_p).astype(np.uint8))
    U, V = gen.factors(m, n, k, seed + 100, scale=scale)
    return X, mask, U, V, 0.7, lam_S


@pytest.mark.parametrize("m,n,k", [(500, 400, 10), (37, 29, 3), (1001, 77, 1), (3000, 260, 5),
                                   (5000, 300, 16), (2100, 130, 8), (64, 8, 2), (9, 5, 4), (4099, 1027, 6),
                                   (777, 333, 12), (1500, 99, 13), (200, 17, 7), (1092, 181, 11),
                                   (640, 90, 9), (333, 120, 15), (2035, 193, 14)])
def test_fg_unmasked(m, n, k):
    X, mask, U, V, lam_L, lam_S = random_case(m, n, k, seed=m + n + k)
    check(*run_case(X, mask, U, V, lam_L, lam_S))


@pytest.mark.parametrize("m,n,k", [(500, 400, 10), (1001, 77, 5), (3000, 260, 16), (37, 29, 3)])
def test_fg_masked(m, n, k):
    X, mask, U, V, lam_L, lam_S = random_case(m, n, k, seed=7 * m + n, mask_p=0.5)
    mask[3, :] = 0
    mask[:, 2] = 0
    check(*run_case(X, mask, U, V, lam_L, lam_S))


def test_fg_empty_mask_leaves_only_the_penalty():
    X, _, U, V, lam_L, lam_S = random_case(300, 50, 4, seed=3)
    mask = np.zeros(X.shape, np.uint8, order="F")
    f, gU, gV, fo, GUo, GVo = run_case(X, mask, U, V, lam_L, lam_S)
    check(f, gU, gV, fo, GUo, GVo)
    assert np.allclose(gU, lam_L * U.astype(np.float64), rtol=1e-6)


def test_fg_least_squares_limit():
    X, mask, U, V, lam_L, _ = random_case(900, 120, 6, seed=5)
    check(*run_case(X, mask, U, V, lam_L, math.inf))


def test_fg_planted_500x400():
    inst = gen.planted_500x400(0)
    U, V = gen.factors(inst.m, inst.n, inst.k, seed=1, scale=0.3)
    check(*run_case(inst.X, None, U, V, inst.lam_L, inst.lam_S))


def test_fg_bitwise_deterministic():
    from paper_1702_02241_gb300.engine import Problem, to_device_colmajor
    X, mask, U, V, lam_L, lam_S = random_case(4000, 500, 5, seed=11, mask_p=0.6)
    P = Problem(X, mask, 5, lam_L, lam_S)
    Ud, Vd = to_device_colmajor(U), to_device_colmajor(V)
    a = P.fg(Ud, Vd)
    b = P.fg(Ud, Vd)
    assert a[0] == b[0] and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    P.close()


@pytest.mark.parametrize("k,masked", [(5, False), (10, True), (3, True)])
def test_apply_products(k, masked):
    from paper_1702_02241_gb300.engine import Problem, from_device_colmajor, to_device_colmajor
    m, n = 1500, 230
    X, mask, U, V, lam_L, lam_S = random_case(m, n, k, seed=k, mask_p=0.5 if masked else None)
    g = np.random.default_rng(4)
    Bv = np.asfortranarray(g.normal(size=(n, 8)).astype(np.float32))
    Bu = np.asfortranarray(g.normal(size=(m, 8)).astype(np.float32))
    P = Problem(X, mask, k, lam_L, lam_S)
    DBv, DtBu = P.apply(to_device_colmajor(U), to_device_colmajor(V), to_device_colmajor(Bv), to_device_colmajor(Bu))
    Y1, Y2 = core.apply_D(X, mask, U, V, lam_S, Bv, Bu)
    assert np.linalg.norm(from_device_colmajor(DBv, m) - Y1) <= G_TOL * np.linalg.norm(Y1)
    assert np.linalg.norm(from_device_colmajor(DtBu, n) - Y2) <= G_TOL * np.linalg.norm(Y2)
    P.close()


@pytest.mark.slow
def test_fg_full_video_76800x1000():
    """Full-size video workload, same launch configuration as the benchmark: f and the whole
    gradient against the oracle (fits in host memory in float64)."""
    inst = gen.video_76800x1000(0)
    U, V = gen.factors(inst.m, inst.n, inst.k, seed=2, scale=0.2)
    check(*run_case(inst.X, None, U, V, inst.lam_L, inst.lam_S))
