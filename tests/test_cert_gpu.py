"""GPU certificate (Sec. 3.4) against the FP64 oracle's explicit computation.

t1..t3 are float64 reductions of float32 products: compared at 1e-6 relative (plus an
absolute floor of 1e-6 * lam_L^2 for terms that vanish).  t4 comes from block Lanczos with
float32 Ritz values: 1e-3 relative (the tolerance stated for the spectral step).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import certificate as ocert  # noqa: E402
from oracle import lbfgs, sketch  # noqa: E402
from paper_1702_02241_gb300 import gen  # noqa: E402

from gpu_util import dev, host, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def compare(c, o, lam_L, t4_rel=1e-3):
    floor = 1e-6 * lam_L ** 2
    for name in ("t1", "t2", "t3"):
        a, b = getattr(c, name), getattr(o, name)
        assert abs(a - b) <= 1e-6 * abs(b) + floor, (name, a, b)
    assert abs(c.t4 - o.t4) <= t4_rel * o.t4 + floor, (c.t4, o.t4)
    assert c.rank_r == o.rank_r
    assert c.normL_F == pytest.approx(o.normL_F, rel=1e-6)
    assert c.F == pytest.approx(o.F, rel=1e-6)
    assert c.F_bound <= o.F_bound * (1 + 1e-6)
    assert c.cert == pytest.approx(o.cert, rel=1e-3, abs=1e-3 * lam_L)
    # Cost of the truncated directions (2 lam_L times their singular values) and its
    # relative form; both zero when nothing was truncated.
    assert c.F_trunc == pytest.approx(o.F_trunc, rel=1e-4, abs=1e-12 * lam_L * max(o.normL_F, 1.0))
    assert c.trunc_rel == pytest.approx(o.trunc_rel, rel=1e-4, abs=1e-12)


@pytest.mark.parametrize("path", ["cluster", "default", "launches"])
@pytest.mark.parametrize("m,n,k,masked", [(300, 200, 5, False), (257, 190, 3, True), (400, 130, 12, False),
                                          (12000, 260, 6, False)])
def test_certificate_random_point(m, n, k, masked, path, monkeypatch):
    """The forms of the Lanczos block orthonormalisation: one thread-block-cluster launch
    wherever the rows fit (RPCA_CERT_CLUSTER=1; 12000 rows take a cluster of eight CTAs), the
    default (one CTA for up to 1024 rows, else the multi-launch form) and the multi-launch form
    throughout (RPCA_CERT_CLUSTER=0)."""
    if path == "default":
        monkeypatch.delenv("RPCA_CERT_CLUSTER", raising=False)
    else:
        monkeypatch.setenv("RPCA_CERT_CLUSTER", "1" if path == "cluster" else "0")
    g = np.random.default_rng(m + k)
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    mask = np.asfortranarray((g.random((m, n)) < 0.6).astype(np.uint8)) if masked else None
    U, V = gen.factors(m, n, k, seed=k, scale=0.3)
    lam_L, lam_S = 2.0, 0.5
    P = make_problem(X, mask, k, lam_L, lam_S)
    c = P.certificate(dev(U), dev(V))
    o = ocert.certificate(X, mask, U, V, lam_L, lam_S)
    compare(c, o, lam_L)
    P.close()


def test_certificate_rank_deficient_factors():
    g = np.random.default_rng(3)
    m, n, k = 200, 150, 6
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    U, V = gen.factors(m, n, k, seed=1, scale=0.5)
    U[:, 4:] = 0.0
    V[:, 4:] = 0.0
    P = make_problem(X, None, k, 1.0, 0.4)
    c = P.certificate(dev(U), dev(V))
    o = ocert.certificate(X, None, U, V, 1.0, 0.4)
    assert c.rank_r == o.rank_r == 4
    compare(c, o, 1.0)
    P.close()


def test_certificate_at_optimum_is_small():
    inst = gen.planted_500x400(0)
    Om = gen.gaussian(inst.n, inst.k + 10, seed=11)
    U0, V0 = sketch.rsvd_init(inst.X, None, inst.k, Om)
    ref = lbfgs.solve(inst.X, None, U0, V0, inst.lam_L, inst.lam_S, gtol=1e-11, max_iter=3000)
    U, V = ref.U.astype(np.float32), ref.V.astype(np.float32)
    P = make_problem(inst.X, None, inst.k, inst.lam_L, inst.lam_S)
    c = P.certificate(dev(U), dev(V))
    o = ocert.certificate(inst.X, None, U, V, inst.lam_L, inst.lam_S)
    assert o.cert_rel < 1e-4 and c.cert_rel < 1e-4
    assert c.t4 == 0.0 and o.t4 == 0.0
    assert c.rank_r == o.rank_r == 5
    assert c.sigma1_perp == pytest.approx(o.sigma_perp[0], rel=1e-3)
    P.close()


def test_certificate_plateau_when_k_too_small():
    g = np.random.default_rng(5)
    m, n = 120, 90
    X = np.asfortranarray((g.normal(size=(m, 4)) @ g.normal(size=(4, n)) * 2.0).astype(np.float32))
    U0, V0 = gen.factors(m, n, 2, seed=2, scale=0.5)
    ref = lbfgs.solve(X, None, U0, V0, 1.0, math.inf, gtol=1e-12, max_iter=5000)
    U, V = ref.U.astype(np.float32), ref.V.astype(np.float32)
    P = make_problem(X, None, 2, 1.0, math.inf)
    c = P.certificate(dev(U), dev(V))
    o = ocert.certificate(X, None, U, V, 1.0, math.inf)
    assert o.t4 > 1.0
    compare(c, o, 1.0)
    P.close()


def test_certificate_with_vanishing_surplus_columns():
    """k above the rank of L: the nuclear penalty drives the surplus factor columns to zero,
    through the float32 subnormal range.  Their Gram entries are then tiny float64 values;
    the Jacobi rotations of the small eigen-problems must stay finite there, and the
    certificate must be that of the rank-5 part."""
    g = np.random.default_rng(17)
    m, n, k = 1092, 181, 11
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    U, V = gen.factors(m, n, k, seed=4, scale=0.5)
    for j in range(5, k):
        s = np.float32(10.0 ** (-19 - (j - 5)))
        U[:, j] *= s
        V[:, j] *= s
    P = make_problem(X, None, k, 2.0, 0.5)
    c = P.certificate(dev(U), dev(V))
    o = ocert.certificate(X, None, U, V, 2.0, 0.5)
    assert math.isfinite(c.cert) and c.rank_r == o.rank_r == 5
    compare(c, o, 2.0)
    P.close()


@pytest.mark.parametrize("zero_optimal", [True, False])
def test_certificate_of_rounding_floor_factors(zero_optimal):
    """Factors at the float32 rounding floor (|U|, |V| ~ 1e-22): L is numerically zero, r = 0,
    and the certificate is the one of L = 0 (t4 from sigma_i(clip(-X)) against lam_L)."""
    g = np.random.default_rng(21)
    m, n, k = 1092, 181, 11
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    lam_S = 0.3
    s0 = np.linalg.svd(np.clip(-X.astype(np.float64), -lam_S, lam_S), compute_uv=False)[0]
    lam_L = 1.1 * s0 if zero_optimal else 0.8 * s0
    U = np.asfortranarray((1e-22 * g.normal(size=(m, k))).astype(np.float32))
    V = np.asfortranarray((1e-22 * g.normal(size=(n, k))).astype(np.float32))
    P = make_problem(X, None, k, lam_L, lam_S)
    c = P.certificate(dev(U), dev(V))
    o = ocert.certificate(X, None, U, V, lam_L, lam_S)
    assert c.rank_r == o.rank_r == 0
    compare(c, o, lam_L)
    if zero_optimal:
        assert c.cert_rel == 0.0
    P.close()


def test_certificate_reports_the_cost_of_a_truncated_direction():
    """A rank-3 point plus a tiny (5e-4 sigma_1) direction that is not stationary: both sides
    move it to the complement block, report F_trunc = 2 lam_L sigma_4 and trunc_rel, and the
    point does not count as certified at 1e-4 although cert_rel may."""
    g = np.random.default_rng(31)
    m, n = 1200, 300
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    U, V = gen.factors(m, n, 4, seed=8, scale=0.5)
    Q, _ = np.linalg.qr(np.c_[U[:, :3], g.normal(size=m)])
    W, _ = np.linalg.qr(np.c_[V[:, :3], g.normal(size=n)])
    s1 = np.linalg.svd(U[:, :3] @ V[:, :3].T, compute_uv=False)[0]
    sig = 5e-4 * s1
    U[:, 3] = math.sqrt(sig) * Q[:, 3]
    V[:, 3] = math.sqrt(sig) * W[:, 3]
    U, V = U.astype(np.float32), V.astype(np.float32)
    # lam_L above the spectrum of D's projection (about 0.5 (sqrt(m) + sqrt(n)) here), so that
    # t4 = 0 and the spectral step is exact; the point is the truncated direction.
    lam_L, lam_S = 40.0, 0.5
    P = make_problem(X, None, 4, lam_L, lam_S)
    c = P.certificate(dev(U), dev(V))
    o = ocert.certificate(X, None, U, V, lam_L, lam_S)
    assert o.rank_r == 3 and o.F_trunc == pytest.approx(2 * lam_L * sig, rel=1e-3)
    compare(c, o, lam_L)
    assert c.gap_bound == pytest.approx(o.gap_bound, rel=1e-3)
    assert not o.certified(1e-4) and not c.certified(1e-4)
    P.close()


def test_spectral_term_where_the_krylov_space_truncates():
    """t4 > 0 at n = 1000: a planted rank-12 instance solved at k = 8, so that about four
    directions of P_U1perp D P_V1perp exceed lam_L among 1000; block Lanczos (<= 256 dims)
    spans a fraction of the space.  t4 and sigma_1 against the oracle's scipy svds at the
    spectral step's 1e-3."""
    from paper_1702_02241_gb300 import rpca
    m, n, k = 20000, 1000, 8
    lam_S = 1.0 / math.sqrt(m)
    inst = gen.planted(m, n, rank=12, k=k, p_outlier=0.05, noise=1e-3,
                       lam_L=2.0 * lam_S * (math.sqrt(m) + math.sqrt(n)), lam_S=lam_S, seed=5)
    P = make_problem(inst.X, None, k, inst.lam_L, inst.lam_S, max_iter=300)
    Ud, Vd = dev(np.zeros((m, k))), dev(np.zeros((n, k)))
    try:
        P.solve(Ud, Vd)
    except rpca.RpcaError as e:            # a rank-8 solve of a rank-12 instance cannot certify
        assert e.status == rpca.RPCA_ENOTCONV
    U = host(Ud, m).astype(np.float32)
    V = host(Vd, n).astype(np.float32)
    c = P.certificate(dev(U), dev(V))
    o = ocert.certificate(inst.X, None, U, V, inst.lam_L, inst.lam_S, t4_method="svds")
    assert o.t4 > 1e-2 * inst.lam_L ** 2 and np.sum(o.sigma_perp > inst.lam_L) >= 2
    assert c.krylov_steps * 8 < n
    compare(c, o, inst.lam_L)
    assert c.sigma1_perp == pytest.approx(o.sigma_perp[0], rel=1e-3)
    P.close()


@pytest.mark.parametrize("masked", [False, True])
def test_solve_certificate_from_gradient_matches_full_pass(masked):
    """Inside a solve the cheap terms take D V and D^T U from the solver's gradient at its
    iterate (G - lam_L x) and F from its objective, with no pass over X.  A solve with a loose
    tolerance certifies at a check and returns that certificate; it must equal rpca_certificate's
    (which makes the pass) at the returned point, and the FP64 oracle's."""
    from paper_1702_02241_gb300 import rpca
    from gpu_util import empty_factors
    inst = gen.planted_500x400(0)
    mask = (np.random.default_rng(5).random(inst.X.shape) < 0.7).astype(np.uint8) if masked else None
    P = make_problem(inst.X, mask, inst.k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH, max_iter=400,
                     cert_every=8, cert_tol=0.3)
    U, V = empty_factors(inst.m, inst.n, inst.k)
    res = P.solve(U, V)
    assert res.status == rpca.RPCA_OK and res.iters < 400, (res.status, res.iters, res.cert.asdict())
    assert res.cert.cert_rel > 1e-4  # stopped at a check well before convergence
    full = P.certificate(U, V)
    compare(res.cert, full, inst.lam_L)
    Uh, Vh = host(U, inst.m), host(V, inst.n)
    o = ocert.certificate(inst.X, mask, Uh.astype(np.float64), Vh.astype(np.float64), inst.lam_L, inst.lam_S)
    compare(res.cert, o, inst.lam_L)
    P.close()
