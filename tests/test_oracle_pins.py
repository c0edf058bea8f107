"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks an oracle function against brute force, finite differences, a closed form
(textbook special case), an explicit construction from the definition, or a planted
solution, chosen so that a dropped term, a wrong sign, a wrong index or a transposed
operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import certificate as ocert
from oracle import convex, core, lbfgs, sketch
from paper_1702_02241_gb300 import gen


# --- Huber marginal (Sec. 1, "Marginalization in S") -------------------------------------

def _golden_min(f, lo, hi, iters=200):
    """Vectorised golden-section minimisation of convex f on [lo, hi]."""
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo.copy(), hi.copy()
    c, d = b - gr * (b - a), a + gr * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        left = fc < fd
        b = np.where(left, d, b)
        a = np.where(left, a, c)
        c, d = b - gr * (b - a), a + gr * (b - a)
        fc, fd = f(c), f(d)
    x = 0.5 * (a + b)
    return x, f(x)


def test_huber_equals_bruteforce_marginal():
    g = np.random.default_rng(1)
    r = g.normal(0, 3, size=10_000)
    lam = g.uniform(0.01, 4.0, size=10_000)
    obj = lambda s: 0.5 * (r + s) ** 2 + lam * np.abs(s)
    s_star, v = _golden_min(obj, -np.abs(r) - 1.0, np.abs(r) + 1.0)
    assert np.max(np.abs(core.psi(r, lam) - v) / np.maximum(1.0, np.abs(v))) < 1e-12
    # Danskin: d/dr min_s f(r, s) = r + s*(r), which must be the clip the oracle uses.  A
    # value-comparing search locates the minimiser only to ~sqrt(eps) * |r|.
    assert np.max(np.abs(core.dpsi(r, lam) - (r + s_star))) < 1e-6


def test_huber_special_values():
    assert core.psi(0.0, 1.0) == 0.0
    assert core.psi(2.0, 1.0) == pytest.approx(1.5)       # lam|r| - lam^2/2
    assert core.psi(-0.5, 1.0) == pytest.approx(0.125)    # r^2/2
    assert core.psi(3.0, np.inf) == pytest.approx(4.5)
    assert core.dpsi(-7.0, 2.0) == -2.0


# --- gradient (Sec. 3.2) vs central differences -----------------------------------------

def _fd_case(seed, masked):
    g = np.random.default_rng(seed)
    m, n, k = 6, 5, 3
    X = g.normal(size=(m, n))
    U = g.normal(size=(m, k))
    V = g.normal(size=(n, k))
    lam_S = 0.7
    mask = (g.random((m, n)) < 0.7).astype(np.uint8) if masked else None
    R = U @ V.T - X
    return X, mask, U, V, 0.3, lam_S, R


@pytest.mark.parametrize("masked", [False, True])
def test_gradient_matches_central_differences(masked):
    for seed in range(20):
        X, mask, U, V, lam_L, lam_S, R = _fd_case(seed, masked)
        if np.min(np.abs(np.abs(R) - lam_S)) > 1e-3:
            break
    f, GU, GV = core.fg(X, mask, U, V, lam_L, lam_S)
    assert f == pytest.approx(core.objective(X, mask, U, V, lam_L, lam_S), rel=1e-15)
    num = np.zeros_like(GU)
    for idx in np.ndindex(U.shape):
        h = 1e-6 * max(1.0, abs(U[idx]))
        Up, Um = U.copy(), U.copy()
        Up[idx] += h
        Um[idx] -= h
        num[idx] = (core.objective(X, mask, Up, V, lam_L, lam_S)
                    - core.objective(X, mask, Um, V, lam_L, lam_S)) / (2 * h)
    assert np.linalg.norm(num - GU) / np.linalg.norm(GU) < 1e-7
    num = np.zeros_like(GV)
    for idx in np.ndindex(V.shape):
        h = 1e-6 * max(1.0, abs(V[idx]))
        Vp, Vm = V.copy(), V.copy()
        Vp[idx] += h
        Vm[idx] -= h
        num[idx] = (core.objective(X, mask, U, Vp, lam_L, lam_S)
                    - core.objective(X, mask, U, Vm, lam_L, lam_S)) / (2 * h)
    assert np.linalg.norm(num - GV) / np.linalg.norm(GV) < 1e-7


def test_masked_entries_contribute_nothing():
    X, _, U, V, lam_L, lam_S, _ = _fd_case(3, False)
    mask = np.ones(X.shape, np.uint8)
    mask[2, :] = 0
    X2 = X.copy()
    X2[2, :] += 100.0  # unobserved entries may hold anything
    a = core.fg(X, mask, U, V, lam_L, lam_S)
    b = core.fg(X2, mask, U, V, lam_L, lam_S)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.all(b[1][2] == lam_L * U[2])  # no data term on a fully unobserved row


def test_sparse_part_reconstructs_objective():
    """phi(L) equals the explicit S-objective at S = soft(X - L) (marginalisation identity)."""
    X, mask, U, V, lam_L, lam_S, _ = _fd_case(4, True)
    L = U @ V.T
    S = core.sparse_part(X, mask, L, lam_S)
    M = mask != 0
    explicit = 0.5 * np.sum(np.where(M, L + S - X, 0) ** 2) + lam_S * np.abs(S).sum()
    assert core.phi_of_R(L - X, mask, lam_S) == pytest.approx(explicit, rel=1e-13)


# --- L-BFGS pieces (Nocedal & Wright) ----------------------------------------------------

def test_two_loop_equals_explicit_bfgs_matrix():
    g = np.random.default_rng(5)
    d = 7
    A = g.normal(size=(d, d))
    Hs = A @ A.T + d * np.eye(d)
    S, Y = [], []
    for _ in range(4):
        s = g.normal(size=d)
        S.append(s)
        Y.append(Hs @ s)
    gamma = S[-1] @ Y[-1] / (Y[-1] @ Y[-1])
    H = gamma * np.eye(d)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        E = np.eye(d) - rho * np.outer(s, y)
        H = E @ H @ E.T + rho * np.outer(s, s)
    v = g.normal(size=d)
    assert np.allclose(lbfgs.two_loop(v, S, Y), H @ v, rtol=1e-12, atol=1e-12)


def test_cubic_interpolation_exact_on_cubic():
    p = lambda x: (x - 0.3) ** 2 * (x + 2.0) / 3.0   # local min at 0.3 inside [0, 1]
    dp = lambda x: (2 * (x - 0.3) * (x + 2.0) + (x - 0.3) ** 2) / 3.0
    t = lbfgs.cubic_min(0.0, p(0.0), dp(0.0), 1.0, p(1.0), dp(1.0))
    assert t == pytest.approx(0.3, abs=1e-12)


def test_wolfe_search_returns_strong_wolfe_point():
    for c, x0 in [(1.0, 3.0), (40.0, 0.2), (1e-3, 5.0)]:
        f = lambda x: c * (x ** 4 - 2 * x ** 2) + x
        df = lambda x: c * (4 * x ** 3 - 4 * x) + 1
        d = -df(x0)
        phi = lambda a: (f(x0 + a * d), df(x0 + a * d) * d, None)
        f0, g0 = f(x0), df(x0) * d
        a, fa, ga, _, _ = lbfgs.wolfe_search(phi, f0, g0, 1.0)
        assert fa <= f0 + lbfgs.C1 * a * g0
        assert abs(ga) <= -lbfgs.C2 * g0


# --- textbook special case: lam_S = inf reduces to singular-value thresholding -----------

def _lowrank_noise(m, n, r, seed, noise=0.05):
    g = np.random.default_rng(seed)
    return g.normal(size=(m, r)) @ g.normal(size=(r, n)) + noise * g.normal(size=(m, n))


def test_svt_special_case_fista_and_split():
    X = _lowrank_noise(20, 15, 3, 0)
    lam_L = 1.5
    Lsvt = convex.svt(X, lam_L)                  # closed form of the convex problem
    Lf = convex.fista(X, None, lam_L, np.inf)
    assert np.linalg.norm(Lf - Lsvt) <= 1e-9 * np.linalg.norm(Lsvt)
    Fc = core.convex_objective(X, None, Lsvt, lam_L, np.inf)
    U0, V0 = gen.factors(20, 15, 6, seed=1, scale=0.5)
    res = lbfgs.solve(X, None, U0, V0, lam_L, np.inf, gtol=1e-12, max_iter=5000)
    assert res.f == pytest.approx(Fc, rel=1e-8)
    assert np.linalg.norm(res.U @ res.V.T - Lsvt) <= 1e-6 * np.linalg.norm(Lsvt)
    # Balanced factors at stationarity (Sec. 3.3 / 3.4: D V = -lam U and D^T U = -lam V).
    assert np.allclose(res.U.T @ res.U, res.V.T @ res.V, atol=1e-6)
    Ub, Vb = convex.balanced_factors(Lsvt, 6)
    c = ocert.certificate(X, None, Ub, Vb, lam_L, np.inf)
    assert c.cert_rel < 1e-9
    c2 = ocert.certificate(X, None, res.U, res.V, lam_L, np.inf)
    assert c2.cert_rel < 1e-5


def test_certificate_sign_reading():
    """The printed 'I - U1^T D V1' would give ~2 sqrt(r) lam_L at the optimum; the reading
    'lam I + U1^T D V1' gives ~0 (the oracle's)."""
    X = _lowrank_noise(20, 15, 3, 2)
    lam_L = 1.0
    Ub, Vb = convex.balanced_factors(convex.svt(X, lam_L), 5)
    U1, V1, _ = ocert.range_bases(Ub, Vb)
    D = Ub @ Vb.T - X
    B = U1.T @ D @ V1
    r = B.shape[0]
    printed = np.linalg.norm(lam_L * np.eye(r) - B)
    assert printed == pytest.approx(2 * math.sqrt(r) * lam_L, rel=1e-8)
    assert ocert.certificate(X, None, Ub, Vb, lam_L, np.inf).t1 < 1e-20


# --- convex vs split on tiny Huber instances (Thm 1 + certificate) -----------------------

@pytest.mark.parametrize("shape,seed", [((20, 15), 0), ((30, 25), 1)])
def test_split_matches_convex_fista(shape, seed):
    m, n = shape
    g = np.random.default_rng(seed)
    L0 = g.normal(size=(m, 2)) @ g.normal(size=(2, n))
    S0 = np.where(g.random((m, n)) < 0.1, g.choice([-3.0, 3.0], size=(m, n)), 0.0)
    X = L0 + S0 + 0.01 * g.normal(size=(m, n))
    lam_S, lam_L = 1.0 / math.sqrt(n), 0.8
    Lc = convex.fista(X, None, lam_L, lam_S, iters=50000, tol=1e-15)
    Fc = core.convex_objective(X, None, Lc, lam_L, lam_S)
    rank = int(np.sum(np.linalg.svd(Lc, compute_uv=False) > 1e-8))
    assert 1 <= rank < 6
    U0, V0 = gen.factors(m, n, 6, seed=seed + 10, scale=0.3)
    res = lbfgs.solve(X, None, U0, V0, lam_L, lam_S, gtol=1e-13, max_iter=20000)
    Fs = core.convex_objective(X, None, res.U @ res.V.T, lam_L, lam_S)
    assert Fs == pytest.approx(Fc, rel=1e-8)
    assert res.f == pytest.approx(Fc, rel=1e-8)
    Ub, Vb = convex.balanced_factors(Lc, 6)
    assert ocert.certificate(X, None, Ub, Vb, lam_L, lam_S).cert_rel < 1e-6
    assert ocert.certificate(X, None, res.U, res.V, lam_L, lam_S).cert_rel < 1e-6


def test_certificate_plateaus_when_k_too_small():
    """k below rank(L*) leaves t4 > 0 at the split optimum (Sec. 3.4, Fig. 1)."""
    g = np.random.default_rng(3)
    X = g.normal(size=(20, 4)) @ g.normal(size=(4, 15)) * 3.0
    lam_L = 1.0
    U0, V0 = gen.factors(20, 15, 2, seed=4, scale=0.5)
    res = lbfgs.solve(X, None, U0, V0, lam_L, np.inf, gtol=1e-12, max_iter=5000)
    c = ocert.certificate(X, None, res.U, res.V, lam_L, np.inf)
    sv = np.linalg.svd(X, compute_uv=False)
    assert c.t1 + c.t2 + c.t3 < 1e-12
    # The two dropped singular directions of X exceed lam_L by sv[2]-lam_L, sv[3]-lam_L.
    assert c.t4 == pytest.approx(np.sum((sv[2:4] - lam_L) ** 2), rel=1e-8)


# --- certificate vs the explicit subdifferential construction ---------------------------

def test_certificate_terms_equal_explicit_construction():
    g = np.random.default_rng(7)
    m, n, k = 14, 11, 3
    X = g.normal(size=(m, n))
    U = g.normal(size=(m, k))
    V = g.normal(size=(n, k))
    mask = (g.random((m, n)) < 0.8).astype(np.uint8)
    lam_L, lam_S = 0.4, 0.6
    c = ocert.certificate(X, mask, U, V, lam_L, lam_S)
    L = U @ V.T
    D = core.D_of_R(L - X, mask, lam_S)
    Uf, s, Vft = np.linalg.svd(L)                 # complete SVD: U~ = [U1 U2], V~ = [V1 V2]
    r = int(np.sum(s > 1e-8 * s[0]))
    assert r == c.rank_r == k
    U1, U2, V1, V2 = Uf[:, :r], Uf[:, r:], Vft[:r].T, Vft[r:].T
    M = U2.T @ D @ V2
    Um, sm, Vmt = np.linalg.svd(M, full_matrices=False)
    Wp = -(Um * np.minimum(sm, lam_L)) @ Vmt     # argmin over the lam_L spectral ball
    Z = U1 @ V1.T + U2 @ (Wp / lam_L) @ V2.T     # element of the nuclear-norm subdifferential
    assert np.allclose(U1.T @ (Z - U1 @ V1.T), 0, atol=1e-12)
    assert np.allclose((Z - U1 @ V1.T) @ V1, 0, atol=1e-12)
    assert np.linalg.norm(Z - U1 @ V1.T, 2) <= 1 + 1e-12
    E = lam_L * Z + D
    assert np.sum(E * E) == pytest.approx(c.t1 + c.t2 + c.t3 + c.t4, rel=1e-10)
    assert c.t1 == pytest.approx(np.sum((U1.T @ E @ V1) ** 2), rel=1e-10)
    assert c.t2 == pytest.approx(np.sum((U1.T @ D @ V2) ** 2), rel=1e-9)
    assert c.t3 == pytest.approx(np.sum((U2.T @ D @ V1) ** 2), rel=1e-9)
    # The paper's shortcut ||U1^T D V2||^2 = ||U1^T D||^2 - ||U1^T D V1||^2 (Sec. 3.4).
    B = U1.T @ D @ V1
    assert c.t2 == pytest.approx(np.sum((U1.T @ D) ** 2) - np.sum(B * B), rel=1e-9)
    assert c.t3 == pytest.approx(np.sum((D @ V1) ** 2) - np.sum(B * B), rel=1e-9)
    # No other feasible W' does better (spot check).
    for _ in range(20):
        W2 = g.normal(size=M.shape)
        W2 *= lam_L * g.uniform(0, 1) / np.linalg.norm(W2, 2)
        E2 = lam_L * (U1 @ V1.T) + U2 @ W2 @ V2.T + D
        assert np.sum(E2 * E2) >= np.sum(E * E) - 1e-12


def test_certificate_svds_matches_dense():
    inst = gen.planted(120, 90, rank=3, k=5, seed=2)
    U, V = gen.factors(120, 90, 5, seed=3)
    X = inst.X.astype(np.float64)
    D = core.D_of_R(U.astype(np.float64) @ V.T.astype(np.float64) - X, None, inst.lam_S)
    U1, V1, _ = ocert.range_bases(U, V)
    lam = 0.02
    dense = ocert.perp_singular_values(D, U1, V1, lam, "dense")
    sv = ocert.perp_singular_values(D, U1, V1, lam, "svds", k_s=8)
    assert np.allclose(sv[:8], dense[:8], rtol=1e-8)
    assert sv[-1] < lam


# --- planted recovery on the 500 x 400 instance -----------------------------------------

@pytest.mark.slow
def test_planted_recovery_500x400():
    inst = gen.planted_500x400(0)
    X = inst.X
    Om = gen.gaussian(inst.n, inst.k + 10, seed=11)
    U0, V0 = sketch.rsvd_init(X, None, inst.k, Om)
    res = lbfgs.solve(X, None, U0, V0, inst.lam_L, inst.lam_S, gtol=1e-11, max_iter=3000)
    L = res.U @ res.V.T
    assert np.linalg.norm(L - inst.L0) / np.linalg.norm(inst.L0) < 1e-2
    S = core.sparse_part(X, None, L, inst.lam_S)
    assert np.array_equal(S != 0, inst.S0 != 0)
    c = ocert.certificate(X, None, res.U, res.V, inst.lam_L, inst.lam_S)
    assert c.rank_r == 5 and c.cert_rel < 1e-4 and c.t4 == 0.0


# --- randomized SVD initialisation (Sec. 4.2) ---------------------------------------------

def test_rsvd_exact_on_low_rank():
    g = np.random.default_rng(9)
    m, n, r, k = 60, 40, 4, 4
    X = g.normal(size=(m, r)) @ g.normal(size=(r, n))
    Om = g.normal(size=(n, k + 10))
    U0, V0 = sketch.rsvd_init(X, None, k, Om, q=2)
    Uf, s, Vft = np.linalg.svd(X)
    assert np.allclose(U0 @ V0.T, X, atol=1e-10 * np.abs(X).max())
    assert np.allclose(np.linalg.norm(U0, axis=0) ** 2, s[:k], rtol=1e-10)
    assert np.allclose(U0.T @ U0, V0.T @ V0, atol=1e-9 * s[0])


def test_rsvd_mask_rescaling():
    g = np.random.default_rng(10)
    X = g.normal(size=(50, 30))
    mask = (g.random((50, 30)) < 0.25).astype(np.uint8)
    A = sketch.sampled(X, mask)
    assert np.allclose(A[mask == 0], 0)
    assert np.allclose(A[mask != 0], X[mask != 0] / mask.mean())


def test_certificate_moves_tiny_inactive_direction_to_complement():
    """A rounding-size extra factor column at the optimum is truncated (the direction goes to
    the W' block): the certificate equals the one of the truncated point, not ~lam_L."""
    X = _lowrank_noise(20, 15, 3, 4)
    lam_L = 1.0
    Ub, Vb = convex.balanced_factors(convex.svt(X, lam_L), 4)
    g = np.random.default_rng(1)
    U, V = Ub.copy(), Vb.copy()
    U[:, 3] = 3e-3 * g.normal(size=20)
    V[:, 3] = 3e-3 * g.normal(size=15)
    c = ocert.certificate(X, np.ones(X.shape, np.uint8), U, V, lam_L, np.inf)
    assert c.rank_r == 3
    assert c.cert_rel < 1e-3
    # Without the rule the extra direction would sit in U1 with u^T D v ~ 0: t1 >= lam_L^2 / 4.
    U1, V1, s = ocert.range_bases(U, V)
    assert s.size == 4 and s[3] / s[0] < 1e-3


@pytest.mark.parametrize("lam_S", [np.inf, 1.0 / math.sqrt(15)])
def test_truncation_cost_bounds_the_gap_of_a_nonstationary_direction(lam_S):
    """A deliberately non-stationary direction of size 5e-4 sigma_1 outside the optimum's
    range is tiny and inactive, so the certificate truncates it; the gap it leaves, G(L) - G*
    with G* from FISTA on the convex problem (Sec. 1, Eq. 4), stays below gap_bound once the
    truncation's cost F_trunc = 2 lam_L sigma is added (convexity of phi and of the nuclear
    norm), and the point does not count as certified at 1e-4.  In the least-squares case
    (lam_S = inf, D = L - X changes only along the added direction) the certificate itself is
    ~0 there, and the bound without F_trunc fails."""
    m, n = 20, 15
    g = np.random.default_rng(0)
    L0 = g.normal(size=(m, 2)) @ g.normal(size=(2, n))
    S0 = np.where(g.random((m, n)) < 0.1, g.choice([-3.0, 3.0], size=(m, n)), 0.0)
    X = L0 + S0 + 0.01 * g.normal(size=(m, n))
    lam_L = 0.8
    Lc = convex.fista(X, None, lam_L, lam_S, iters=50000, tol=1e-15)
    Gstar = core.convex_objective(X, None, Lc, lam_L, lam_S)
    Uc, sc, Vct = np.linalg.svd(Lc)
    r = int(np.sum(sc > 1e-8 * sc[0]))
    assert 1 <= r < min(m, n)
    U, V = convex.balanced_factors(Lc, r + 1)
    assert ocert.certificate(X, None, U, V, lam_L, lam_S).certified(1e-6)
    # The added direction: unit u, v orthogonal to the optimum's ranges, sigma = 5e-4 sigma_1.
    u = Uc[:, r:] @ g.normal(size=m - r)
    v = Vct[r:].T @ g.normal(size=n - r)
    u, v = u / np.linalg.norm(u), v / np.linalg.norm(v)
    sig = 5e-4 * sc[0]
    U[:, r] = math.sqrt(sig) * u
    V[:, r] = math.sqrt(sig) * v
    c = ocert.certificate(X, None, U, V, lam_L, lam_S)
    gap = core.convex_objective(X, None, U @ V.T, lam_L, lam_S) - Gstar
    assert c.rank_r == r                                  # the direction went to the complement
    assert c.F_trunc == pytest.approx(2.0 * lam_L * sig, rel=1e-9)
    assert gap > 0.1 * lam_L * sig                        # it is not stationary
    assert gap <= c.gap_bound
    assert c.trunc_rel > 1e-4 and not c.certified(1e-4)
    if lam_S == np.inf:
        old = c.cert * (c.normL_F + c.F_bound / lam_L)    # the bound without the truncation
        assert c.cert_rel < 1e-9 and old < 1e-3 * gap


def test_certificate_of_rounding_floor_factors_is_that_of_zero():
    """Factors at the float32 rounding floor (|L| ~ 1e-44) when the solution is L = 0: every
    direction is negligible, r = 0, and the certificate equals the closed form at L = 0:
    t1 = t2 = t3 = 0, t4 = sum_i (sigma_i(D0) - lam_L)_+^2 with D0 = clip(-X) (Sec. 3.4),
    computed here from a dense SVD of D0 directly."""
    g = np.random.default_rng(8)
    m, n, k = 60, 40, 4
    X = g.normal(size=(m, n))
    lam_S = 0.3
    D0 = np.clip(-X, -lam_S, lam_S)
    sv = np.linalg.svd(D0, compute_uv=False)
    for lam_L in (0.8 * sv[0], 1.1 * sv[0]):   # zero is not optimal / optimal
        U = 1e-22 * g.normal(size=(m, k))
        V = 1e-22 * g.normal(size=(n, k))
        c = ocert.certificate(X, None, U, V, lam_L, lam_S)
        assert c.rank_r == 0
        assert c.t1 == 0.0 and c.t2 == 0.0 and c.t3 == 0.0
        assert c.t4 == pytest.approx(np.sum(np.maximum(sv - lam_L, 0.0) ** 2), rel=1e-9, abs=1e-12)
    # Without the rule the same point keeps a direction in U1 with u^T D v far from -lam_L.
    U1, V1, s = ocert.range_bases(U, V)
    assert s.size == k


def test_certificate_keeps_small_but_significant_direction():
    """A direction far below sigma_1 but not negligible against F stays in U1 when active
    (the negligibility floor is absolute in F, not relative to sigma_1)."""
    X = _lowrank_noise(20, 15, 3, 4)
    lam_L = 1.0
    Ub, Vb = convex.balanced_factors(convex.svt(X, lam_L), 3)
    c = ocert.certificate(X, np.ones(X.shape, np.uint8), Ub, Vb, lam_L, np.inf)
    U1, V1, s = ocert.range_bases(Ub, Vb)
    assert s.size == 3 and lam_L * s[-1] > 1e-12 * c.F
    assert c.rank_r == 3 and c.cert_rel < 1e-6


@pytest.mark.parametrize("lam_S", [0.3, math.inf])
def test_grow_column_decreases_by_the_quadratic_bound(lam_S):
    """Rank increase (Sec. 4.1): with k below the rank of the solution the certificate's
    spectral term is positive (sigma_1 > lam_L), and the added column lowers F by at least
    (sigma_1 - lam_L)^2 / 2 -- the bound that psi'' <= 1 gives along a unit rank-one
    direction -- computed here from F itself, not from the column's construction."""
    g = np.random.default_rng(12)
    m, n = 60, 45
    X = g.normal(size=(m, 5)) @ g.normal(size=(5, n)) * 1.5 + 0.05 * g.normal(size=(m, n))
    lam_L = 1.0
    U0, V0 = gen.factors(m, n, 2, seed=3, scale=0.5)
    r = lbfgs.solve(X, None, U0, V0, lam_L, lam_S, gtol=1e-11, max_iter=4000)
    U, V = r.U, r.V
    F0 = core.objective(X, None, U, V, lam_L, lam_S)
    U2, V2, s1 = ocert.grow_column(X, None, U, V, lam_L, lam_S)
    assert s1 > lam_L
    F1 = core.objective(X, None, U2, V2, lam_L, lam_S)
    assert F1 <= F0 - 0.5 * (s1 - lam_L) ** 2 + 1e-9 * abs(F0)
    # The pair is the top singular pair of the projected residual gradient: its value is the
    # certificate's largest perpendicular singular value.
    c = ocert.certificate(X, None, U, V, lam_L, lam_S)
    assert s1 == pytest.approx(c.sigma_perp[0], rel=1e-10)


def test_grow_column_adds_nothing_at_a_solution():
    """At a solution (sigma_1 <= lam_L) the new column is zero and F is unchanged."""
    X = _lowrank_noise(20, 15, 3, 4)
    Ub, Vb = convex.balanced_factors(convex.svt(X, 1.0), 3)
    U2, V2, s1 = ocert.grow_column(X, np.ones(X.shape, np.uint8), Ub, Vb, 1.0, np.inf)
    assert s1 <= 1.0 + 1e-9
    assert np.all(U2[:, 3] == 0) and np.all(V2[:, 3] == 0)


def test_grow_columns_decrease_by_the_summed_bound():
    """Several columns at once: F drops by at least sum_i (sigma_i - lam_L)^2 / 2 (orthonormal
    pairs), and every added sigma_i exceeds lam_L."""
    g = np.random.default_rng(13)
    m, n = 70, 50
    X = g.normal(size=(m, 6)) @ g.normal(size=(6, n)) * 1.5 + 0.05 * g.normal(size=(m, n))
    lam_L, lam_S = 1.0, 0.4
    U0, V0 = gen.factors(m, n, 2, seed=4, scale=0.5)
    r = lbfgs.solve(X, None, U0, V0, lam_L, lam_S, gtol=1e-11, max_iter=4000)
    F0 = core.objective(X, None, r.U, r.V, lam_L, lam_S)
    U2, V2, ss = ocert.grow_columns(X, None, r.U, r.V, lam_L, lam_S, 10)
    assert ss.size >= 2 and np.all(ss > lam_L)
    F1 = core.objective(X, None, U2, V2, lam_L, lam_S)
    assert F1 <= F0 - 0.5 * np.sum((ss - lam_L) ** 2) + 1e-9 * abs(F0)
