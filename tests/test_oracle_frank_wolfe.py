"""Pins of the Frank-Wolfe-with-marginalization oracle (oracle/frank_wolfe.py; Sec. 6.2,
Algorithm 1), each against something other than the oracle's own formula:

* the closed-form step equals a brute-force minimisation of the printed line-search
  objective over a fine grid of eta (S_k fixed);
* F(L, t) never increases, and ||L||_* <= t holds for every iterate;
* the Frank-Wolfe gap bounds F - F*, with F* from the convex FISTA/SVT reference solver
  (oracle/convex.py), and it shrinks with the iterations;
* at an iterate where sigma_1(G) <= lam_L the step is the pure shrink toward 0.
"""
import numpy as np
import pytest

from oracle import convex, core
from oracle import frank_wolfe as fw


def _case(seed=0, m=40, n=30, rank=3, p=0.1):
    g = np.random.default_rng(seed)
    L0 = g.normal(size=(m, rank)) @ g.normal(size=(rank, n))
    S0 = np.where(g.random((m, n)) < p, g.uniform(1, 5, (m, n)) * np.sign(g.normal(size=(m, n))), 0.0)
    return L0 + S0 + 0.01 * g.normal(size=(m, n))


def test_step_size_is_the_line_search_minimiser():
    X = _case(1)
    lam_L, lam_S = 2.0, 0.3
    steps = fw.solve(X, None, lam_L, lam_S, 6)
    L, t, B = steps[4].L, steps[4].t, steps[4].B
    base = fw.radius0(X, None, np.zeros_like(X), lam_L, lam_S)
    s = fw.step(X, None, L, t, B, base, lam_L, lam_S)
    # The printed objective, S_k fixed: 1/2 ||P(L_eta + S_k - X)||^2 + lam_L t_eta.
    G = core.D_of_R(L - X, None, lam_S)
    Uu, ss, Vt = np.linalg.svd(G)
    V = -B * np.outer(Uu[:, 0], Vt[0]) if ss[0] > lam_L else 0 * L
    Vt_ = B if ss[0] > lam_L else 0.0
    S_k = np.sign(X - L) * np.maximum(np.abs(X - L) - lam_S, 0.0)
    etas = np.linspace(0.0, 1.0, 20001)
    q = [0.5 * np.sum(((1 - e) * L + e * V + S_k - X) ** 2) + lam_L * ((1 - e) * t + e * Vt_) for e in etas]
    assert abs(s.eta - etas[int(np.argmin(q))]) <= 1e-4


def test_objective_never_increases_and_t_bounds_the_nuclear_norm():
    X = _case(2)
    lam_L, lam_S = 1.5, 0.25
    steps = fw.solve(X, None, lam_L, lam_S, 60)
    Fs = [fw.objective(X, None, np.zeros_like(X), 0.0, lam_L, lam_S)] + [s.F for s in steps]
    assert all(b <= a + 1e-9 * abs(a) for a, b in zip(Fs, Fs[1:]))
    for s in steps:
        assert np.linalg.svd(s.L, compute_uv=False).sum() <= s.t * (1 + 1e-9) + 1e-12


def test_gap_bounds_distance_to_the_convex_optimum():
    """Once the radius bound B covers ||L*||_* (B grows with t), the gap at (L_k, t_k) bounds
    F(L_k, t_k) - F*; F approaches F* (slowly, as the paper reports for this method)."""
    X = _case(3)
    lam_L, lam_S = 2.5, 0.3
    Lstar = convex.fista(X, None, lam_L, lam_S, iters=4000)
    nuc = np.linalg.svd(Lstar, compute_uv=False).sum()
    Fstar = lam_L * nuc + core.phi_of_R(Lstar - X, None, lam_S)
    L, t = np.zeros_like(X), 0.0
    base = fw.radius0(X, None, L, lam_L, lam_S)
    B = base
    gaps, checked = [], 0
    for _ in range(1000):
        s = fw.step(X, None, L, t, B, base, lam_L, lam_S)
        if B >= nuc:
            assert s.gap >= fw.objective(X, None, L, t, lam_L, lam_S) - Fstar - 1e-6 * abs(Fstar)
            checked += 1
        gaps.append(s.gap)
        L, t, B = s.L, s.t, s.B
    assert checked > 500
    assert gaps[-1] < 0.15 * gaps[0]
    assert fw.objective(X, None, L, t, lam_L, lam_S) - Fstar <= 0.01 * abs(Fstar)


def test_shrink_step_at_a_solution():
    X = _case(4)
    lam_L, lam_S = 50.0, 0.3       # lam_L above sigma_1 of the gradient at L = 0: L* = 0
    base = fw.radius0(X, None, np.zeros_like(X), lam_L, lam_S)
    s = fw.step(X, None, np.zeros_like(X), 0.0, base, base, lam_L, lam_S)
    assert s.sigma1 <= lam_L and np.all(s.L == 0) and s.t == 0.0 and s.gap == pytest.approx(0.0, abs=1e-9)
