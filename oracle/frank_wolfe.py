"""Frank-Wolfe method with marginalization (Sec. 6.2, Algorithm 1), float64 host.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

The program is min over ||L||_* <= t of lam_L t + min_S 1/2 ||P_Omega(L + S - X)||_F^2 +
lam_S ||S||_1; with S marginalised the inner minimum is phi(L) = sum_Omega psi(L - X), and the
iterate is (L, t).  One iteration, in the algorithm's order:

  S_k = shrink(X - L_k, lam_S)                      (so L_k + S_k - X = clip(L_k - X) on Omega)
  G   = P_Omega(L_k + S_k - X)                        (= D, the gradient of phi)
  Y_k = argmin_{||Y||_* <= 1} <G, Y> = -u_1 v_1^T     (u_1, v_1: top singular pair of G)
  if lam_L >= -<G, Y_k> (= sigma_1(G)):  V_k = 0, Vt_k = 0
  else:                                  V_k = B_k Y_k, Vt_k = B_k        (B_k: the radius bound)
  eta* = argmin_{eta in [0, 1]} 1/2 ||P_Omega((1-eta) L_k + eta V_k + S_k - X)||^2
                                + lam_L ((1-eta) t_k + eta Vt_k)
  L_{k+1} = (1 - eta*) L_k + eta* V_k,   t_{k+1} = (1 - eta*) t_k + eta* Vt_k
  B_{k+1} = (1 / (2 lam_L)) ||P_Omega(L_0 + S_0 - X)||_F^2 + t_k

Readings (the printed algorithm is ambiguous here):
* The radius bound is written U_k in the paper; B here (U is the factor elsewhere).
* The line-search objective prints "(1-eta) lam_L t_k + eta lam_L t_k"; the second t_k is read
  as Vt_k, which makes it the objective lam_L t + quadratic at the new point.  It is a quadratic
  in eta with S_k fixed, minimised in closed form (clipped to [0, 1]).
* B_0 = (1 / (2 lam_L)) ||P_Omega(L_0 + S_0 - X)||^2 and B_{k+1} as printed (with t_k).
* Stopping: the Frank-Wolfe gap <G, L_k - V_k> + lam_L (t_k - Vt_k), an upper bound on
  F(L_k, t_k) - F* whenever the optimal t lies within the radius bound.
* The objective reported is F(L, t) = phi(L) + lam_L t (S re-marginalised at L).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import core


@dataclasses.dataclass
class FWStep:
    L: np.ndarray
    t: float
    B: float
    eta: float
    gap: float
    sigma1: float
    F: float


def _obs(X, mask):
    return np.ones(np.shape(X), bool) if mask is None else np.asarray(mask) != 0


def objective(X, mask, L, t, lam_L, lam_S):
    """F(L, t) = phi(L) + lam_L t with phi(L) = sum_Omega psi(L - X)."""
    R = np.asarray(L, np.float64) - np.asarray(X, np.float64)
    return float(core.phi_of_R(R, mask, lam_S) + lam_L * t)


def radius0(X, mask, L0, lam_L, lam_S):
    """B_0 = (1 / (2 lam_L)) ||P_Omega(L_0 + S_0 - X)||^2 with S_0 = shrink(X - L_0)."""
    D = core.D_of_R(np.asarray(L0, np.float64) - np.asarray(X, np.float64), mask, lam_S)
    return float(0.5 * np.sum(D * D) / lam_L)


def step(X, mask, L, t, B, B0_base, lam_L, lam_S, top_pair=None):
    """One iteration.  top_pair (optional): (sigma_1, u_1, v_1) of G to use instead of the
    dense SVD.  B0_base = (1 / (2 lam_L)) ||P_Omega(L_0 + S_0 - X)||^2."""
    X = np.asarray(X, np.float64)
    L = np.asarray(L, np.float64)
    obs = _obs(X, mask)
    G = core.D_of_R(L - X, mask, lam_S)              # P_Omega(L + S - X), S = shrink(X - L)
    if top_pair is None:
        Uu, ss, Vt = np.linalg.svd(G, full_matrices=False)
        s1, u1, v1 = float(ss[0]), Uu[:, 0], Vt[0]
    else:
        s1, u1, v1 = top_pair
    if lam_L >= s1:
        V = np.zeros_like(L)
        Vt_ = 0.0
    else:
        V = -B * np.outer(u1, v1)
        Vt_ = B
    W = np.where(obs, V - L, 0.0)
    gw = float(np.sum(G * W))
    ww = float(np.sum(W * W))
    # d/d eta of 1/2 ||G + eta W||^2 + lam_L ((1 - eta) t + eta Vt) = <G, W> + eta ||W||^2 + lam_L (Vt - t)
    num = -(gw + lam_L * (Vt_ - t))
    eta = 0.0 if ww <= 0.0 else min(max(num / ww, 0.0), 1.0)
    gap = float(np.sum(G * (L - V)) + lam_L * (t - Vt_))
    L2 = (1.0 - eta) * L + eta * V
    t2 = (1.0 - eta) * t + eta * Vt_
    B2 = B0_base + t
    return FWStep(L=L2, t=t2, B=B2, eta=eta, gap=gap, sigma1=s1, F=objective(X, mask, L2, t2, lam_L, lam_S))


def solve(X, mask, lam_L, lam_S, iters, L0=None):
    """Runs the algorithm from L_0 (zero by default), t_0 = 0; returns the list of steps."""
    X = np.asarray(X, np.float64)
    L = np.zeros_like(X) if L0 is None else np.asarray(L0, np.float64)
    t = 0.0
    base = radius0(X, mask, L, lam_L, lam_S)
    B = base
    out = []
    for _ in range(iters):
        s = step(X, mask, L, t, B, base, lam_L, lam_S)
        out.append(s)
        L, t, B = s.L, s.t, s.B
    return out
