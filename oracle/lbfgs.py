"""L-BFGS (memory 10) with a strong-Wolfe line search, float64, on the factored objective.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

Sec. 5.1 picks L-BFGS with 10 pairs in memory as the solver for Split-SPCP (Table 1).  The
paper is silent on the line search and on the constants (its solvers came from minFunc), so
this follows the textbook it cites (Nocedal & Wright): two-loop recursion for H g with
H0 = gamma I, gamma = s^T y / y^T y; strong Wolfe conditions with c1 = 1e-4, c2 = 0.9,
bracketing phase then zoom with safeguarded cubic interpolation.  First trial step
alpha = 1, except on the first iteration where alpha = min(1, 1/||g||_1).  A pair with
s^T y <= 1e-10 ||s|| ||y|| is not stored.  A line search that has not finished after 25
trial points resets the memory; two failures in a row stop the solver.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import core

C1 = 1e-4
C2 = 0.9
MAX_TRIALS = 25
ALPHA_MAX = 1e10
CURV_EPS = 1e-10


def two_loop(g, S, Y):
    """Return H g for the L-BFGS inverse-Hessian approximation built from pairs (S[i], Y[i]),
    oldest first (Nocedal & Wright Alg. 7.4)."""
    q = g.copy()
    a = np.zeros(len(S))
    rho = [1.0 / float(y @ s) for s, y in zip(S, Y)]
    for i in range(len(S) - 1, -1, -1):
        a[i] = rho[i] * float(S[i] @ q)
        q -= a[i] * Y[i]
    gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1]) if S else 1.0
    r = gamma * q
    for i in range(len(S)):
        b = rho[i] * float(Y[i] @ r)
        r += S[i] * (a[i] - b)
    return r


def cubic_min(a, fa, ga, b, fb, gb):
    """Minimiser of the cubic interpolating (a, fa, ga) and (b, fb, gb) (N&W Eq. 3.59).
    Returns None when the cubic has no real minimiser."""
    if a == b:
        return None
    d1 = ga + gb - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - ga * gb
    if not np.isfinite(disc) or disc < 0:
        return None
    d2 = np.sign(b - a) * np.sqrt(disc)
    den = gb - ga + 2.0 * d2
    if den == 0 or not np.isfinite(den):
        return None
    return b - (b - a) * (gb + d2 - d1) / den


def interpolate(lo, flo, glo, hi, fhi, ghi):
    """Safeguarded trial point inside the bracket: cubic minimiser clamped to the middle 80%
    of [min(lo,hi), max(lo,hi)], bisection when the cubic fails."""
    left, right = min(lo, hi), max(lo, hi)
    width = right - left
    t = cubic_min(lo, flo, glo, hi, fhi, ghi)
    if t is None or not np.isfinite(t):
        return 0.5 * (lo + hi)
    return min(max(t, left + 0.1 * width), right - 0.1 * width)


def wolfe_search(phi, f0, g0, alpha1):
    """Strong-Wolfe line search (N&W Alg. 3.5 with zoom Alg. 3.6).

    ``phi(alpha) -> (f, dphi, payload)`` evaluates the objective and the directional
    derivative at x + alpha d.  ``g0`` is the directional derivative at alpha = 0 (< 0).
    Returns (alpha, f, dphi, payload, n_evals) or None after MAX_TRIALS evaluations.
    """
    evals = 0
    prev_a, prev_f, prev_g = 0.0, f0, g0
    a = alpha1
    first = True
    while evals < MAX_TRIALS:
        fa, ga, pay = phi(a)
        evals += 1
        if (not np.isfinite(fa)) or fa > f0 + C1 * a * g0 or ((not first) and fa >= prev_f):
            return _zoom(phi, f0, g0, prev_a, prev_f, prev_g, a, fa, ga, evals)
        if abs(ga) <= -C2 * g0:
            return a, fa, ga, pay, evals
        if ga >= 0:
            return _zoom(phi, f0, g0, a, fa, ga, prev_a, prev_f, prev_g, evals)
        prev_a, prev_f, prev_g = a, fa, ga
        a = min(4.0 * a, ALPHA_MAX)
        first = False
    return None


def _zoom(phi, f0, g0, lo, flo, glo, hi, fhi, ghi, evals):
    while evals < MAX_TRIALS:
        if not np.isfinite(fhi):
            a = 0.5 * (lo + hi)
        else:
            a = interpolate(lo, flo, glo, hi, fhi, ghi)
        fa, ga, pay = phi(a)
        evals += 1
        if (not np.isfinite(fa)) or fa > f0 + C1 * a * g0 or fa >= flo:
            hi, fhi, ghi = a, fa, ga
        else:
            if abs(ga) <= -C2 * g0:
                return a, fa, ga, pay, evals
            if ga * (hi - lo) >= 0:
                hi, fhi, ghi = lo, flo, glo
            lo, flo, glo = a, fa, ga
    return None


@dataclasses.dataclass
class Result:
    U: np.ndarray
    V: np.ndarray
    f: float
    iters: int
    evals: int
    gnorm: float
    history: list


def solve(X, mask, U0, V0, lam_L, lam_S, mem=10, max_iter=2000, gtol=1e-10, ftol=0.0,
          callback=None):
    """Minimise F(U, V) of Eq. (Thm5) from (U0, V0) with L-BFGS(mem).

    Stops when ||grad F||_F <= gtol * max(1, |F|), when the relative decrease of F over an
    iteration is below ``ftol``, after ``max_iter`` iterations, or when the line search fails
    twice in a row.  ``callback(it, U, V, f)`` may return True to stop early.
    """
    m, k = np.shape(U0)
    n = np.shape(V0)[0]
    x = np.concatenate([np.asarray(U0, np.float64).ravel(order="F"),
                        np.asarray(V0, np.float64).ravel(order="F")])

    def unpack(z):
        return z[: m * k].reshape((m, k), order="F"), z[m * k:].reshape((n, k), order="F")

    def fgrad(z):
        U, V = unpack(z)
        f, GU, GV = core.fg(X, mask, U, V, lam_L, lam_S)
        return f, np.concatenate([GU.ravel(order="F"), GV.ravel(order="F")])

    f, g = fgrad(x)
    evals = 1
    S, Y = [], []
    hist = [f]
    fails = 0
    it = 0
    while it < max_iter:
        gn = float(np.linalg.norm(g))
        if gn <= gtol * max(1.0, abs(f)):
            break
        d = -two_loop(g, S, Y)
        gd = float(g @ d)
        if not gd < 0:
            S, Y = [], []
            d = -g
            gd = float(g @ d)
        alpha1 = min(1.0, 1.0 / float(np.abs(g).sum())) if (it == 0 or not S) else 1.0

        def phi(a, x=x, d=d):
            fa, ga = fgrad(x + a * d)
            return fa, float(ga @ d), ga

        res = wolfe_search(phi, f, gd, alpha1)
        if res is None:
            evals += MAX_TRIALS
            fails += 1
            S, Y = [], []
            if fails >= 2:
                break
            continue
        fails = 0
        a, fa, _, ga, ne = res
        evals += ne
        s = a * d
        y = ga - g
        sy = float(s @ y)
        if sy > CURV_EPS * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > mem:
                S.pop(0)
                Y.pop(0)
        fold = f
        x = x + s
        f, g = fa, ga
        it += 1
        hist.append(f)
        if callback is not None:
            U, V = unpack(x)
            if callback(it, U, V, f):
                break
        if ftol > 0 and (fold - f) <= ftol * max(1.0, abs(f)):
            break
    U, V = unpack(x)
    return Result(U=U, V=V, f=f, iters=it, evals=evals, gnorm=float(np.linalg.norm(g)), history=hist)
