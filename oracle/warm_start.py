"""Learned warm start, float64 host.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

The paper starts L-BFGS from the SVD or a randomized SVD of the data and shows that the start
matters (Sec. 4.2: random starts can stall).  The learned warm start keeps the randomized
sketch's singular directions (Sec. 4.2 with Halko et al.'s range finder) and learns how much
of each component the solution keeps: the sketch's components beyond the rank of L* are
outlier energy that the solver otherwise spends its first iterations removing.

* Sketch start: U_s = U_k Sigma_k^(1/2), V_s = V_k Sigma_k^(1/2) (the rSVD start) and the l
  sketch singular values s_1 >= ... >= s_l (l = k + p).
* Features x (FEAT = 40 values, float32): x_j = log(s_j / s_l) for j < l (0 for j >= l),
  x_32 = log(lam_L / s_l), x_33 = log(lam_S sqrt(m n) / s_l), x_34 = k / 16, x_35 = l / 32,
  x_36 = log(m / n) / 4, x_37 = log(m n) / 20, x_38 = x_39 = 0.  Invariant to a common
  scaling of X, lam_L and lam_S.
* Network (three layers, hidden 256): h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
  z = W3 h2 + b3 (16 outputs), w = sigmoid(z).  The weight matrices are used rounded to
  bfloat16 (oracle.quant.bf16_round of the float32 masters); biases are float32.
* Start: U0 = U_s diag(sqrt(w_1 .. w_k)), V0 = V_s diag(sqrt(w_1 .. w_k)).
* Target: w*_j = u_j^T L* v_j / s_j clipped to [0, 1], with u_j, v_j the sketch's unit
  singular vectors (U_s[:, j] / sqrt(s_j), V_s[:, j] / sqrt(s_j)) and L* = U* V*^T the plain
  solver's solution.  It depends on L* only, not on how L* is factored (rotation-invariant).
* Loss: (1 / B) sum over the B samples of sum_{j < k} (w_j - w*_j)^2.
* Optimiser: Adam (Kingma & Ba 2015) on the float32 masters; the gradient is taken with
  respect to the rounded weights and applied to the masters (straight-through).

Packed parameter vector (the layout the library's model uses), float32:
  W1 (HID x FEAT, row-major: W1[u, i]) | b1 (HID) | W2T (HID x HID, W2T[i, u] = W2[u, i]) |
  b2 (HID) | W3 (OUT x HID, row-major) | b3 (OUT).
"""
from __future__ import annotations

import math

import numpy as np

from . import quant

FEAT, HID, OUT = 40, 256, 16
SIZES = [("W1", (HID, FEAT)), ("b1", (HID,)), ("W2T", (HID, HID)), ("b2", (HID,)),
         ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    """Packed vector -> dict of arrays (views)."""
    out, o = {}, 0
    for name, shape in SIZES:
        cnt = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + cnt]).reshape(shape)
        o += cnt
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name]).ravel() for name, _ in SIZES])


def features(s, k, lam_L, lam_S, m, n):
    """Feature vector of one instance from its l sketch singular values s (descending)."""
    s = np.asarray(s, np.float64)
    l = s.size
    s_ref = max(s[-1], 1e-30 * s[0], 1e-300)
    x = np.zeros(FEAT)
    x[:l] = np.log(np.maximum(s, 1e-300) / s_ref)
    x[32] = math.log(lam_L / s_ref)
    x[33] = math.log(lam_S * math.sqrt(m * n) / s_ref) if math.isfinite(lam_S) else 0.0
    x[34] = k / 16.0
    x[35] = l / 32.0
    x[36] = math.log(m / n) / 4.0
    x[37] = math.log(m * n) / 20.0
    return x.astype(np.float32).astype(np.float64)


def effective(theta, rounded=True):
    """The parameters the network computes with.  rounded: the library's form -- float32
    masters, weight matrices rounded to bfloat16, float32 biases.  Otherwise theta as given
    (float64; used by the finite-difference pin)."""
    if not rounded:
        return {k: np.asarray(v, np.float64) for k, v in unpack(np.asarray(theta, np.float64)).items()}
    p = {k: v.astype(np.float64) for k, v in unpack(np.asarray(theta, np.float32)).items()}
    for name in ("W1", "W2T", "W3"):
        p[name] = quant.bf16_round(np.asarray(p[name], np.float32)).astype(np.float64)
    return p


def forward(theta, X, rounded=True):
    """w (B x OUT) and the intermediate activations for the batch X (B x FEAT)."""
    p = effective(theta, rounded)
    X = np.asarray(X, np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2T"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    w = 1.0 / (1.0 + np.exp(-z))
    return w, (p, X, h1, h2, w)


def loss_and_grad(theta, X, target, kk, rounded=True):
    """Loss and its gradient (packed) with respect to the parameters the network uses.
    target: B x OUT; kk: B factor ranks (outputs j >= k are ignored)."""
    w, (p, X, h1, h2, _) = forward(theta, X, rounded)
    B = X.shape[0]
    valid = (np.arange(OUT)[None, :] < np.asarray(kk)[:, None]).astype(np.float64)
    diff = (w - np.asarray(target, np.float64)) * valid
    loss = float(np.sum(diff * diff) / B)
    dz = (2.0 / B) * diff * w * (1.0 - w)
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = (dz @ p["W3"]) * (h2 > 0)
    g["W2T"] = h1.T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2T"].T) * (h1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return loss, pack(g)


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def targets(Us, Vs, s, U, V):
    """w*_j of the start (Us, Vs) = (U_k Sigma^(1/2), V_k Sigma^(1/2)) against L* = U V^T."""
    Us = np.asarray(Us, np.float64)
    Vs = np.asarray(Vs, np.float64)
    k = Us.shape[1]
    s = np.asarray(s, np.float64)[:k]
    L = np.asarray(U, np.float64) @ np.asarray(V, np.float64).T
    t = np.einsum("ij,ij->j", Us, L @ Vs) / s          # u_j^T L v_j with u_j = Us_j / sqrt(s_j)
    w = np.where(s > 0, t / np.where(s > 0, s, 1.0), 0.0)
    return np.clip(w, 0.0, 1.0)


def start(Us, Vs, w):
    """U0, V0 of the learned start from the sketch start and the network's w (first k)."""
    k = np.shape(Us)[1]
    r = np.sqrt(np.asarray(w, np.float64)[:k])
    return np.asarray(Us, np.float64) * r, np.asarray(Vs, np.float64) * r
