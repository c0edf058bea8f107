"""Pins of the learned-warm-start oracle (oracle/warm_start.py) and of the planted-rank
choice of lam_L for the batched workload.

* Backward: central finite differences of the loss (weights not rounded, so that the loss
  is smooth) against the analytic gradient, every parameter block.
* Adam: the first step of Adam moves every parameter by -lr g / (|g| + eps) (bias
  corrections cancel), a closed form of Kingma & Ba's update.
* Targets: closed forms -- L* equal to the sketch start gives w* = 1, L* = 0 gives 0, and
  L* = U_k diag(a s) V_k^T gives a.
* Features: invariant to one common scale of (s, lam_L, lam_S).
"""
import math

import numpy as np
import pytest

from oracle import lbfgs, sketch
from oracle import warm_start as ws
from paper_1702_02241_gb300 import gen


def _theta(seed, scale=0.3):
    g = np.random.default_rng(seed)
    return (scale * g.standard_normal(ws.NPARAM)).astype(np.float32)


def test_packed_layout_size():
    assert ws.NPARAM == 256 * 40 + 256 + 256 * 256 + 256 + 16 * 256 + 16
    th = _theta(0)
    assert np.array_equal(ws.pack(ws.unpack(th)), th)


def test_backward_matches_central_differences():
    g = np.random.default_rng(1)
    B = 5
    X = g.standard_normal((B, ws.FEAT))
    T = g.random((B, ws.OUT))
    kk = np.array([3, 16, 7, 1, 12])
    th = _theta(2, 0.15).astype(np.float64)
    loss, grad = ws.loss_and_grad(th, X, T, kk, rounded=False)
    parts = ws.unpack(np.arange(ws.NPARAM))
    for name, _ in ws.SIZES:
        idx = parts[name].ravel()
        for i in g.choice(idx, size=min(6, idx.size), replace=False):
            h = 1e-6
            tp = th.copy(); tp[i] += h
            tm = th.copy(); tm[i] -= h
            fd = (ws.loss_and_grad(tp, X, T, kk, rounded=False)[0] -
                  ws.loss_and_grad(tm, X, T, kk, rounded=False)[0]) / (2 * h)
            assert fd == pytest.approx(grad[i], rel=1e-5, abs=1e-9), (name, i)


def test_outputs_beyond_k_do_not_contribute():
    g = np.random.default_rng(3)
    X = g.standard_normal((2, ws.FEAT))
    T = g.random((2, ws.OUT))
    th = _theta(4)
    l1, g1 = ws.loss_and_grad(th, X, T, [4, 9])
    T2 = T.copy(); T2[0, 4:] = 7.0; T2[1, 9:] = -3.0
    l2, g2 = ws.loss_and_grad(th, X, T2, [4, 9])
    assert l1 == l2 and np.array_equal(g1, g2)


def test_adam_first_step_closed_form():
    g = np.random.default_rng(5)
    th = g.standard_normal(50)
    grad = g.standard_normal(50)
    new, m, v = ws.adam_step(th, grad, np.zeros(50), np.zeros(50), 1, lr=0.01)
    assert np.allclose(new - th, -0.01 * grad / (np.abs(grad) + 1e-8), rtol=1e-12, atol=0)


def test_targets_closed_forms():
    g = np.random.default_rng(6)
    m, n, k = 40, 30, 4
    Uk, _ = np.linalg.qr(g.standard_normal((m, k)))
    Vk, _ = np.linalg.qr(g.standard_normal((n, k)))
    s = np.array([9.0, 5.0, 2.0, 0.5])
    Us, Vs = Uk * np.sqrt(s), Vk * np.sqrt(s)
    assert np.allclose(ws.targets(Us, Vs, s, Us, Vs), 1.0)
    assert np.allclose(ws.targets(Us, Vs, s, 0 * Us, 0 * Vs), 0.0)
    a = np.array([0.9, 0.0, 0.4, 0.25])
    U = Uk * np.sqrt(a * s)
    V = Vk * np.sqrt(a * s)
    assert np.allclose(ws.targets(Us, Vs, s, U, V), a)
    # A rotation of the solution's factors changes nothing.
    Qr, _ = np.linalg.qr(g.standard_normal((k, k)))
    assert np.allclose(ws.targets(Us, Vs, s, U @ Qr, V @ Qr), a)
    U0, V0 = ws.start(Us, Vs, a)
    assert np.allclose(U0 @ V0.T, Uk @ np.diag(a * s) @ Vk.T)


def test_features_scale_invariant():
    s = np.array([40.0, 33.0, 9.0, 3.0, 2.5, 2.0])
    x1 = ws.features(s, 3, 1.5, 0.1, 500, 80)
    x2 = ws.features(7.0 * s, 3, 7.0 * 1.5, 7.0 * 0.1, 500, 80)
    assert np.allclose(x1, x2, atol=1e-6)
    assert x1[5] == 0.0 and x1[6] == 0.0 and x1[0] == pytest.approx(math.log(20.0), rel=1e-6)


def test_batch_lambda_recovers_planted_rank():
    """lam_L = lam_S (sqrt(m) + sqrt(n)) of the batched workload gives a solution of the
    planted rank (the rule it follows), on two small instances of the same recipe."""
    insts = gen.batch_c4(2, seed=3, m_range=(1024, 1100), n_range=(50, 70), k_range=(4, 8))
    for inst in insts:
        rank = max(1, inst.k // 2)
        U0, V0 = sketch.rsvd_init(inst.X, None, inst.k, gen.gaussian(inst.n, inst.k + 10, seed=1))
        r = lbfgs.solve(inst.X, None, U0, V0, inst.lam_L, inst.lam_S, gtol=1e-10, max_iter=3000)
        sv = np.linalg.svd(r.U @ r.V.T, compute_uv=False)
        assert int(np.sum(sv > 1e-6 * sv[0])) == rank
        assert np.linalg.norm(r.U @ r.V.T - inst.L0) <= 0.05 * np.linalg.norm(inst.L0)
