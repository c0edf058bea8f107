"""GPU parity of the learned warm start and of the device instance generator.

* Philox4x32-10: device words equal the host implementation bit for bit (the host one is
  pinned by the published known-answer vectors in test_gen_philox.py).
* Planted generator: the same outliers (exact), A B^T and X within float32 rounding of the
  host's float64 evaluation of the same draws.
* Network: forward outputs, the training gradient and loss, and one Adam step against the
  FP64 oracle (oracle/warm_start.py) on the same parameters.
* Sketch spectrum, features and targets against the oracle on the same test matrix.
* The learned start: kept when its objective is lower, dropped (sketch start) otherwise.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sketch  # noqa: E402
from oracle import warm_start as ows  # noqa: E402
from paper_1702_02241_gb300 import gen, rpca  # noqa: E402
from paper_1702_02241_gb300.engine import ld_for  # noqa: E402

from gpu_util import dev, empty_factors, host, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def _theta(seed, scale=0.1):
    g = np.random.default_rng(seed)
    th = (scale * g.standard_normal(ows.NPARAM)).astype(np.float32)
    return th


def test_philox_words_match_host():
    count = 1000
    out = torch.zeros(4 * count, dtype=torch.int32, device="cuda")
    ctr = (0xFFFFFF00, 7, 2, 123456)
    key = 0x0123456789ABCDEF
    rpca.rpca_philox4x32_10(out, count, ctr, key)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(count, 4)
    c = np.stack([(ctr[0] + np.arange(count)) & 0xFFFFFFFF, np.full(count, ctr[1]), np.full(count, ctr[2]),
                  np.full(count, ctr[3])], axis=-1)
    want = gen.philox4x32_10(c, (key & 0xFFFFFFFF, key >> 32))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("m,n,rank,p", [(300, 70, 3, 0.05), (1031, 257, 10, 0.08)])
def test_planted_generator_matches_host(m, n, rank, p):
    ld = ld_for(m)
    X = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    L0 = torch.zeros((n, m), dtype=torch.float32, device="cuda")
    rpca.rpca_gen_planted(m, n, rank, p, 1e-3, 99, 5, X, ld, L0)
    torch.cuda.synchronize()
    Xd = X.cpu().numpy()[:, :m].T.astype(np.float64)
    Ld = L0.cpu().numpy().T.astype(np.float64)
    Xh, Lh, out = gen.planted_philox(m, n, rank, p, 1e-3, 99, 5)
    assert np.max(np.abs(Ld - Lh)) <= 1e-5 * (1 + np.max(np.abs(Lh)))
    assert np.array_equal(np.abs(Xd - Ld) > 0.5, out)
    assert np.max(np.abs(Xd - Xh)) <= 2e-5 * (1 + np.max(np.abs(Xh)))
    assert abs(out.mean() - p) < 5 * math.sqrt(p * (1 - p) / out.size)


def test_network_forward_matches_oracle():
    th = _theta(1)
    w = rpca.rpca_ws_create(th)
    g = np.random.default_rng(2)
    B = 37
    X = g.standard_normal((B, ows.FEAT)).astype(np.float32)
    Wd = torch.zeros((B, ows.OUT), dtype=torch.float32, device="cuda")
    rpca.rpca_ws_predict(w, torch.from_numpy(X).cuda(), B, Wd)
    torch.cuda.synchronize()
    want, _ = ows.forward(th, X)
    assert np.max(np.abs(Wd.cpu().numpy() - want)) <= 2e-5
    rpca.rpca_ws_destroy(w)


def test_training_gradient_and_adam_step_match_oracle():
    th = _theta(3)
    w = rpca.rpca_ws_create(th)
    g = np.random.default_rng(4)
    B = 45
    X = g.standard_normal((B, ows.FEAT)).astype(np.float32)
    T = g.random((B, ows.OUT)).astype(np.float32)
    K = g.integers(1, 17, size=B).astype(np.int32)
    Xd, Td, Kd = (torch.from_numpy(a).cuda() for a in (X, T, K))
    loss = rpca.rpca_ws_train_step(w, Xd, Td, Kd, B, 0.0)
    th0, grad = rpca.rpca_ws_get_params(w)
    assert np.array_equal(th0, th)  # lr = 0 leaves the masters
    lo, go = ows.loss_and_grad(th, X, T, K)
    assert loss == pytest.approx(lo, rel=1e-5)
    assert np.linalg.norm(grad - go) <= 1e-4 * np.linalg.norm(go)
    # One real step from fresh optimiser state: Adam on the device's own gradient.
    rpca.rpca_ws_set_params(w, th)
    rpca.rpca_ws_train_step(w, Xd, Td, Kd, B, 1e-3)
    th1, grad1 = rpca.rpca_ws_get_params(w)
    want, _, _ = ows.adam_step(th.astype(np.float64), grad1.astype(np.float64), 0.0, 0.0, 1, lr=1e-3)
    assert np.max(np.abs(th1 - want)) <= 1e-6 + 1e-6 * np.max(np.abs(want))
    rpca.rpca_ws_destroy(w)


def _planted_ctx(m, n, rank, k, p, seed):
    lam_S = 1.0 / math.sqrt(max(m, n))
    lam_L = lam_S * (math.sqrt(m) + math.sqrt(n))
    inst = gen.planted(m, n, rank=rank, k=k, p_outlier=p, noise=1e-3, lam_L=lam_L, lam_S=lam_S, seed=seed)
    return inst


def test_spectrum_features_targets_match_oracle():
    inst = _planted_ctx(1500, 180, 4, 8, 0.05, 11)
    m, n, k = inst.m, inst.n, inst.k
    l = k + 10
    Om = gen.gaussian(n, l, seed=5).astype(np.float32)
    P = make_problem(inst.X, None, k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_USER, max_iter=3000,
                     cert_every=10)
    Us, Vs = empty_factors(m, n, k)
    P.init_sketch(Us, Vs, dev(Om))
    s_dev = rpca.rpca_sketch_spectrum(P.ctx)
    _, s_or, _ = sketch.rsvd_parts(inst.X, None, Om)
    assert s_dev.size == l
    assert np.allclose(s_dev, s_or, rtol=2e-4, atol=1e-5 * s_or[0])
    U, V = Us.clone(), Vs.clone()
    r = P.solve(U, V)
    assert r.status == rpca.RPCA_OK
    x = torch.zeros(ows.FEAT, dtype=torch.float32, device="cuda")
    wst = torch.zeros(ows.OUT, dtype=torch.float32, device="cuda")
    rpca.rpca_ws_sample(P.ctx, Us, Vs, U, V, x, wst)
    torch.cuda.synchronize()
    xo = ows.features(s_dev.astype(np.float64), k, inst.lam_L, inst.lam_S, m, n)
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 2e-6
    wo = ows.targets(host(Us, m), host(Vs, n), s_dev, host(U, m), host(V, n))
    wd = wst.cpu().numpy()
    assert np.max(np.abs(wd[:k] - wo)) <= 1e-4 and np.all(wd[k:] == 0)
    # The solution keeps the planted components and drops the outlier ones.
    assert np.all(wo[:4] > 0.9) and np.all(wo[4:] < 0.05)
    P.close()


def _const_model(w_first, w_rest, rank):
    """A model whose output ignores its input: W3 = 0, b3 = logit of the wanted shares."""
    th = np.zeros(ows.NPARAM, np.float32)
    b3 = np.full(ows.OUT, w_rest)
    b3[:rank] = w_first
    parts = ows.unpack(th)
    parts["b3"][:] = np.log(b3 / (1 - b3))
    return ows.pack(parts).astype(np.float32)


def test_learned_start_kept_when_better_and_dropped_when_worse():
    inst = _planted_ctx(2000, 200, 4, 8, 0.05, 21)
    m, n, k = inst.m, inst.n, inst.k
    base = make_problem(inst.X, None, k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH, max_iter=3000,
                        cert_every=10)
    U0, V0 = empty_factors(m, n, k)
    r0 = base.solve(U0, V0)
    base.close()
    assert r0.status == rpca.RPCA_OK and r0.init_used == rpca.RPCA_INIT_SKETCH
    # Keep the planted rank's components, drop the rest: a better start.
    good = rpca.rpca_ws_create(_const_model(0.999, 1e-4, 4))
    P = make_problem(inst.X, None, k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_LEARNED, max_iter=3000,
                     cert_every=10)
    rpca.rpca_set_warm_start(P.ctx, good)
    U, V = empty_factors(m, n, k)
    r = P.solve(U, V)
    assert r.status == rpca.RPCA_OK and r.init_used == rpca.RPCA_INIT_LEARNED
    assert r.F == pytest.approx(r0.F, rel=1e-6)
    assert r.iters < r0.iters
    # Drop everything: the start's objective is F(0) > F(sketch start): falls back.
    bad = rpca.rpca_ws_create(_const_model(1e-4, 1e-4, 4))
    rpca.rpca_set_warm_start(P.ctx, bad)
    U, V = empty_factors(m, n, k)
    r2 = P.solve(U, V)
    assert r2.status == rpca.RPCA_OK and r2.init_used == rpca.RPCA_INIT_SKETCH
    assert r2.iters == r0.iters
    P.close()
    rpca.rpca_ws_destroy(good)
    rpca.rpca_ws_destroy(bad)


def test_trained_start_needs_fewer_iterations_on_heldout():
    """End to end on a small protocol: instances generated on the device, solved from the
    sketch, the network trained on (features, targets), then held-out instances solved from
    the learned start need fewer iterations than from the sketch start, to the same objective."""
    from paper_1702_02241_gb300 import warm_start as W
    specs = W.instance_params(240, 7, m=1024, n=128)
    x, t, K, _ = W.make_samples(specs, 7)
    w, losses = W.train(x, t, K, epochs=150, batch=64, seed=3)
    assert losses[-1][1] < 0.5 * losses[0][1]
    held = W.instance_params(16, 8, m=1024, n=128)
    res = W.evaluate(w, held, 8, starts=("sketch", "learned"))
    assert res["sketch"]["ok"] == res["learned"]["ok"] == len(held)
    assert np.mean(res["learned"]["iters"]) < np.mean(res["sketch"]["iters"])
    for a, b in zip(res["learned"]["F"], res["sketch"]["F"]):
        assert a == pytest.approx(b, rel=1e-5)
    rpca.rpca_ws_destroy(w)
