"""GPU tests of the batched form (rpca_create_batch / rpca_solve_batch): independent
problems of varied m, n, k solved concurrently reach their certificates, with the objective of
the same problem solved alone (1e-6 relative) and the oracle's objective at the result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_1702_02241_gb300 import gen, rpca  # noqa: E402
from paper_1702_02241_gb300.engine import ld_for, to_device_colmajor  # noqa: E402

from gpu_util import empty_factors, host, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


DRIVERS = {"grouped": rpca.RPCA_DRIVER_GROUPED, "rounds": rpca.RPCA_DRIVER_ROUNDS, "threads": rpca.RPCA_DRIVER_THREADS}


@pytest.mark.parametrize("mode", ["grouped", "rounds", "threads"])
def test_batch_solves_match_single_solves(mode, monkeypatch):
    """The three drivers of the batched form: grouped (shared launches over all instances, the
    default), rounds (one graph launch advances every instance) and host threads stepping each
    instance's own graph."""
    monkeypatch.setenv("RPCA_BATCH_MODE", mode)
    insts = gen.batch_c4(6, seed=1, m_range=(1024, 3000), n_range=(50, 200))
    Xs = [to_device_colmajor(i.X, pad=True) for i in insts]
    opt = rpca.rpca_default_options()
    opt.init = rpca.RPCA_INIT_SKETCH
    opt.max_iter = 3000
    opt.cert_every = 10
    b = rpca.rpca_create_batch(Xs, [(i.m, ld_for(i.m)) for i in insts], [i.k for i in insts],
                               [i.lam_L for i in insts], [i.lam_S for i in insts], opt)
    assert rpca.rpca_batch_size(b) == len(insts)
    Us, Vs = zip(*[empty_factors(i.m, i.n, i.k) for i in insts])
    st, res = rpca.rpca_solve_batch(b, Us, Vs)
    torch.cuda.synchronize()
    assert st == rpca.RPCA_OK, rpca.rpca_batch_last_error(b)
    assert rpca.rpca_batch_driver(b) == DRIVERS[mode]
    for i, inst in enumerate(insts):
        r = res[i]
        assert r.status == rpca.RPCA_OK and r.cert.certified(1e-4)
        U, V = host(Us[i], inst.m), host(Vs[i], inst.n)
        assert r.F == pytest.approx(core.objective(inst.X, None, U, V, inst.lam_L, inst.lam_S), rel=1e-6)
        P = make_problem(inst.X, None, inst.k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH,
                         max_iter=3000, cert_every=10)
        U1, V1 = empty_factors(inst.m, inst.n, inst.k)
        r1 = P.solve(U1, V1)
        P.close()
        assert r1.status == rpca.RPCA_OK
        assert r.F == pytest.approx(r1.F, rel=1e-6)
    # A second solve of the same batch (the rounds graph is kept) gives the same results.
    Us2, Vs2 = zip(*[empty_factors(i.m, i.n, i.k) for i in insts])
    st2, res2 = rpca.rpca_solve_batch(b, Us2, Vs2)
    assert st2 == rpca.RPCA_OK
    for a, c in zip(res, res2):
        assert a.iters == c.iters and a.F == pytest.approx(c.F, rel=1e-9)
    rpca.rpca_destroy_batch(b)


def _batch(insts, **opts):
    Xs = [to_device_colmajor(i.X, pad=True) for i in insts]
    opt = rpca.rpca_default_options()
    opt.init = rpca.RPCA_INIT_SKETCH
    opt.max_iter = 3000
    opt.cert_every = 10
    for key, val in opts.items():
        setattr(opt, key, val)
    b = rpca.rpca_create_batch(Xs, [(i.m, ld_for(i.m)) for i in insts], [i.k for i in insts],
                               [i.lam_L for i in insts], [i.lam_S for i in insts], opt)
    return b, Xs


def test_grouped_iterates_are_the_single_solves_iterates(monkeypatch):
    """The grouped driver runs each instance's trials with the kernels and grids of its own
    iteration graph: the per-iteration log (F, ||grad F||, step, trials, outcome, pairs) of
    every instance equals, bit for bit, that of rpca_solve on the same context over the
    iterations both ran.  Ranks 2..16 put the instances in many fused-pass groups (small and
    large instantiations, several block sizes), and the certified results meet the oracle's
    objective."""
    monkeypatch.delenv("RPCA_BATCH_MODE", raising=False)
    insts = gen.batch_c4(15, seed=3, m_range=(1024, 4000), n_range=(50, 260))
    for q, inst in enumerate(insts):  # every rank from 2 to 16 once
        k = 2 + q
        insts[q] = gen.planted(inst.m, inst.n, rank=max(1, k // 2), k=k, p_outlier=0.05, noise=1e-3,
                               lam_L=inst.lam_L, lam_S=inst.lam_S, seed=1000 + q)
    b, Xs = _batch(insts)
    Us, Vs = zip(*[empty_factors(i.m, i.n, i.k) for i in insts])
    st, res = rpca.rpca_solve_batch(b, Us, Vs)
    torch.cuda.synchronize()
    assert st == rpca.RPCA_OK, rpca.rpca_batch_last_error(b)
    assert rpca.rpca_batch_driver(b) == rpca.RPCA_DRIVER_GROUPED
    logs = [rpca.rpca_solve_log(rpca.rpca_batch_context(b, i)) for i in range(len(insts))]
    for i, inst in enumerate(insts):
        r = res[i]
        assert r.status == rpca.RPCA_OK and r.cert.certified(1e-4)
        U, V = host(Us[i], inst.m), host(Vs[i], inst.n)
        assert r.F == pytest.approx(core.objective(inst.X, None, U, V, inst.lam_L, inst.lam_S), rel=1e-6)
        ctx = rpca.rpca_batch_context(b, i)
        U1, V1 = empty_factors(inst.m, inst.n, inst.k)
        r1 = rpca.rpca_solve(ctx, U1, V1)
        assert r1.status == rpca.RPCA_OK
        single = rpca.rpca_solve_log(ctx)
        common = min(len(single), len(logs[i]))
        assert common >= min(r.iters, r1.iters, 256) > 0
        assert logs[i][:common] == single[:common], f"instance {i} (k = {inst.k})"
        assert r.F == pytest.approx(r1.F, rel=1e-6)
    rpca.rpca_destroy_batch(b)


def test_grouped_driver_mixed_lengths_and_repeat(monkeypatch):
    """Instances that finish at very different times (a tight and a loose tolerance share the
    batch through their sizes): every one is certified, a second solve of the same batch repeats
    the first exactly, and the threads driver reaches the same objectives."""
    monkeypatch.delenv("RPCA_BATCH_MODE", raising=False)
    insts = gen.batch_c4(10, seed=5, m_range=(1024, 6000), n_range=(50, 400))
    b, Xs = _batch(insts)
    Us, Vs = zip(*[empty_factors(i.m, i.n, i.k) for i in insts])
    st, res = rpca.rpca_solve_batch(b, Us, Vs)
    assert st == rpca.RPCA_OK and rpca.rpca_batch_driver(b) == rpca.RPCA_DRIVER_GROUPED
    Us2, Vs2 = zip(*[empty_factors(i.m, i.n, i.k) for i in insts])
    st2, res2 = rpca.rpca_solve_batch(b, Us2, Vs2)
    assert st2 == rpca.RPCA_OK
    for a, c in zip(res, res2):
        assert a.iters == c.iters and a.evals == c.evals and a.F == c.F
    monkeypatch.setenv("RPCA_BATCH_MODE", "threads")
    Us3, Vs3 = zip(*[empty_factors(i.m, i.n, i.k) for i in insts])
    st3, res3 = rpca.rpca_solve_batch(b, Us3, Vs3)
    assert st3 == rpca.RPCA_OK and rpca.rpca_batch_driver(b) == rpca.RPCA_DRIVER_THREADS
    for a, c in zip(res, res3):
        assert c.status == rpca.RPCA_OK and a.F == pytest.approx(c.F, rel=1e-6)
    rpca.rpca_destroy_batch(b)
