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


@pytest.mark.parametrize("mode", ["rounds", "threads"])
def test_batch_solves_match_single_solves(mode, monkeypatch):
    """Both drivers of the batched form: rounds (one graph launch advances every instance, the
    default) and host threads stepping each instance's own graph."""
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
