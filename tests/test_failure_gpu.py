"""Failure detection on the GPU, in the forms that fault nothing.

* A bounded device wait that runs out: the fused kernel's producer is told to issue no
  copies (rpca_inject_fault), so the consumers' waits on the stage barriers give up after
  1 ms; the call reports RPCA_ETIMEOUT and the context stays usable (the next evaluation
  matches the FP64 oracle).
* Device allocation failure at context set-up, injected on the host: RPCA_ENOMEM, and a
  later rpca_create succeeds.
* Non-finite observed X is rejected at rpca_create (RPCA_EINVAL); a non-finite value at an
  unobserved entry is accepted and contributes nothing (Sec. 6.2: only Omega enters phi).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_1702_02241_gb300 import gen  # noqa: E402

from gpu_util import dev, host, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def _check_fg(P, X, mask, U, V, lam_L, lam_S):
    f, gU, gV = P.fg(dev(U), dev(V))
    fo, GUo, GVo = core.fg(X, mask, U, V, lam_L, lam_S)
    assert abs(f - fo) <= 1e-6 * abs(fo)
    assert np.linalg.norm(host(gU, X.shape[0]) - GUo) <= 1e-5 * np.linalg.norm(GUo)
    assert np.linalg.norm(host(gV, X.shape[1]) - GVo) <= 1e-5 * np.linalg.norm(GVo)


def test_bounded_wait_runs_out_and_context_stays_usable():
    from paper_1702_02241_gb300 import rpca
    g = np.random.default_rng(0)
    m, n, k = 3000, 260, 5
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    U, V = gen.factors(m, n, k, seed=1, scale=0.2)
    P = make_problem(X, None, k, 0.7, 0.3)
    rpca.rpca_inject_fault(P.ctx, rpca.RPCA_FAULT_FG_STARVE, 1)
    with pytest.raises(rpca.RpcaError) as ei:
        P.fg(dev(U), dev(V))
    assert ei.value.status == rpca.RPCA_ETIMEOUT
    assert "wait" in rpca.rpca_last_error(P.ctx)
    torch.cuda.synchronize()
    _check_fg(P, X, None, U, V, 0.7, 0.3)       # the fault was consumed; same context
    P.close()


@pytest.mark.parametrize("nth", [1, 3])
def test_allocation_failure_at_create(nth):
    from paper_1702_02241_gb300 import rpca
    g = np.random.default_rng(1)
    m, n, k = 500, 300, 4
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    mask = np.asfortranarray((g.random((m, n)) < 0.7).astype(np.uint8))
    rpca.rpca_inject_fault(None, rpca.RPCA_FAULT_ALLOC, nth)
    try:
        with pytest.raises(rpca.RpcaError) as ei:
            make_problem(X, mask, k, 1.0, 0.5)
        assert ei.value.status == rpca.RPCA_ENOMEM
    finally:
        rpca.rpca_inject_fault(None, rpca.RPCA_FAULT_ALLOC, 0)
    U, V = gen.factors(m, n, k, seed=2, scale=0.3)
    P = make_problem(X, mask, k, 1.0, 0.5)
    _check_fg(P, X, mask, U, V, 1.0, 0.5)
    P.close()


@pytest.mark.parametrize("bad", [math.nan, math.inf, -math.inf])
def test_nonfinite_observed_x_rejected_unobserved_accepted(bad):
    from paper_1702_02241_gb300 import rpca
    g = np.random.default_rng(2)
    m, n, k = 400, 150, 3
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    X[123, 45] = bad
    with pytest.raises(rpca.RpcaError) as ei:
        make_problem(X, None, k, 1.0, 0.5)
    assert ei.value.status == rpca.RPCA_EINVAL
    assert "non-finite" in rpca.rpca_last_error(None)
    mask = np.ones((m, n), np.uint8, order="F")
    mask[123, 45] = 0
    U, V = gen.factors(m, n, k, seed=3, scale=0.3)
    P = make_problem(X, mask, k, 1.0, 0.5)
    Xo = X.copy()
    Xo[123, 45] = 0.0   # the oracle never reads an unobserved entry either; keep it finite
    _check_fg(P, Xo, mask, U, V, 1.0, 0.5)
    P.close()
