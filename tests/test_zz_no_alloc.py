"""rpca_fg_noalloc: the evaluation entry point for callers that cannot allocate device
memory (it takes its scratch from a fixed device array inside the library).

Checked through the C ABI against rpca_fg (the context-based entry point) on the same
inputs, within the tolerances of the parity tests (objective 1e-6 relative, gradient 1e-5
relative, each gradient block on its own), on two calls in a row (the second call reuses the
array the first one left behind), then on a different point; against the FP64 oracle
directly as well; over k = 1 .. 16 and small m (where the fixed launch configuration takes
its narrowest CTA), and the over-size rejection.  This file is collected last on purpose; it
passes on its own in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1702_02241_gb300 import gen  # noqa: E402

F_TOL, G_TOL = 1e-6, 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def rel(a, b):
    a = a.double().flatten()
    b = b.double().flatten()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("m,n,k", [(3000, 260, 5), (501, 403, 10), (76800, 1000, 5), (100, 300, 16),
                                   (2000, 150, 1), (5000, 200, 16), (130, 77, 3)])
def test_noalloc_matches_rpca_fg_twice(m, n, k):
    from oracle import core
    from paper_1702_02241_gb300 import rpca
    from paper_1702_02241_gb300.engine import Problem, from_device_colmajor, to_device_colmajor
    if m == 76800:
        inst = gen.video_76800x1000(0)
        X, lam_L, lam_S = inst.X, inst.lam_L, inst.lam_S
    else:
        g = np.random.default_rng(m + k)
        X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
        lam_L, lam_S = 0.7, 0.3
    P = Problem(X, None, k, lam_L, lam_S)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (1, 2):
        U, V = gen.factors(m, n, k, seed=seed, scale=0.2)
        Ud, Vd = to_device_colmajor(U), to_device_colmajor(V)
        f_ref, gU_ref, gV_ref = P.fg(Ud, Vd)
        fo, GUo, GVo = core.fg(X, None, U, V, lam_L, lam_S)
        for _ in range(2):  # two calls in a row on the same inputs
            gU = torch.full_like(Ud, float("nan"))
            gV = torch.full_like(Vd, float("nan"))
            f = rpca.rpca_fg_noalloc(m, n, P.Xd, P.ldx, k, lam_L, lam_S, Ud, Vd, gU, gV, stream)
            assert abs(f - f_ref) <= F_TOL * abs(f_ref), (f, f_ref)
            assert rel(gU, gU_ref) <= G_TOL and rel(gV, gV_ref) <= G_TOL
            # and against the FP64 oracle on the same values
            assert abs(f - fo) <= F_TOL * abs(fo), (f, fo)
            gUh, gVh = from_device_colmajor(gU, m), from_device_colmajor(gV, n)
            assert np.linalg.norm(gUh - GUo) <= G_TOL * np.linalg.norm(GUo)
            assert np.linalg.norm(gVh - GVo) <= G_TOL * np.linalg.norm(GVo)
    P.close()


def test_noalloc_rejects_shapes_beyond_its_scratch():
    from paper_1702_02241_gb300 import rpca
    m, n, k = 1 << 21, 64, 16
    X = torch.empty((n, m), dtype=torch.float32, device="cuda")
    U = torch.zeros((k, m), dtype=torch.float32, device="cuda")
    V = torch.zeros((k, n), dtype=torch.float32, device="cuda")
    with pytest.raises(rpca.RpcaError) as ei:
        rpca.rpca_fg_noalloc(m, n, X, m, k, 1.0, 1.0, U, V, torch.empty_like(U), torch.empty_like(V))
    assert ei.value.status == rpca.RPCA_EINVAL
    assert "scratch" in rpca.rpca_last_error(None)
