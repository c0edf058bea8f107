"""Randomized-SVD initialisation (Sec. 4.2) on the GPU against the oracle with the same
Gaussian test matrix.  Compared on the rank-k product U0 V0^T (unique when the k-th and
(k+1)-th singular values are separated) and on the balance U0^T U0 = V0^T V0."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sketch  # noqa: E402
from paper_1702_02241_gb300 import gen  # noqa: E402

from gpu_util import dev, empty_factors, host, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


@pytest.mark.parametrize("m,n,k,masked", [(600, 300, 5, False), (1000, 200, 4, True), (700, 500, 16, False)])
def test_sketch_matches_oracle(m, n, k, masked):
    inst = gen.planted(m, n, rank=k, k=k, p_outlier=0.0, noise=1e-3, seed=k,
                       mask_p=0.6 if masked else None)
    l = k + 10
    Om = gen.gaussian(n, l, seed=5)
    U0, V0 = sketch.rsvd_init(inst.X, inst.mask, k, Om, q=2)
    P = make_problem(inst.X, inst.mask, k, inst.lam_L, inst.lam_S)
    Ud, Vd = empty_factors(m, n, k)
    P.init_sketch(Ud, Vd, Omega=dev(Om))
    U, V = host(Ud, m), host(Vd, n)
    Lg, Lo = U @ V.T, U0 @ V0.T
    assert np.linalg.norm(Lg - Lo) <= 1e-4 * np.linalg.norm(Lo)
    assert np.allclose(U.T @ U, V.T @ V, atol=1e-4 * np.abs(U.T @ U).max())
    assert np.allclose(np.linalg.norm(U, axis=0), np.linalg.norm(U0, axis=0), rtol=1e-4)
    P.close()
