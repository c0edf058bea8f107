"""GPU parity of the precision form: X stored as bfloat16 or FP8 E4M3 (per-column scale).

* Storage: the library's copy of X equals the oracle's rounding of X bit for bit (bfloat16
  bits; E4M3 codes decoded to values; the FP8 column scales).
* Objective pass: F and its gradient read from the stored copy equal the FP64 oracle on the
  stored values (oracle.quant.stored_x) at the float32 tolerances (1e-6 / 1e-5 relative).
* Solve: iterations on the stored copy, then float32 refinement, reach cert_rel <= 1e-4 on
  the float32 problem with the float32 solve's objective (1e-6 relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core, quant  # noqa: E402
from paper_1702_02241_gb300 import gen, rpca  # noqa: E402

from gpu_util import empty_factors, host, make_problem  # noqa: E402

F_TOL, G_TOL = 1e-6, 1e-5
DTYPES = {"bf16": rpca.RPCA_BF16, "e4m3": rpca.RPCA_FP8E4M3}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def case(m, n, k, seed, mask_p):
    g = np.random.default_rng(seed)
    X = np.asfortranarray((g.normal(size=(m, n)) * np.exp(g.uniform(-3, 3, size=(1, n)))).astype(np.float32))
    mask = None if mask_p is None else np.asfortranarray((g.random((m, n)) < mask_p).astype(np.uint8))
    U, V = gen.factors(m, n, k, seed + 100, scale=0.5)
    return X, mask, U, V


def decode_e4m3(codes):
    vals = np.zeros(256)
    for e in range(16):
        for f in range(8):
            v = f * 2.0 ** -9 if e == 0 else (1 + f / 8) * 2.0 ** (e - 7)
            vals[(e << 3) | f] = v
            vals[0x80 | (e << 3) | f] = -v
    return vals[codes]


@pytest.mark.parametrize("dt", ["bf16", "e4m3"])
@pytest.mark.parametrize("mask_p", [None, 0.5])
def test_storage_matches_oracle(dt, mask_p):
    X, mask, U, V = case(777, 130, 5, 3, mask_p)
    P = make_problem(X, mask, 5, 0.7, 0.3, x_dtype=DTYPES[dt])
    got_dt, stored, scales = rpca.rpca_x_storage(P.ctx, X.shape[0], X.shape[1])
    P.close()
    assert got_dt == DTYPES[dt]
    obs = np.ones(X.shape, bool) if mask is None else mask != 0
    X0 = np.where(obs, X, np.float32(0))
    if dt == "bf16":
        want = (quant.bf16_round(X0).view(np.uint32) >> 16).astype(np.uint16)
        assert np.array_equal(stored, want)
    else:
        s = quant.e4m3_scales(X, mask)
        assert np.array_equal(scales, s)
        want = quant.e4m3_round((X0 / s[None, :]).astype(np.float32))
        assert np.array_equal(decode_e4m3(stored.astype(np.int64)), want)


@pytest.mark.parametrize("dt", ["bf16", "e4m3"])
@pytest.mark.parametrize("m,n,k,mask_p", [(3000, 260, 5, None), (2100, 130, 8, 0.5), (1001, 77, 1, None),
                                          (4099, 301, 6, 0.3), (64, 8, 2, None)])
def test_fg_on_stored_values(dt, m, n, k, mask_p):
    from paper_1702_02241_gb300.engine import from_device_colmajor, to_device_colmajor
    X, mask, U, V = case(m, n, k, m + n + k, mask_p)
    P = make_problem(X, mask, k, 0.7, 0.3, x_dtype=DTYPES[dt])
    f, gU, gV = P.fg(to_device_colmajor(U), to_device_colmajor(V))
    torch.cuda.synchronize()
    gU = from_device_colmajor(gU, m)
    gV = from_device_colmajor(gV, n)
    P.close()
    Xs = quant.stored_x(X, mask, dt)
    fo, GUo, GVo = core.fg(Xs, mask, U, V, 0.7, 0.3)
    assert abs(f - fo) <= F_TOL * abs(fo), (f, fo)
    G = np.concatenate([gU.ravel(), gV.ravel()])
    Go = np.concatenate([GUo.ravel(), GVo.ravel()])
    assert np.linalg.norm(G - Go) <= G_TOL * np.linalg.norm(Go)


@pytest.mark.parametrize("dt", ["bf16", "e4m3"])
def test_precision_form_solve_refines_to_float32(dt):
    inst = gen.video(h=48, w=64, n=200, rank=3, k=5, mask_p=0.5, seed=2)
    ref = make_problem(inst.X, inst.mask, inst.k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH,
                       max_iter=3000, cert_every=10)
    U0, V0 = empty_factors(inst.m, inst.n, inst.k)
    r0 = ref.solve(U0, V0)
    ref.close()
    assert r0.status == rpca.RPCA_OK
    P = make_problem(inst.X, inst.mask, inst.k, inst.lam_L, inst.lam_S, init=rpca.RPCA_INIT_SKETCH,
                     max_iter=3000, cert_every=10, x_dtype=DTYPES[dt], refine_fp32=1)
    Ud, Vd = empty_factors(inst.m, inst.n, inst.k)
    r = P.solve(Ud, Vd)
    assert r.status == rpca.RPCA_OK, rpca.rpca_last_error(P.ctx)
    assert r.cert.cert_rel <= 1e-4
    U, V = host(Ud, inst.m), host(Vd, inst.n)
    Fo = core.objective(inst.X, inst.mask, U, V, inst.lam_L, inst.lam_S)
    assert r.F == pytest.approx(Fo, rel=1e-6)
    assert Fo == pytest.approx(r0.F, rel=1e-6)
    P.close()


# Bounds on the narrow phase alone (iterations on the stored copy of X, no float32
# refinement) against the FP64 oracle's optimum on float32 X: relative objective error,
# ||L - L*||_F / ||L*||_F, and the symmetric difference of the supports of S as a fraction of
# the observed entries.  The paper prints no such bounds; these are the ones proposed for
# bfloat16 and for E4M3 with per-column scales, checked here on a masked video-shaped instance.
NARROW_BOUNDS = {"bf16": (1e-2, 5e-3, 0.01), "e4m3": (5e-2, 3e-2, 0.05)}


@pytest.mark.parametrize("dt", ["bf16", "e4m3"])
def test_narrow_phase_error_against_fp64_oracle(dt):
    from oracle import lbfgs, sketch
    inst = gen.video(h=48, w=64, n=200, rank=3, k=5, mask_p=0.5, seed=4)
    X, mask, k, lam_L, lam_S = inst.X, inst.mask, inst.k, inst.lam_L, inst.lam_S
    Om = gen.gaussian(inst.n, k + 10, seed=5)
    U0, V0 = sketch.rsvd_init(X, mask, k, Om)
    ref = lbfgs.solve(X, mask, U0, V0, lam_L, lam_S, gtol=1e-10, max_iter=5000)
    Ls = ref.U @ ref.V.T
    Fs = core.objective(X, mask, ref.U, ref.V, lam_L, lam_S)
    # The narrow phase alone: iterate on the stored copy until its gradient test stops it.
    P = make_problem(X, mask, k, lam_L, lam_S, init=rpca.RPCA_INIT_SKETCH, max_iter=3000, cert_every=0,
                     gtol=1e-6, x_dtype=DTYPES[dt], refine_fp32=0)
    Ud, Vd = empty_factors(inst.m, inst.n, k)
    P.solve(Ud, Vd)
    U, V = host(Ud, inst.m), host(Vd, inst.n)
    P.close()
    L = U @ V.T
    obj = abs(core.objective(X, mask, U, V, lam_L, lam_S) - Fs) / Fs
    lerr = np.linalg.norm(L - Ls) / np.linalg.norm(Ls)
    obs = mask != 0
    X64 = X.astype(np.float64)
    supp = (np.abs(X64 - L) > lam_S) & obs
    supp_s = (np.abs(X64 - Ls) > lam_S) & obs
    serr = np.count_nonzero(supp ^ supp_s) / np.count_nonzero(obs)
    print(f"narrow phase {dt}: objective {obj:.3e}, L {lerr:.3e}, support {serr:.3e}")
    b = NARROW_BOUNDS[dt]
    assert obj <= b[0] and lerr <= b[1] and serr <= b[2], (obj, lerr, serr)
