"""GPU parity of the row-partitioned objective pass: G = 2, 3, 4 virtual shards on one GPU.

Each shard is a context on a row block of the same device X (rpca_fg_rows); the column-side
partials and the objective partials are summed over the shards in a fixed order (what the
all-reduce of a multi-GPU run does), and rpca_fg_rows_finish adds the shared V terms.  The
result must equal the unpartitioned evaluation (rpca_fg) to float32 rounding -- objective
1e-8 relative, gradient 1e-6 relative per block (the shards' tiles differ from the
unpartitioned tiling, so the float32 partial sums regroup) -- and the FP64 oracle at
the parity tolerances (1e-6, 1e-5), masked and unmasked, on the video workload too.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_1702_02241_gb300 import gen  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02241_gb300 import build
    build.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def sharded(Xd, ldx, m, n, k, lam_L, lam_S, U, V, G, Md=None):
    from paper_1702_02241_gb300 import rpca
    from paper_1702_02241_gb300.engine import from_device_colmajor, to_device_colmajor
    from paper_1702_02241_gb300.shard import RowShard, row_bounds
    b = row_bounds(m, G)
    Vd = to_device_colmajor(V)
    parts = []
    for g in range(G):
        sh = RowShard(Xd, ldx, b[g], b[g + 1], n, k, lam_L, lam_S, Md=Md, ldmask=ldx)
        Ug = to_device_colmajor(np.ascontiguousarray(U[b[g]:b[g + 1]]))
        gU, PV, f_part = sh.partials(Ug, Vd)
        parts.append((sh, gU, PV, f_part))
    PV_sum = parts[0][2].clone()
    for g in range(1, G):      # fixed order, as the exchange sums them
        PV_sum += parts[g][2]
    f_sum = 0.0
    for g in range(G):
        f_sum += parts[g][3]
    gV = torch.empty_like(Vd)
    f = rpca.rpca_fg_rows_finish(parts[0][0].ctx, Vd, PV_sum, f_sum, gV)
    torch.cuda.synchronize()
    gU = np.concatenate([from_device_colmajor(p[1], b[g + 1] - b[g]) for g, p in enumerate(parts)], axis=0)
    out = f, gU, from_device_colmajor(gV, n)
    for p in parts:
        p[0].close()
    return out


@pytest.mark.parametrize("G", [2, 3, 4])
@pytest.mark.parametrize("m,n,k,masked", [(3001, 260, 5, False), (9000, 130, 8, True), (512, 700, 3, False),
                                          (2050, 90, 12, True)])
def test_virtual_shards_match_unpartitioned(G, m, n, k, masked):
    from paper_1702_02241_gb300.engine import Problem, from_device_colmajor, to_device_colmajor
    g = np.random.default_rng(m + G)
    X = np.asfortranarray(g.normal(size=(m, n)).astype(np.float32))
    mask = np.asfortranarray((g.random((m, n)) < 0.6).astype(np.uint8)) if masked else None
    U, V = gen.factors(m, n, k, seed=G, scale=0.3)
    lam_L, lam_S = 0.8, 0.4
    P = Problem(X, mask, k, lam_L, lam_S)
    f1, gU1, gV1 = P.fg(to_device_colmajor(U), to_device_colmajor(V))
    gU1, gV1 = from_device_colmajor(gU1, m), from_device_colmajor(gV1, n)
    f, gU, gV = sharded(P.Xd, P.ldx, m, n, k, lam_L, lam_S, U, V, G, Md=P.Md)
    # The psi sums of each tile are float32 (Kahan-compensated) before float64: the shards'
    # tiles regroup them, which moves f by a few 1e-10 relative (measured 2.4e-10 at most).
    assert abs(f - f1) <= 1e-8 * abs(f1)
    assert rel(gU, gU1) <= 1e-6 and rel(gV, gV1) <= 1e-6
    fo, GUo, GVo = core.fg(X, mask, U, V, lam_L, lam_S)
    assert abs(f - fo) <= 1e-6 * abs(fo)
    assert rel(gU, GUo) <= 1e-5 and rel(gV, GVo) <= 1e-5
    P.close()


def test_virtual_shards_video_76800x1000():
    from paper_1702_02241_gb300.engine import Problem
    inst = gen.video_76800x1000(0)
    U, V = gen.factors(inst.m, inst.n, inst.k, seed=3, scale=0.2)
    P = Problem(inst.X, None, inst.k, inst.lam_L, inst.lam_S)
    f, gU, gV = sharded(P.Xd, P.ldx, inst.m, inst.n, inst.k, inst.lam_L, inst.lam_S, U, V, 4)
    fo, GUo, GVo = core.fg(inst.X, None, U, V, inst.lam_L, inst.lam_S)
    assert abs(f - fo) <= 1e-6 * abs(fo)
    assert rel(gU, GUo) <= 1e-5 and rel(gV, GVo) <= 1e-5
    P.close()
