"""The row-partitioned form of the objective pass on CPU: the host-side split and exchange.

* row_bounds: the blocks cover the rows exactly once, start on 16-byte boundaries of the
  column-major X (multiples of 4 rows), and are balanced.
* Two gloo ranks (127.0.0.1), each holding a row block of X and U and all of V: the FP64
  oracle stands in for the library's per-block pass (rpca_fg_rows computes the same terms on
  the GPU); shard.exchange sums the column-side partials and the objective partials over the
  ranks; adding the shared V terms gives F and the gradient of the unpartitioned problem.
  This is the separation F = sum_g (phi_g + lam_L/2 ||U_g||^2) + lam_L/2 ||V||^2,
  G_V = sum_g D_g^T U_g + lam_L V of Eq. (Thm5) and Sec. 3.2 over row blocks.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("m,parts", [(100, 2), (1001, 3), (76800, 8), (8, 2), (13, 3), (4096, 4)])
def test_row_bounds_cover_align_balance(m, parts):
    from paper_1702_02241_gb300.shard import row_bounds
    b = row_bounds(m, parts)
    assert b[0] == 0 and b[-1] == m and len(b) == parts + 1
    assert all(b[g] < b[g + 1] for g in range(parts))
    assert all(r % 4 == 0 for r in b[:-1])
    sizes = [b[g + 1] - b[g] for g in range(parts)]
    assert max(sizes) - min(sizes) <= 4 + (m % 4)


def test_row_bounds_rejects_too_many_parts():
    from paper_1702_02241_gb300.shard import row_bounds
    with pytest.raises(ValueError):
        row_bounds(7, 3)


def _problem():
    g = np.random.default_rng(4)
    m, n, k = 203, 57, 3
    X = g.normal(size=(m, n))
    mask = (g.random((m, n)) < 0.8).astype(np.uint8)
    U = 0.4 * g.normal(size=(m, k))
    V = 0.4 * g.normal(size=(n, k))
    return X, mask, U, V, 0.7, 0.3


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from oracle import core
    from paper_1702_02241_gb300.shard import exchange, row_bounds
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, mask, U, V, lam_L, lam_S = _problem()
        b = row_bounds(X.shape[0], world)
        r0, r1 = b[rank], b[rank + 1]
        Xg, Mg, Ug = X[r0:r1], mask[r0:r1], U[r0:r1]
        # This block's terms (what rpca_fg_rows computes on a GPU), from the oracle.
        R = core.residual(Xg, Ug, V)
        D = core.D_of_R(R, Mg, lam_S)
        f_part = core.phi_of_R(R, Mg, lam_S) + 0.5 * lam_L * float(np.sum(Ug * Ug))
        gU = D @ V + lam_L * Ug
        PV = torch.from_numpy(D.T @ Ug)
        PV_sum, f_sum = exchange(PV, f_part)
        gV = PV_sum.numpy() + lam_L * V
        f = f_sum + 0.5 * lam_L * float(np.sum(V * V))
        dist.barrier()
    finally:
        dist.destroy_process_group()
    out[rank] = (f, gU, gV, r0, r1)


def test_two_ranks_exchange_gives_the_unpartitioned_objective_and_gradient():
    import torch.multiprocessing as mp

    from oracle import core
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
        res = dict(out)
    X, mask, U, V, lam_L, lam_S = _problem()
    fo, GUo, GVo = core.fg(X, mask, U, V, lam_L, lam_S)
    for r in (0, 1):
        f, gU, gV, r0, r1 = res[r]
        assert f == pytest.approx(fo, rel=1e-13)
        assert np.allclose(gV, GVo, rtol=1e-12, atol=1e-12)
        assert np.allclose(gU, GUo[r0:r1], rtol=1e-12, atol=1e-12)
    assert res[0][3] == 0 and res[0][4] == res[1][3] and res[1][4] == X.shape[0]
