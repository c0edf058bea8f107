"""Row partition of one problem over several devices: the multi-GPU form of the objective pass.

X (m x n) and U (m x k) are split by rows over the ranks of a process group, V (n x k) is
held by every rank.  The objective of Eq. (Thm5) and its gradient (Sec. 3.2) separate over the
row blocks except for the column-side product, so one evaluation is

  1. on every rank, the fused pass over its rows (``rpca_fg_rows``): G_{U_g} = D_g V + lam_L U_g
     (complete), the partial D_g^T U_g (n x k) and f_g = sum psi + lam_L/2 ||U_g||^2;
  2. one all-reduce (sum) of [D_g^T U_g | f_g]: n k + 1 values;
  3. on every rank, ``rpca_fg_rows_finish``: G_V = sum_g D_g^T U_g + lam_L V and
     F = sum_g f_g + lam_L/2 ||V||^2.

This module holds only the host side of that: where the row blocks start (aligned so that a
block's first row is a 16-byte boundary of the column-major X, as the tiled TMA copies need),
and the exchange through ``torch.distributed``.  Every arithmetic step of the method runs in
the library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rpca

ROW_ALIGN = 4  # rows per 16 bytes of float32: a row block must start on a 16-byte boundary


def row_bounds(m: int, parts: int, align: int = ROW_ALIGN) -> list:
    """Boundaries r_0 = 0 < r_1 < ... < r_parts = m of `parts` row blocks of nearly equal size,
    every interior boundary a multiple of `align`.  Raises ValueError when m cannot give every
    part at least one aligned block."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    units = -(-m // align)  # aligned row groups (the last may be ragged)
    if units < parts:
        raise ValueError(f"{m} rows cannot be split into {parts} blocks aligned to {align} rows")
    b = [0]
    for g in range(1, parts):
        b.append(min(m, (units * g // parts) * align))
    b.append(m)
    return b


def exchange(PV: torch.Tensor, f_part: float, group=None):
    """Sums this rank's column-side partial PV (n x k, any device) and objective partial f_part
    over the ranks of `group` (torch.distributed, initialised): returns (PV_sum, f_sum).  The
    objective goes in float64; PV keeps its own type."""
    import torch.distributed as dist
    fs = torch.tensor([float(f_part)], dtype=torch.float64, device=PV.device)
    dist.all_reduce(PV, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(fs, op=dist.ReduceOp.SUM, group=group)
    return PV, float(fs.item())


class RowShard:
    """One rank's row block of a partitioned problem: the context on X[r0:r1], and the
    evaluation of F and the gradient of the whole problem at (U, V) where U is this block's
    rows of the factor (device, column-major (k, m_g)) and V is shared (device, (k, n))."""

    def __init__(self, Xd: torch.Tensor, ldx: int, r0: int, r1: int, n: int, k: int, lam_L: float, lam_S: float,
                 opt=None, stream=None, group=None, Md: torch.Tensor | None = None, ldmask: int = 0):
        if r0 % ROW_ALIGN:
            raise ValueError("a row block must start at a multiple of 4 rows")
        self.r0, self.r1, self.n, self.k = r0, r1, n, k
        self.group = group
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._X, self._M = Xd, Md  # keep the borrowed X and mask alive
        ptr = Xd.data_ptr() + 4 * r0
        mptr = Md.data_ptr() + r0 if Md is not None else None
        self.ctx = rpca.rpca_create(r1 - r0, n, ptr, ldx, mptr, ldmask if Md is not None else 0, k, lam_L, lam_S,
                                    opt, self.stream.cuda_stream)

    def close(self):
        if self.ctx:
            rpca.rpca_destroy(self.ctx)
            self.ctx = None

    def partials(self, U, V):
        """This block's terms: (gU, PV, f_part)."""
        gU = torch.empty_like(U)
        PV = torch.empty_like(V)
        f_part = rpca.rpca_fg_rows(self.ctx, U, V, gU, PV)
        return gU, PV, f_part

    def fg(self, U, V):
        """F of the whole problem and this rank's gradient blocks (gU rows of this block, gV
        shared), with one exchange over the process group."""
        gU, PV, f_part = self.partials(U, V)
        PV_sum, f_sum = exchange(PV, f_part, self.group)
        gV = torch.empty_like(V)
        f = rpca.rpca_fg_rows_finish(self.ctx, V, PV_sum, f_sum, gV)
        return f, gU, gV


def split_rows(A: np.ndarray, bounds) -> list:
    """Row blocks of a host matrix at the given boundaries."""
    return [A[bounds[g]:bounds[g + 1]] for g in range(len(bounds) - 1)]
