"""Python-side convenience over the C ABI: device copies of numpy inputs, column-major
layout helpers, and a ``Problem`` object that owns an rpca context.

PyTorch is used only for device memory and streams; all arithmetic of the method runs in
librpca.so.  Column-major convention: an m x n matrix lives in a contiguous torch tensor of
shape (n, ld) (ld >= m, padded to a multiple of 4 so rows start 16-byte aligned for TMA).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import rpca


def ld_for(m: int) -> int:
    return (m + 3) // 4 * 4


def to_device_colmajor(A: np.ndarray, dtype=torch.float32, pad: bool = False, device="cuda") -> torch.Tensor:
    """Copy an m x n numpy array to a contiguous (n, ld) device tensor (column-major m x n)."""
    m, n = A.shape
    ld = ld_for(m) if pad else m
    host = torch.zeros((n, ld), dtype=dtype)
    host[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T).astype(torch_to_np(dtype), copy=False))
    return host.to(device)


def torch_to_np(dtype):
    return {torch.float32: np.float32, torch.uint8: np.uint8, torch.float64: np.float64}[dtype]


def from_device_colmajor(T: torch.Tensor, m: int) -> np.ndarray:
    """Inverse of to_device_colmajor: (n, ld) tensor -> m x n float64 numpy array."""
    return T[:, :m].double().cpu().numpy().T


def empty_factor(rows: int, k: int, device="cuda") -> torch.Tensor:
    return torch.zeros((k, rows), dtype=torch.float32, device=device)


class Problem:
    """Device copy of one instance and its rpca context."""

    def __init__(self, X: np.ndarray, mask: np.ndarray | None, k: int, lam_L: float, lam_S: float,
                 opt: rpca.rpca_options | None = None, stream: torch.cuda.Stream | None = None, Xd=None, Md=None):
        self.m, self.n = X.shape if X is not None else (None, None)
        self.k = k
        self.lam_L, self.lam_S = lam_L, lam_S
        self.Xd = Xd if Xd is not None else to_device_colmajor(X, pad=True)
        if self.m is None:
            self.n, ld = self.Xd.shape
        self.ldx = self.Xd.shape[1]
        if mask is not None or Md is not None:
            self.Md = Md if Md is not None else to_device_colmajor(mask.astype(np.uint8), dtype=torch.uint8, pad=True)
        else:
            self.Md = None
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = rpca.rpca_create(self.m, self.n, self.Xd, self.ldx, self.Md, self.ldx if self.Md is not None else 0,
                                    k, lam_L, lam_S, opt, self.stream.cuda_stream)

    def close(self):
        if self.ctx:
            rpca.rpca_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factors(self, U: np.ndarray, V: np.ndarray):
        return to_device_colmajor(U), to_device_colmajor(V)

    def fg(self, U: torch.Tensor, V: torch.Tensor):
        gU = torch.empty_like(U)
        gV = torch.empty_like(V)
        f = rpca.rpca_fg(self.ctx, U, V, gU, gV)
        return f, gU, gV

    def apply(self, U, V, Bv, Bu):
        b = Bv.shape[0]
        DBv = torch.empty((b, self.m), dtype=torch.float32, device=U.device)
        DtBu = torch.empty((b, self.n), dtype=torch.float32, device=U.device)
        rpca.rpca_apply(self.ctx, U, V, b, Bv, Bu, DBv, DtBu)
        return DBv, DtBu

    def solve(self, U, V):
        return rpca.rpca_solve(self.ctx, U, V)

    def certificate(self, U, V):
        return rpca.rpca_certificate(self.ctx, U, V)

    def init_sketch(self, U, V, Omega=None):
        rpca.rpca_init_sketch(self.ctx, Omega, U, V)


def rel(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def isinf(x) -> bool:
    return isinstance(x, float) and math.isinf(x)
