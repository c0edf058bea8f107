"""Shared helpers of the GPU parity tests (device copies, context construction)."""
import numpy as np
import torch

from paper_1702_02241_gb300 import rpca
from paper_1702_02241_gb300.engine import Problem, from_device_colmajor, to_device_colmajor


def make_problem(X, mask, k, lam_L, lam_S, **opts):
    o = rpca.rpca_default_options()
    for key, v in opts.items():
        setattr(o, key, v)
    return Problem(X, mask, k, lam_L, lam_S, opt=o)


def dev(A):
    return to_device_colmajor(np.asfortranarray(np.asarray(A, np.float32)))


def host(T, rows):
    return from_device_colmajor(T, rows)


def empty_factors(m, n, k):
    return (torch.zeros((k, m), dtype=torch.float32, device="cuda"),
            torch.zeros((k, n), dtype=torch.float32, device="cuda"))
