"""TSQR: the QR factorisation of a tall-skinny matrix by a reduction tree of small QRs, in
float64 (Sec. 6.1, which takes it from Demmel, Grigori, Hoemmen and Langou, "Communication-
optimal parallel and sequential QR and LU factorizations", 2012).

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

For A (rows x l, rows >= l):
  1. split the rows into blocks A_1 .. A_P and factor each, A_p = Q_p R_p (l x l R_p);
  2. stack the R_p in groups, factor each stack, and repeat on the new R's until one R is left;
  3. Q is the product of the block-diagonal Q's of every level, applied top-down: the root's
     Q, sliced l rows per child, multiplies each child's Q, down to the leaves.
The library QR (LAPACK Householder through numpy) serves as the small QR of each node.  The
factorisation is normalised so that R has a non-negative diagonal; for A of full column rank
that QR is unique, so every tree shape gives the same Q and R (up to rounding).
"""
from __future__ import annotations

import numpy as np


def _split(rows, block_rows):
    """Row ranges of the leaves: blocks of block_rows, the last one taking the remainder."""
    nb = max(1, rows // block_rows)
    edges = [p * block_rows for p in range(nb)] + [rows]
    return list(zip(edges[:-1], edges[1:]))


def tsqr(A, block_rows=64, fan_in=4):
    """Return (Q, R): Q rows x l with orthonormal columns, R l x l upper triangular with a
    non-negative diagonal, A = Q R."""
    A = np.asarray(A, np.float64)
    rows, l = A.shape
    if rows < l:
        raise ValueError("TSQR needs rows >= columns")
    block_rows = max(block_rows, l)
    ranges = _split(rows, block_rows)
    # Level 0: the leaves.
    leaf_Q, Rs = [], []
    for a, b in ranges:
        q, r = np.linalg.qr(A[a:b])
        leaf_Q.append(q)
        Rs.append(r)
    # Upper levels: groups of fan_in stacked R's.
    levels = []  # per level: list of (children indices, Q of the stack)
    while len(Rs) > 1:
        groups = [list(range(g, min(len(Rs), g + fan_in))) for g in range(0, len(Rs), fan_in)]
        nodes, newR = [], []
        for ch in groups:
            q, r = np.linalg.qr(np.vstack([Rs[c] for c in ch]))
            nodes.append((ch, q))
            newR.append(r)
        levels.append(nodes)
        Rs = newR
    R = Rs[0]
    d = np.where(np.diag(R) < 0, -1.0, 1.0)
    R = d[:, None] * R
    # Top-down: E (l x l) of every node maps its subtree's Q to the final Q.
    E = [np.diag(d)]
    for nodes in reversed(levels):
        nxt = {}
        for (ch, q), e in zip(nodes, E):
            for s, c in enumerate(ch):
                nxt[c] = q[s * l:(s + 1) * l] @ e
        E = [nxt[c] for c in range(len(nxt))]
    Q = np.vstack([leaf_Q[p] @ E[p] for p in range(len(ranges))])
    return Q, R
