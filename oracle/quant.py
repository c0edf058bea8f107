"""Reduced-precision storage of X for the precision form of the objective pass, float64 host.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product.

The paper evaluates F and its gradient with X in float32 (Sec. 5).  The precision form stores
X in a narrower type, evaluates the same objective on the stored values (everything else in
float32), and finishes with float32 X.  What the stored values are is fixed by the formats
alone, and this module writes that down from their definitions:

* bfloat16: the top 16 bits of an IEEE-754 binary32 (8 exponent bits, 7 fraction bits), rounded
  to nearest with ties to even on the 16 dropped bits.
* FP8 E4M3 (the OCP 8-bit floating-point format): 1 sign bit, 4 exponent bits with bias 7,
  3 fraction bits; exponent field 0 holds subnormals (fraction * 2^-9); the largest finite
  magnitude is 448 (exponent field 15, fraction 110); there is no infinity; conversion rounds
  to nearest with ties to even and saturates to +-448 ("satfinite").  Each column j is stored
  as x / s_j with s_j = max_i |x_ij| / 448 over its observed entries (float32 division; s_j = 1
  for an all-zero column), and read back as float32(e4m3 value) * s_j in float32.

Unobserved entries (mask 0) are stored as 0.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def bf16_round(x):
    """float32 array -> float32 values representable in bfloat16 (round to nearest even)."""
    x = np.ascontiguousarray(np.asarray(x, np.float32))
    bits = x.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return out.reshape(np.shape(x))


def _e4m3_grid():
    """All non-negative finite E4M3 values, ascending, with their bit patterns."""
    vals, codes = [], []
    for e in range(16):
        for f in range(8):
            if e == 15 and f == 7:
                continue  # NaN encoding
            if e == 0:
                v = f * 2.0 ** -9
            else:
                v = (1.0 + f / 8.0) * 2.0 ** (e - 7)
            vals.append(v)
            codes.append((e << 3) | f)
    order = np.argsort(vals, kind="stable")
    return np.asarray(vals, np.float64)[order], np.asarray(codes, np.int64)[order]


_E4M3_VALS, _E4M3_CODES = _e4m3_grid()


def e4m3_round(y):
    """Nearest E4M3 value (ties to the even code, saturating at +-448) of float32 inputs,
    returned as float64."""
    y = np.asarray(y, np.float32).astype(np.float64)
    a = np.minimum(np.abs(y), E4M3_MAX)
    idx = np.searchsorted(_E4M3_VALS, a, side="left")
    idx = np.clip(idx, 0, len(_E4M3_VALS) - 1)
    hi = _E4M3_VALS[idx]
    lo = _E4M3_VALS[np.maximum(idx - 1, 0)]
    code_hi = _E4M3_CODES[idx]
    d_hi = hi - a
    d_lo = a - lo
    pick_lo = (d_lo < d_hi) | ((d_lo == d_hi) & (code_hi % 2 == 1))
    pick_lo &= idx > 0
    v = np.where(pick_lo, lo, hi)
    return np.sign(y) * v


def e4m3_scales(X, mask=None):
    """Per-column scales s_j = max |X_ij| / 448 over observed entries, in float32."""
    X = np.asarray(X, np.float32)
    A = np.abs(X)
    if mask is not None:
        A = np.where(np.asarray(mask) != 0, A, np.float32(0))
    mx = A.max(axis=0).astype(np.float32)
    s = (mx / np.float32(E4M3_MAX)).astype(np.float32)
    return np.where(mx > 0, s, np.float32(1.0)).astype(np.float32)


def stored_x(X, mask, dtype):
    """The values the objective pass reads for X stored as `dtype` ("f32", "bf16", "e4m3"),
    as float64 (unobserved entries 0)."""
    X = np.asarray(X, np.float32)
    obs = np.ones(X.shape, bool) if mask is None else np.asarray(mask) != 0
    X0 = np.where(obs, X, np.float32(0))
    if dtype == "f32":
        return X0.astype(np.float64)
    if dtype == "bf16":
        return bf16_round(X0).astype(np.float64)
    if dtype == "e4m3":
        s = e4m3_scales(X, mask)
        q = e4m3_round((X0 / s[None, :]).astype(np.float32))
        return (q.astype(np.float32) * s[None, :]).astype(np.float32).astype(np.float64)
    raise ValueError(dtype)
