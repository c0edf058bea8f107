"""Pins of the reduced-precision storage formats of the oracle (oracle/quant.py).

Each check is against the formats' definitions: exactly representable values, halfway cases
of round-to-nearest-even, saturation, subnormals, and an independent brute-force rounding
(frexp / an argmin over every code) on random inputs.
"""
import math

import numpy as np

from oracle import quant


def _bf16_by_frexp(x):
    """bfloat16 rounding done independently: 8 significant bits, Python's round-half-even."""
    out = []
    for v in np.asarray(x, np.float64).ravel():
        if v == 0.0:
            out.append(0.0)
            continue
        m, e = math.frexp(v)          # v = m 2^e, 0.5 <= |m| < 1
        q = round(m * 256.0) / 256.0  # 8 significant bits; exact halves tie to even
        out.append(math.ldexp(q, e))
    return np.asarray(out).reshape(np.shape(x))


def test_bf16_exact_values_unchanged():
    vals = np.array([0.0, 1.0, -2.5, 0.15625, 3.0e38, -1.0e-30], np.float32)
    vals = quant.bf16_round(vals)  # project once, then it must be a fixed point
    assert np.array_equal(quant.bf16_round(vals), vals)
    assert quant.bf16_round(np.float32(1.0)) == 1.0


def test_bf16_ties_to_even():
    one = 1.0
    assert quant.bf16_round(np.float32(one + 2.0 ** -8)) == np.float32(1.0)                 # half of 2^-7, even is 1.0
    assert quant.bf16_round(np.float32(one + 3 * 2.0 ** -8)) == np.float32(1.0 + 2.0 ** -6)  # odd neighbour loses
    assert quant.bf16_round(np.float32(one + 2.0 ** -8 + 2.0 ** -20)) == np.float32(1.0 + 2.0 ** -7)


def test_bf16_matches_independent_rounding():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(4000) * np.exp(rng.uniform(-20, 20, 4000))).astype(np.float32)
    assert np.array_equal(quant.bf16_round(x).astype(np.float64), _bf16_by_frexp(x.astype(np.float64)))


def test_e4m3_grid_definition():
    vals = quant._E4M3_VALS
    assert len(vals) == 127               # 16 exponents x 8 fractions, minus the NaN code
    assert vals[0] == 0.0 and vals[1] == 2.0 ** -9   # smallest subnormal
    assert 2.0 ** -6 in vals                         # smallest normal
    assert vals[-1] == 448.0                         # largest finite
    assert np.all(np.diff(vals) > 0)


def test_e4m3_special_cases():
    r = quant.e4m3_round
    assert r(np.float32(1.0)) == 1.0
    assert r(np.float32(1.0625)) == 1.0       # halfway 1 .. 1.125: even code (fraction 0)
    assert r(np.float32(1.1875)) == 1.25      # halfway 1.125 .. 1.25: even code (fraction 2)
    assert r(np.float32(500.0)) == 448.0      # saturates, no infinity
    assert r(np.float32(-1e6)) == -448.0
    assert r(np.float32(2.0 ** -10)) == 0.0   # halfway 0 .. 2^-9: code 0 is even
    assert r(np.float32(3 * 2.0 ** -10)) == 2.0 ** -8
    assert r(np.float32(-0.3)) == -0.3125     # 0.3 lies between 0.28125 and 0.3125, nearer the latter


def test_e4m3_matches_bruteforce_argmin():
    rng = np.random.default_rng(5)
    y = (rng.standard_normal(3000) * np.exp(rng.uniform(-8, 6, 3000))).astype(np.float32)
    got = quant.e4m3_round(y)
    vals, codes = quant._E4M3_VALS, quant._E4M3_CODES
    for yi, gi in zip(y.astype(np.float64), got):
        a = min(abs(yi), 448.0)
        d = np.abs(vals - a)
        best = np.flatnonzero(d == d.min())
        pick = best[0] if len(best) == 1 else best[codes[best] % 2 == 0][0]
        assert gi == math.copysign(vals[pick], yi)


def test_e4m3_scales_and_stored_values():
    X = np.array([[1.0, 0.0, -3.0],
                  [-896.0, 0.0, 2.0]], np.float32)
    mask = np.array([[1, 1, 1],
                     [1, 1, 0]], np.uint8)
    s = quant.e4m3_scales(X, mask)
    assert s[0] == np.float32(896.0 / 448.0)
    assert s[1] == 1.0                             # all-zero column
    assert s[2] == np.float32(3.0 / 448.0)         # the unobserved 2.0 is ignored
    Xs = quant.stored_x(X, mask, "e4m3")
    assert Xs[1, 0] == -896.0 and Xs[1, 2] == 0.0  # column maximum is exact; unobserved -> 0
    assert Xs[0, 2] == -3.0
    Xb = quant.stored_x(X, mask, "bf16")
    assert Xb[1, 2] == 0.0 and Xb[0, 0] == 1.0
