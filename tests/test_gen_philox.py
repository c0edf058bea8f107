"""Host Philox4x32-10 (paper_1702_02241_gb300.gen) against the published known-answer
vectors of Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
(SC 2011; the Random123 distribution's philox4x32_10 test vectors), and the planted
generator's draw statistics."""
import numpy as np

from paper_1702_02241_gb300 import gen

KAT = [  # (counter, key, output)
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


def test_known_answer_vectors():
    for ctr, key, want in KAT:
        assert tuple(int(v) for v in gen.philox4x32_10(ctr, key)) == want


def test_vectorised_equals_scalar():
    g = np.random.default_rng(0)
    c = g.integers(0, 2 ** 32, size=(50, 4), dtype=np.uint64)
    out = gen.philox4x32_10(c, (123, 456))
    for i in range(50):
        assert np.array_equal(out[i], gen.philox4x32_10(c[i], (123, 456)))


def test_planted_draw_statistics():
    X, L0, out = gen.planted_philox(400, 300, 5, 0.06, 1e-2, 7, 3)
    assert abs(out.mean() - 0.06) < 0.004
    assert abs(np.var(L0) - 1.0) < 0.15           # unit-variance entries of A B^T
    N = X - L0 - np.where(out, X - L0, 0.0)
    assert abs(np.std(N[~out]) - 1e-2) < 1e-3
    mag = np.abs((X - L0)[out])
    assert mag.min() > 0.95 and mag.max() < 5.05  # magnitude U[1, 5] plus noise
    assert np.linalg.matrix_rank(L0, tol=1e-8 * np.linalg.norm(L0)) == 5
