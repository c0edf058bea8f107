"""Seeded synthetic RPCA instances (X = L + S + N) shared by the oracle side and the CUDA side.

This module holds no arithmetic of the method itself (no Huber function, no gradient, no
solver): it only draws random matrices.  Everything is NumPy PCG64, seeded, so the same
call returns bit-identical arrays on every machine.

Matrices are returned column-major (NumPy Fortran order): X is m x n with the frames of a
video as columns, U is m x k and V is n x k.  X is handed out in float32, which is the
precision the data is stored in on both sides; the oracle promotes it to float64.

Instance families (the paper's own datasets are not available, these stand in for them):

* ``planted``   -- the small planted problem: L = A B^T (A, B iid normal with variance
  1/sqrt(rank), so L has unit-variance entries), outliers on an iid Bernoulli(p) support with
  random sign and magnitude U[1, 5], Gaussian noise.  Stands in for the paper's synthetic
  experiment (Sec. 5.3), scaled down.
* ``video``     -- a surveillance-video-shaped matrix (Sec. 5.2 and 5.4 work on unfolded
  videos, one frame per column): a rank-r smooth background with per-frame gain drift,
  three moving opaque rectangles as foreground, Gaussian sensor noise and an optional
  Bernoulli observation mask.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Instance:
    """One synthetic problem.  ``X`` float32 (m, n) Fortran order; ``mask`` uint8 or None."""

    X: np.ndarray
    mask: np.ndarray | None
    k: int
    lam_L: float
    lam_S: float
    L0: np.ndarray | None = None  # planted low-rank part (float64), when known
    S0: np.ndarray | None = None  # planted sparse part (float64), when known
    name: str = ""

    @property
    def m(self) -> int:
        return self.X.shape[0]

    @property
    def n(self) -> int:
        return self.X.shape[1]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def planted(m: int = 500, n: int = 400, rank: int = 5, k: int = 10, p_outlier: float = 0.05,
            noise: float = 1e-3, lam_L: float = 1.0, lam_S: float | None = None, seed: int = 0,
            mask_p: float | None = None) -> Instance:
    """Planted low-rank + sparse + noise.  Defaults are the 500 x 400, rank-5 problem.

    A, B ~ N(0, 1/sqrt(rank)) (variance), so each entry of L = A B^T has unit variance.
    Outliers: iid Bernoulli(p_outlier) positions, sign +-1 with probability 1/2, magnitude
    U[1, 5].  Noise: iid N(0, noise^2).  lam_S defaults to 1/sqrt(n).
    """
    g = rng(seed)
    std = (1.0 / math.sqrt(rank)) ** 0.5
    A = g.normal(0.0, std, size=(m, rank))
    B = g.normal(0.0, std, size=(n, rank))
    L0 = A @ B.T
    supp = g.random((m, n)) < p_outlier
    sign = np.where(g.random((m, n)) < 0.5, -1.0, 1.0)
    mag = g.uniform(1.0, 5.0, size=(m, n))
    S0 = np.where(supp, sign * mag, 0.0)
    N = g.normal(0.0, noise, size=(m, n))
    X = np.asfortranarray((L0 + S0 + N).astype(np.float32))
    mask = None
    if mask_p is not None:
        mask = np.asfortranarray((g.random((m, n)) < mask_p).astype(np.uint8))
    if lam_S is None:
        lam_S = 1.0 / math.sqrt(n)
    return Instance(X=X, mask=mask, k=k, lam_L=lam_L, lam_S=lam_S, L0=L0, S0=S0,
                    name=f"planted{m}x{n}r{rank}")


def _smooth_field(g: np.random.Generator, h: int, w: int, n_cos: int = 3) -> np.ndarray:
    """A smooth random image: random affine ramp plus a few low-frequency cosines, in [-1, 1]."""
    yy, xx = np.meshgrid(np.linspace(0.0, 1.0, h), np.linspace(0.0, 1.0, w), indexing="ij")
    f = g.uniform(-1, 1) * (xx - 0.5) + g.uniform(-1, 1) * (yy - 0.5)
    for _ in range(n_cos):
        fx, fy = g.uniform(0.2, 2.0, size=2)
        ph = g.uniform(0, 2 * math.pi)
        f = f + g.uniform(0.2, 0.6) * np.cos(2 * math.pi * (fx * xx + fy * yy) + ph)
    f = f - f.mean()
    return f / max(np.abs(f).max(), 1e-12)


def video(h: int = 240, w: int = 320, n: int = 1000, rank: int = 3, k: int = 5,
          n_rect: int = 3, rect: int = 30, noise: float = 0.01, mask_p: float | None = None,
          lam_L: float | None = None, lam_S: float | None = None, seed: int = 0,
          keep_parts: bool = False) -> Instance:
    """Video-shaped instance: m = h*w pixels per frame (column-major inside a frame), n frames.

    Background: L[:, t] = g_t * (B_0 + sum_q beta_q(t) B_q), q = 1..rank-1, where B_0 is a
    smooth field mapped to [0.2, 0.6], B_q are smooth fields scaled to +-0.05, beta_q(t) are
    slow sinusoids in [-1, 1] with random period and phase, and g_t ~ U[0.95, 1.05] is the
    per-frame gain.  The background therefore has rank `rank` and values in about [0.1, 0.7].
    Foreground: `n_rect` opaque rect x rect squares of constant intensity U[0.3, 1] moving at
    1-3 px/frame and bouncing off the frame edges; where they are, X shows the square
    instead of the background (so S = fg - L there).  Noise N(0, noise^2) everywhere.
    Optional Bernoulli(mask_p) observation mask.  lam_S defaults to 1/sqrt(n); lam_L defaults
    to 4 * lam_S * (sqrt(m) + sqrt(n)).
    """
    g = rng(seed)
    m = h * w
    B = np.empty((m, rank))
    f0 = _smooth_field(g, h, w)
    B[:, 0] = (0.4 + 0.2 * f0).ravel(order="F")
    for q in range(1, rank):
        B[:, q] = (0.05 * _smooth_field(g, h, w)).ravel(order="F")
    t = np.arange(n)
    C = np.empty((rank, n))
    gain = g.uniform(0.95, 1.05, size=n)
    C[0] = gain
    for q in range(1, rank):
        period = g.uniform(150.0, 900.0)
        C[q] = gain * np.sin(2 * math.pi * t / period + g.uniform(0, 2 * math.pi))
    # X = background + noise, then paint the foreground squares frame by frame.
    X = np.asfortranarray((B @ C + g.normal(0.0, noise, size=(m, n))).astype(np.float32))
    fg_mask = np.zeros((m, n), dtype=bool, order="F") if keep_parts else None
    pos = np.stack([g.uniform(0, h - rect, size=n_rect), g.uniform(0, w - rect, size=n_rect)], 1)
    ang = g.uniform(0, 2 * math.pi, size=n_rect)
    spd = g.uniform(1.0, 3.0, size=n_rect)
    vel = np.stack([spd * np.sin(ang), spd * np.cos(ang)], 1)
    inten = g.uniform(0.3, 1.0, size=n_rect)
    fnoise = g.normal(0.0, noise, size=(n, n_rect, rect, rect)).astype(np.float32)
    for j in range(n):
        frame = X[:, j].reshape((h, w), order="F")  # view into X
        for q in range(n_rect):
            y0, x0 = int(round(pos[q, 0])), int(round(pos[q, 1]))
            frame[y0:y0 + rect, x0:x0 + rect] = inten[q] + fnoise[j, q]
            if fg_mask is not None:
                fm = fg_mask[:, j].reshape((h, w), order="F")
                fm[y0:y0 + rect, x0:x0 + rect] = True
        pos += vel
        for d, lim in ((0, h - rect), (1, w - rect)):
            lo, hi = pos[:, d] < 0, pos[:, d] > lim
            pos[lo, d] = -pos[lo, d]
            pos[hi, d] = 2 * lim - pos[hi, d]
            vel[lo | hi, d] = -vel[lo | hi, d]
    mask = None
    if mask_p is not None:
        mask = np.asfortranarray((g.random((m, n)) < mask_p).astype(np.uint8))
    if lam_S is None:
        lam_S = 1.0 / math.sqrt(n)
    if lam_L is None:
        lam_L = 4.0 * lam_S * (math.sqrt(m) + math.sqrt(n))
    inst = Instance(X=X, mask=mask, k=k, lam_L=lam_L, lam_S=lam_S, name=f"video{h}x{w}x{n}r{rank}")
    if keep_parts:
        inst.L0 = B @ C
        inst.S0 = np.where(fg_mask, X.astype(np.float64) - inst.L0, 0.0)
    return inst


def factors(m: int, n: int, k: int, seed: int, scale: float = 1.0):
    """Random factors U (m x k), V (n x k), float32 Fortran order, iid N(0, scale^2)."""
    g = rng(seed)
    U = np.asfortranarray(g.normal(0.0, scale, size=(m, k)).astype(np.float32))
    V = np.asfortranarray(g.normal(0.0, scale, size=(n, k)).astype(np.float32))
    return U, V


def gaussian(rows: int, cols: int, seed: int) -> np.ndarray:
    """iid N(0, 1) float32 matrix, Fortran order (a sketching matrix)."""
    return np.asfortranarray(rng(seed).normal(0.0, 1.0, size=(rows, cols)).astype(np.float32))


# Named workloads -------------------------------------------------------------------------

def planted_500x400(seed: int = 0) -> Instance:
    """500 x 400, rank 5, 5% outliers, noise 1e-3, k = 10, lam_S = 1/sqrt(400), lam_L = 1."""
    return planted(500, 400, rank=5, k=10, p_outlier=0.05, noise=1e-3, lam_L=1.0,
                   lam_S=1.0 / math.sqrt(400), seed=seed)


def video_76800x1000(seed: int = 0, **kw) -> Instance:
    """320 x 240 frames, 1000 frames, background rank 3, k = 5, float32, fully observed."""
    return video(h=240, w=320, n=1000, rank=3, k=5, seed=seed, **kw)


def video_110592x2000(seed: int = 0, **kw) -> Instance:
    """384 x 288 frames, 2000 frames, background rank 5, k = 5, 50% Bernoulli mask."""
    return video(h=288, w=384, n=2000, rank=5, k=5, mask_p=0.5, seed=seed, **kw)


def batch_c4(count: int = 256, seed: int = 0, m_range=(1024, 20000), n_range=(50, 600),
             k_range=(2, 16)) -> list:
    """Independent planted instances of varied shape (the batched workload): m ~ U[1024, 20000],
    n ~ U[50, 600], k ~ U{2..16}, planted rank max(1, k // 2), outliers Bernoulli(U[0.02, 0.10])
    with +-U[1, 5], noise 1e-3, fully observed.  lam_S = 1 / sqrt(max(m, n)) and
    lam_L = lam_S (sqrt(m) + sqrt(n)): the first value of the rule "lam_S (sqrt(m) + sqrt(n)),
    doubled until the solution has the planted rank", which these unit-variance planted
    instances already meet (a larger lam_L shrinks L far below the planted part).  Instance i
    is drawn from its own seed (seed * 100003 + i), so any prefix of the batch is reproducible
    alone."""
    g = rng(seed)
    ms = g.integers(m_range[0], m_range[1] + 1, size=count)
    ns = g.integers(n_range[0], n_range[1] + 1, size=count)
    ks = g.integers(k_range[0], k_range[1] + 1, size=count)
    ps = g.uniform(0.02, 0.10, size=count)
    out = []
    for i in range(count):
        m, n, k = int(ms[i]), int(ns[i]), int(ks[i])
        lam_S = 1.0 / math.sqrt(max(m, n))
        inst = planted(m, n, rank=max(1, k // 2), k=k, p_outlier=float(ps[i]), noise=1e-3,
                       lam_L=lam_S * (math.sqrt(m) + math.sqrt(n)), lam_S=lam_S,
                       seed=seed * 100003 + i)
        inst.name = f"c4_{i}_{m}x{n}k{k}"
        out.append(inst)
    return out


def synthetic_sec53(seed: int = 0, m: int = 1000, n: int = 1000, rank: int = 150, p_sparse: float = 0.5,
                    rel_noise: float = 8.12e-5, k: int = 200) -> Instance:
    """The synthetic problem of Sec. 5.3: L = A B^T with A (m x rank), B (n x rank) iid N(0, 1);
    S with N(0, 1) entries on a Bernoulli(p_sparse) set (50 %), zero elsewhere; X = L + S + N with
    white Gaussian N scaled so that ||L + S - X||_F / ||X||_F = rel_noise (8.12e-5); k = 200,
    lam_L = 2.95, lam_S = 0.1."""
    g = rng(seed)
    A = g.normal(size=(m, rank))
    B = g.normal(size=(n, rank))
    L0 = A @ B.T
    S0 = np.where(g.random((m, n)) < p_sparse, g.normal(size=(m, n)), 0.0)
    N = g.normal(size=(m, n))
    Y = L0 + S0
    # ||N_s|| / ||Y + N_s|| = rel  ->  ||N_s|| ~= rel ||Y|| / sqrt(1 - rel^2) (N nearly orthogonal to Y)
    N *= rel_noise * np.linalg.norm(Y) / math.sqrt(1.0 - rel_noise ** 2) / np.linalg.norm(N)
    X = np.asfortranarray((Y + N).astype(np.float32))
    return Instance(X=X, mask=None, k=k, lam_L=2.95, lam_S=0.1, L0=L0, S0=S0, name=f"sec53_{m}x{n}r{rank}")


# ---- Counter-based generator (Philox4x32-10, Salmon et al., SC 2011) -------------------------
# The same stream the library's device generator draws (rpca_gen_planted); used by tests to
# check that generator and by anything that needs an instance's values on the host.

_PH_M0, _PH_M1, _PH_W0, _PH_W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.  ctr: (..., 4) uint32 counters; key: (k0, k1).  Returns the
    (..., 4) uint32 output words.  Rounds: (x, y, z, w) -> (hi(M1 z) ^ y ^ k0, lo(M1 z),
    hi(M0 x) ^ w ^ k1, lo(M0 x)), the key advanced by (W0, W1) before each round but the first."""
    c = np.array(ctr, dtype=np.uint64) & 0xFFFFFFFF
    x, y, z, w = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = np.uint64(key[0] & 0xFFFFFFFF), np.uint64(key[1] & 0xFFFFFFFF)
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(_PH_W0)) & mask
            k1 = (k1 + np.uint64(_PH_W1)) & mask
        p0 = np.uint64(_PH_M0) * x
        p1 = np.uint64(_PH_M1) * z
        x, y, z, w = ((p1 >> np.uint64(32)) ^ y ^ k0, p1 & mask, (p0 >> np.uint64(32)) ^ w ^ k1, p0 & mask)
    return np.stack([x, y, z, w], axis=-1).astype(np.uint32)


def _uniform24(wd):
    return (wd >> np.uint32(8)).astype(np.float64) * 2.0 ** -24


def _normal(wa, wb):
    u1 = ((wa >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * _uniform24(wb))


def planted_philox(m, n, rank, p_outlier, noise, seed, instance):
    """The planted instance rpca_gen_planted writes (float64 values of the same draws): returns
    X, L0, the outlier mask.  Counter layout and transforms as documented in include/rpca.h."""
    k = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    sc = rank ** -0.25
    def factor(rows, which):
        r, c = np.meshgrid(np.arange(rows), np.arange(rank), indexing="ij")
        ctr = np.stack([r, c, np.full_like(r, which), np.full_like(r, instance)], axis=-1)
        wd = philox4x32_10(ctr, k)
        return sc * _normal(wd[..., 0], wd[..., 1])
    A = factor(m, 0)
    B = factor(n, 1)
    L0 = A @ B.T
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    ctr = np.stack([ii, jj, np.full_like(ii, 2), np.full_like(ii, instance)], axis=-1)
    wd = philox4x32_10(ctr, k)
    out = _uniform24(wd[..., 0]) < p_outlier
    mag = 1.0 + 4.0 * (wd[..., 1] & np.uint32(0xFFFFFF)).astype(np.float64) * 2.0 ** -24
    S = np.where(out, np.where(wd[..., 1] >> np.uint32(31), -mag, mag), 0.0)
    N = noise * _normal(wd[..., 2], wd[..., 3])
    return L0 + S + N, L0, out
