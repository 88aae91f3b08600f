"""Seeded synthetic point sets for nonrigid registration (model X, scene Y).

This module is the one piece shared by the CUDA path's tests/benchmark and by
the FP64 oracle's tests: it makes inputs and ground truth, and holds none of
the registration method's arithmetic (no posterior, no Gram matrix of X, no
M-step).

Paper context (Fast Coherent Point Drift, Sec. IV): the paper registers 3-D
scans (TOSCA wolf, 4344 points; Stanford bunny resampled to 4000..24000
points) normalised to [-1, 1].  Those datasets are not available here, so the
workloads are synthetic stand-ins with the same sizes and value range:

    GEN(M, N_out, amp, noise, seed)
      X      ~ U[-1, 1]^3                                   (M model points)
      v(x)   = sum_{j<32} a_j exp(-|x - c_j|^2 / (2 * 2^2)),  c_j ~ U[-1,1]^3,
               a_j ~ N(0, I_3), rescaled so sqrt(mean_m |v(x_m)|^2) = amp
      Yhat_m = x_m + v(x_m)          noise-free ground truth, for RMSE (Eq. 22)
      inliers  Yhat_m + N(0, noise^2 I)
      outliers N_out points ~ U(bounding box of the inliers)
      Y      = seeded permutation of [inliers; outliers]

Random numbers come from SplitMix64 used as a counter-based generator
(output i of stream s is mix(s + (i+1) * gamma)), turned into 53-bit uniform
doubles; normals use the Box-Muller transform.  Everything is numpy on the
host; results are bit-identical for a given numpy on a given machine.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 sequence started at `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) with 53 random bits each."""
        z = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller (two per uniform pair)."""
        h = (n + 1) // 2
        u1 = 1.0 - self.uniform(h)          # (0, 1]: log is finite
        u2 = self.uniform(h)
        r = np.sqrt(-2.0 * np.log(u1))
        th = 2.0 * np.pi * u2
        return np.concatenate([r * np.cos(th), r * np.sin(th)])[:n]


@dataclass
class PointSets:
    X: np.ndarray          # (M, 3) model points, float64
    Y: np.ndarray          # (N, 3) scene points, float64
    Yhat: np.ndarray       # (M, 3) noise-free ground-truth position of each x_m
    n_inliers: int
    perm: np.ndarray       # Y[i] came from row perm[i] of [inliers; outliers]


def gen(M: int, n_out: int = 0, amp: float = 0.15, noise: float = 0.01,
        seed: int = 0, centers: int = 32, beta_gen: float = 2.0,
        n_in: int | None = None) -> PointSets:
    """GEN(M, N_out, amp, noise, seed) described in the module docstring.

    `n_in` < M keeps only a seeded random subset of n_in deformed points as
    scene inliers (points missing from the scene side)."""
    if M < 1:
        raise ValueError("M must be >= 1")
    s = Stream(seed)
    X = s.uniform(3 * M).reshape(M, 3) * 2.0 - 1.0
    C = s.uniform(3 * centers).reshape(centers, 3) * 2.0 - 1.0
    A = s.normal(3 * centers).reshape(centers, 3)
    d2 = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    V = np.exp(-d2 / (2.0 * beta_gen * beta_gen)) @ A
    rms = np.sqrt((V * V).sum(1).mean())
    if rms > 0:
        V *= amp / rms
    Yhat = X + V
    noisy = Yhat + noise * s.normal(3 * M).reshape(M, 3)
    if n_in is not None and n_in < M:
        keep = np.sort(np.argsort(s.uniform(M), kind="stable")[:n_in])
        noisy = noisy[keep]
    lo, hi = noisy.min(0), noisy.max(0)
    out = lo + (hi - lo) * s.uniform(3 * n_out).reshape(n_out, 3) if n_out > 0 \
        else np.zeros((0, 3))
    allY = np.concatenate([noisy, out], 0)
    perm = np.argsort(s.uniform(allY.shape[0]), kind="stable")
    return PointSets(X=X, Y=allY[perm].copy(), Yhat=Yhat, n_inliers=noisy.shape[0], perm=perm)


def gen_from_template(X: np.ndarray, seed: int, amp: float = 0.15, noise: float = 0.01, centers: int = 32,
                      beta_gen: float = 2.0) -> PointSets:
    """A new deformation of a fixed model X (same recipe as gen: a random
    Gaussian-RBF displacement of RMS `amp`, noise, seeded permutation); many
    such scenes against one template X are the warm-start training pairs."""
    X = np.asarray(X, dtype=np.float64)
    M = X.shape[0]
    s = Stream(seed)
    C = s.uniform(3 * centers).reshape(centers, 3) * 2.0 - 1.0
    A = s.normal(3 * centers).reshape(centers, 3)
    d2 = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    V = np.exp(-d2 / (2.0 * beta_gen * beta_gen)) @ A
    rms = np.sqrt((V * V).sum(1).mean())
    if rms > 0:
        V *= amp / rms
    Yhat = X + V
    noisy = Yhat + noise * s.normal(3 * M).reshape(M, 3)
    perm = np.argsort(s.uniform(M), kind="stable")
    return PointSets(X=X, Y=noisy[perm].copy(), Yhat=Yhat, n_inliers=M, perm=perm)


def pair_sizes(n_pairs: int, lo: int, hi: int, seed: int) -> list[tuple[int, int]]:
    """(M_i, N_i) for a batch of registrations: both drawn independently and
    uniformly from the integers lo..hi (one SplitMix64 stream)."""
    u = Stream(seed).uniform(2 * n_pairs)
    v = lo + np.floor(u * (hi - lo + 1)).astype(np.int64)
    v = np.minimum(v, hi)
    return [(int(v[2 * i]), int(v[2 * i + 1])) for i in range(n_pairs)]


def gen_pair(M: int, N: int, seed: int, amp: float = 0.15, noise: float = 0.01) -> PointSets:
    """One registration of uneven sizes: with N >= M the scene holds the M
    deformed, noisy model points plus N - M uniform outliers; with N < M it
    holds the deformed, noisy images of a seeded random N-subset of X
    (scene-side missing points)."""
    return gen(M, n_out=max(N - M, 0), amp=amp, noise=noise, seed=seed, n_in=min(M, N))


def gen_batch(n_pairs: int, lo: int, hi: int, seed0: int) -> list[PointSets]:
    """Pairs i < n_pairs with sizes from pair_sizes(n_pairs, lo, hi, seed0)
    and point sets gen_pair(M_i, N_i, seed0 + i)."""
    return [gen_pair(M, N, seed0 + i) for i, (M, N) in enumerate(pair_sizes(n_pairs, lo, hi, seed0))]


# Named workloads (sizes and parameters of the paper-scale runs; Sec. IV).
# omega, lam, beta: outlier weight, regularisation weight, kernel width.
WORKLOADS = {
    # small FP64 case: M = N = 500, full eigenbasis, 50 EM iterations
    "fp64_m500": dict(M=500, n_out=0, amp=0.1, noise=0.01, seed=0,
                      omega=0.1, lam=2.0, beta=2.0, iters=50, K=0),
    # FP32 case: M = N = 5000, full eigenbasis, 100 EM iterations
    "fp32_m5000": dict(M=5000, n_out=0, amp=0.15, noise=0.01, seed=0,
                       omega=0.1, lam=2.0, beta=2.0, iters=100, K=0),
    # M = N = 8000, full eigenbasis: the basis (256 MB) exceeds L2 but the
    # whole case fits a few GB -- the size used for detailed profiler captures
    "fp32_m8000_full": dict(M=8000, n_out=0, amp=0.15, noise=0.01, seed=0,
                            omega=0.1, lam=2.0, beta=2.0, iters=50, K=0),
    # bunny-scale case: M = N = 20000, full eigenbasis (Table IV's largest
    # reported size with both methods)
    "fp32_m20000_full": dict(M=20000, n_out=0, amp=0.15, noise=0.01, seed=0,
                             omega=0.1, lam=2.0, beta=2.0, iters=50, K=0),
    # same, low-rank basis K = 200
    "fp32_m20000_k200": dict(M=20000, n_out=0, amp=0.15, noise=0.01, seed=0,
                             omega=0.1, lam=2.0, beta=2.0, iters=50, K=200),
    # outlier case: M = 20000, N = 25000 (20% extra uniform outliers), K = 200
    "fp32_m20000_n25000_k200": dict(M=20000, n_out=5000, amp=0.15, noise=0.01, seed=0,
                                    omega=0.2, lam=3.0, beta=2.0, iters=150, K=200),
}

# Learned warm start: one template X (gen(M, seed=seed_x).X) and scenes
# gen_from_template(X, seed0 + i); K eigen-coefficients; training pairs
# registered from W = 0 for `iters` iterations.
WARMSTART_WORKLOADS = {
    # the template size and rank of the warm-start configuration (M = N =
    # 2048, K = 64), with a training set of a few thousand scenes
    "fp32_warmstart_m2048_k64": dict(M=2048, K=64, seed_x=7, amp=0.15, noise=0.01, omega=0.1, lam=2.0, beta=2.0,
                                     iters=100, n_train=2048, n_val=64, n_test=32, seed0=100000,
                                     steps=4000, batch=32, lr=3e-4),
    # small version for tests
    "fp32_warmstart_m512_k32": dict(M=512, K=32, seed_x=7, amp=0.15, noise=0.01, omega=0.1, lam=2.0, beta=2.0,
                                    iters=80, n_train=768, n_val=32, n_test=16, seed0=200000,
                                    steps=2000, batch=32, lr=3e-4),
}

# Batches of independent registrations (gen_batch): n_pairs pairs with M_i,
# N_i uniform in lo..hi, pair i seeded seed0 + i, basis K = min(M_i, 128).
BATCH_WORKLOADS = {
    # 256 uneven pairs, sizes 500..8000 (the sizes of the paper's single scans)
    "fp32_batch256_m500_8000_k128": dict(n_pairs=256, lo=500, hi=8000, seed0=1000, K=128,
                                         omega=0.1, lam=2.0, beta=2.0, iters=100),
    # same with sizes 500..3000: a batch whose 256 eigendecompositions take
    # seconds rather than minutes
    "fp32_batch256_m500_3000_k128": dict(n_pairs=256, lo=500, hi=3000, seed0=1000, K=128,
                                         omega=0.1, lam=2.0, beta=2.0, iters=100),
    # 64 pairs, 5 iterations per launch: the small case for profiler captures
    "fp32_batch64_m500_3000_k128": dict(n_pairs=64, lo=500, hi=3000, seed0=1000, K=128,
                                        omega=0.1, lam=2.0, beta=2.0, iters=5),
}
