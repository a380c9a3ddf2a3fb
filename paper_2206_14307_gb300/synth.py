"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the method: it only draws parameters and
spin configurations and converts between the two configuration encodings.

Recipe (the paper trains on no dataset; these stand in for its workloads,
Sec. 3.4): complex RBM parameters with independent N(0, std^2) real and
imaginary parts (std 0.01 by default, 0.05 for the "stress" variant), drawn
from numpy's PCG64 stream of the given seed; configurations uniform over the
Sz = 0 sector (a random permutation of N/2 up and N/2 down spins per row).
Mixed batches of instances draw (L, J2, alpha, K) from numpy's Philox stream
of the given seed: L in {4, 6, 8, 10}, J2/J1 uniform in [0, 0.7], alpha in
{1, 2, 4} (M = alpha N), K in {1, 2}.
"""
from __future__ import annotations

import numpy as np


def n_params(N: int, M: int, K: int = 1) -> int:
    """Complex parameters: K blocks of [log c_r, a[N], b[M], W[M][N]]."""
    return K * (1 + N + M + M * N)


def random_params(N: int, M: int, K: int = 1, std: float = 0.01, seed: int = 2206,
                  logc_std: float | None = None) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    P = n_params(N, M, K)
    p = rng.normal(0.0, std, P) + 1j * rng.normal(0.0, std, P)
    if logc_std is not None:
        P1 = P // K
        for r in range(K):
            p[r * P1] = rng.normal(0.0, logc_std) + 1j * rng.normal(0.0, logc_std)
    return p.astype(np.complex128)


def random_sz0(N: int, n: int, seed: int = 307) -> np.ndarray:
    """n uniformly random Sz=0 configurations as int8 spins (+1/-1), [n][N]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.where(np.arange(N) < N // 2, 1, -1).astype(np.int8)
    out = np.empty((n, N), np.int8)
    for k in range(n):
        out[k] = rng.permutation(base)
    return out


def words(N: int) -> int:
    return (N + 63) // 64


def pack(spins: np.ndarray) -> np.ndarray:
    """int8 spins [n][N] -> uint64 words [n][ceil(N/64)], bit i set <=> s_i=+1."""
    s = np.asarray(spins)
    if s.ndim == 1:
        s = s[None]
    n, N = s.shape
    W = words(N)
    out = np.zeros((n, W), np.uint64)
    bits = (s > 0).astype(np.uint64)
    for i in range(N):
        out[:, i // 64] |= bits[:, i] << np.uint64(i % 64)
    return out


def unpack(words_: np.ndarray, N: int) -> np.ndarray:
    w = np.asarray(words_, np.uint64)
    if w.ndim == 1:
        w = w[None]
    out = np.empty((w.shape[0], N), np.int8)
    for i in range(N):
        out[:, i] = np.where((w[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1), 1, -1)
    return out


def mixed_batch(n: int = 64, seed: int = 5) -> list[dict]:
    """n instance shapes of a mixed batch: dicts with L, J2, alpha, K, M."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for _ in range(n):
        L = int(rng.choice([4, 6, 8, 10]))
        J2 = float(rng.uniform(0.0, 0.7))
        alpha = int(rng.choice([1, 2, 4]))
        K = int(rng.choice([1, 2]))
        out.append(dict(L=L, J2=J2, alpha=alpha, K=K, M=alpha * L * L))
    return out
