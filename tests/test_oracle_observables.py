"""Oracle pins for the static spin structure factor (Sec. 4.1):
S(q) = (1/N^2) sum_ij <sz_i sz_j> e^{i q.(r_i - r_j)}, sz = s/2."""
import numpy as np

import oracle
from paper_2206_14307_gb300 import synth


def test_structure_factor_equals_fft_power_spectrum():
    # per configuration S(q) = |sum_j sz_j e^{-i q.r_j}|^2 / N^2: numpy's 2D FFT
    for L in (4, 6):
        N = L * L
        s = synth.random_sz0(N, 5, seed=L)
        got = oracle.structure_factor(L, s)
        grid = s.reshape(5, L, L) / 2.0          # [k][y][x]
        f = np.fft.fft2(grid)                     # axes (y, x): f[k, qy, qx]
        want = (np.abs(f) ** 2).mean(0) / N ** 2
        np.testing.assert_allclose(got, want.reshape(-1), rtol=1e-12, atol=1e-15)


def test_structure_factor_sum_rule_zero_mode_and_neel():
    L, N = 6, 36
    s = synth.random_sz0(N, 7, seed=3)
    w = np.arange(1, 8, dtype=float)
    sq = oracle.structure_factor(L, s, w)
    assert abs(sq.sum() - 0.25) < 1e-13          # sum_q S(q) = <sz_i^2> = 1/4
    assert abs(sq[0]) < 1e-15                    # Sz = 0: no uniform component
    neel = np.array([1 if (i % L + i // L) % 2 == 0 else -1 for i in range(N)], np.int8)
    sn = oracle.structure_factor(L, neel[None])
    qpp = L // 2 + L * (L // 2)
    assert abs(sn[qpp] - 0.25) < 1e-14 and abs(np.delete(sn, qpp)).max() < 1e-14
    # weights: the weighted mean of single-configuration values
    each = np.array([oracle.structure_factor(L, x[None]) for x in s])
    np.testing.assert_allclose(sq, (w[:, None] * each).sum(0) / w.sum(), rtol=1e-12, atol=1e-16)
