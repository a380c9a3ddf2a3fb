"""Fourth moment, p = 1 variance / variance extrapolation (Sec. 3.3 Eq. 16,
Sec. 4.3) and the static spin structure factor (Sec. 4.1) on the GPU against
the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import make_pair, to_complex

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,M,proj,inv", [(4, 16, False, 0), (4, 32, True, 1), (6, 36, True, 0)])
def test_fourth_moment_and_variance(L, M, proj, inv):
    om, gm, _ = make_pair(L, M=M, proj=proj, spin_inv=inv, std=0.05, seed=31)
    cfg, _ = gm.sample(777, 32, 4, 5, 50)
    h1, h2, mo, lz = gm.lanczos(cfg)
    gm.status()
    H1, H2 = to_complex(h1), to_complex(h2)
    mo_h = mo.cpu().numpy()
    # the kernel's m4 is the mean of |h2|^2 of its own h2
    assert abs(mo_h[7] - np.mean(np.abs(H2) ** 2)) <= 1e-12 * mo_h[7]
    # against the oracle's h2 on the same configurations
    s = synth.unpack(cfg.cpu().numpy().view(np.uint64), L * L)
    sel = slice(0, 16 if L == 4 else 4)
    w1, w2 = om.lanczos_h(s[sel])
    ref = oracle.moments(w1, w2)
    got = oracle.moments(H1[sel], H2[sel])
    assert abs(got["m4"] - ref["m4"]) <= 5e-5 * ref["m4"]
    # device variance step == oracle formula on the same moments
    var = nnqs.lanczos_variance(mo, lz).cpu().numpy()
    m5 = np.concatenate([mo_h[:4], [mo_h[7]]])
    want = oracle.lanczos_variance(m5, lz.cpu().numpy())
    E1 = want["E1"]
    np.testing.assert_allclose(var[0], want["var0"], rtol=1e-10, atol=1e-12 * mo_h[2])
    np.testing.assert_allclose(var[1], E1, rtol=1e-12)
    np.testing.assert_allclose(var[2], want["var1"], rtol=1e-6, atol=1e-11 * E1 * E1)
    np.testing.assert_allclose(var[3], want["E_extrap"], rtol=1e-6, atol=1e-10 * abs(E1))
    assert abs(var[1] - lz.cpu().numpy()[0]) <= 1e-9 * abs(E1)   # E1 is the closed-form E_p1


@pytest.mark.parametrize("L", [4, 6, 10])
def test_structure_factor_matches_oracle(L):
    N = L * L
    om, gm, _ = make_pair(L, M=N, proj=L < 10, std=0.05, seed=32)
    cfg, _ = gm.sample(888, 64, 4, 5, 50)
    n = cfg.shape[0]
    sq = gm.structure_factor(cfg).cpu().numpy()
    s = synth.unpack(cfg.cpu().numpy().view(np.uint64), N)
    # all samples: numpy's 2D FFT power spectrum; a subset: the oracle's double sum
    f = np.fft.fft2(s.reshape(n, L, L) / 2.0)
    np.testing.assert_allclose(sq, ((np.abs(f) ** 2).mean(0) / N ** 2).reshape(-1), rtol=1e-12, atol=1e-16)
    k = 24 if L == 10 else n
    sub = gm.structure_factor(cfg[:k]).cpu().numpy()
    np.testing.assert_allclose(sub, oracle.structure_factor(L, s[:k]), rtol=1e-12, atol=1e-16)
    assert abs(sq.sum() - 0.25) < 1e-12 and abs(sq[0]) < 1e-15
    # weighted mean
    w = np.linspace(0.5, 2.0, k)
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    sw = gm.structure_factor(cfg[:k], weights=wt).cpu().numpy()
    np.testing.assert_allclose(sw, oracle.structure_factor(L, s[:k], w), rtol=1e-12, atol=1e-16)
