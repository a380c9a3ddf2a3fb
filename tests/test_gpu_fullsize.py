"""Parity at the workloads' full sizes, on sampled outputs the oracle can
compute one by one, and properties that hold at any size.

  6x6   M=72 |G|=288 + inversion, 1024 chains x 16 samples (the bench's launch),
        BF16X2 model: sampler, tensor-core log psi, E_loc and its FP64 sums;
  10x10 K=4 M=400 |G|=800, 8192 configurations: log psi, E_loc, O_k;
  8x8   M=128 |G|=512, 4096 samples: one Lanczos step (h1, h2, moments, E_p1).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import annihilated, assert_logpsi_close, make_pair, to_complex

pytestmark = pytest.mark.gpu


def _pick(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False))


def test_6x6_bench_launch_sampled_outputs():
    om, gm, _ = make_pair(6, K=1, M=72, proj=True, spin_inv=1, std=0.01, precision=nnqs.BF16X2)
    cfg, acc = gm.sample(14307, 1024, 16, 10, 100)
    lp = to_complex(gm.log_psi(cfg))
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    e = to_complex(gm.local_energy(cfg, sums=sums))
    gm.status()
    s = synth.unpack(cfg.cpu().numpy().view(np.uint64), 36)
    assert s.shape == (16384, 36) and np.all((s == 1).sum(1) == 18)
    a = acc.cpu().numpy()
    assert np.all((a >= 0) & (a <= 1))
    sm = sums.cpu().numpy()
    assert sm[3] == 16384 and abs(sm[0] - e.real.sum()) <= 1e-12 * np.abs(e.real).sum()
    idx = _pick(16384, 6, 1)
    assert_logpsi_close(lp[idx], om.log_psi(s[idx]), 1e-5)
    want = om.local_energy(s[idx])
    assert np.max(np.abs(e[idx] - want) / (np.abs(want) + 1)) <= 1e-5


def test_10x10_K4_full_batch_sampled_outputs():
    L, N, M, K = 10, 100, 400, 4
    om, gm, p = make_pair(L, K=K, M=M, proj=True, spin_inv=0, std=0.01, precision=nnqs.FP32, logc_std=0.2)
    assert gm.G == 800
    s = synth.random_sz0(N, 8192, seed=21)
    cfg = nnqs.cfg_tensor(synth.pack(s))
    lp = to_complex(gm.log_psi(cfg))
    e = to_complex(gm.local_energy(cfg))
    gm.status()
    idx = _pick(8192, 2, 2)
    idx = idx[~annihilated(L, s[idx], True)]
    assert_logpsi_close(lp[idx], om.log_psi(s[idx]), 1e-5)
    want = om.local_energy(s[idx])
    assert np.max(np.abs(e[idx] - want) / (np.abs(want) + 1)) <= 1e-5
    # O_k of two configurations (the full batch would be 8192 x 162004 complex numbers)
    sub = nnqs.cfg_tensor(synth.pack(s[idx]))
    O = to_complex(gm.grad_logpsi(sub))
    Ow = om.grad_logpsi(s[idx])
    assert O.shape == (len(idx), K * (1 + N + M + M * N))
    assert np.max(np.abs(O - Ow)) <= 1e-5 * max(1.0, np.abs(Ow).max())
    # the tensor-core form (theta' of the rows from the tcgen05 GEMM)
    bm = nnqs.Model(L, 1.0, 0.5, K=K, M=M, proj_t=True, proj_p=True, spin_inv=0, precision=nnqs.BF16X2)
    bm.set_params(p)
    Ob = to_complex(bm.grad_logpsi(sub))
    bm.status()
    assert np.max(np.abs(Ob - Ow)) <= 1e-5 * max(1.0, np.abs(Ow).max())


def test_8x8_lanczos_step_full_batch():
    L, N, M = 8, 64, 128
    om, gm, _ = make_pair(L, K=1, M=M, proj=True, spin_inv=0, std=0.01, precision=nnqs.FP32)
    assert gm.G == 512
    cfg, _ = gm.sample(2206, 512, 8, 10, 100)           # 4096 samples from |psi|^2
    h1, h2, mo, lz = gm.lanczos(cfg)
    gm.status()
    h1, h2 = to_complex(h1), to_complex(h2)
    mo, lz = mo.cpu().numpy(), lz.cpu().numpy()
    # moments and the 2x2 step are those of the returned h1, h2 (any size)
    ref = oracle.moments(h1, h2)
    np.testing.assert_allclose(mo[:4], ref["m"], rtol=1e-12)
    assert mo[4] == 4096
    ref_l = oracle.lanczos_step(mo[:4])
    np.testing.assert_allclose(lz, [ref_l["E"], ref_l["v"], ref_l["alpha"]], rtol=1e-12, atol=1e-14)
    assert lz[0] <= mo[1] + 1e-12                       # variational: E_p1 <= <H>
    # one sampled configuration against the oracle's explicit double enumeration
    s = synth.unpack(cfg.cpu().numpy().view(np.uint64), N)
    k = int(_pick(4096, 1, 3)[0])
    w1, w2 = om.lanczos_h(s[k:k + 1])
    assert abs(h1[k] - w1[0]) <= 1e-5 * (abs(w1[0]) + 1)
    assert abs(h2[k] - w2[0]) <= 1e-4 * (abs(w2[0]) + 1)
