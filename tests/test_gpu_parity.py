"""GPU (C ABI) vs FP64 oracle on identical seeded inputs.

Tolerances: log psi absolute <= 1e-5 (imaginary part modulo 2 pi) in the
FP32 forms and <= 1e-9 in the FP64 form; E/N and <H^n> relative <= 1e-6;
per-sample E_loc, h1, h2 relative <= 1e-5 (FP32) / 1e-10 (FP64); O_k
absolute <= 1e-5 relative to max |O|.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14307_gb300 import synth
from tests.helpers import annihilated, assert_logpsi_close, fp32_rtol, make_pair, to_complex

pytestmark = pytest.mark.gpu

FP64, FP32, BF16X2, BF16X3 = 0, 1, 2, 3
TOL = {FP64: 1e-9, FP32: 1e-5}


def rtol(prec, std):
    return 1e-10 if prec == FP64 else fp32_rtol(std)


def live_configs(L, n, seed, case):
    """Random Sz=0 configurations, without those annihilated by the projection."""
    _, K, M, proj, inv, bias, mom, irr, std = case
    s = synth.random_sz0(L * L, 4 * n, seed=seed)
    s = s[~annihilated(L, s, proj, mom, irr, inv, bias)]
    return s[:n]


def cfg_of(spins):
    from paper_2206_14307_gb300 import nnqs
    return nnqs.cfg_tensor(synth.pack(spins))


CASES = [
    # (L, K, M, proj, spin_inv, use_bias, momentum, irrep, std)
    (4, 1, 16, False, 0, True, 0, 0, 0.01),
    (4, 1, 16, False, 0, True, 0, 0, 0.3),
    (4, 2, 12, True, 1, True, 1, 2, 0.2),
    (4, 1, 40, True, -1, True, 2, 0, 0.1),
    (6, 1, 72, True, 1, True, 0, 0, 0.01),
    (6, 1, 72, True, 1, True, 0, 0, 0.05),
    (6, 2, 20, True, 0, False, 3, 3, 0.1),
]


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", CASES)
def test_log_psi(case, prec):
    L, K, M, proj, inv, bias, mom, irr, std = case
    om, gm, _ = make_pair(L, K=K, M=M, proj=proj, spin_inv=inv, use_bias=bias, momentum=mom, irrep=irr,
                          std=std, precision=prec, logc_std=0.2 if K > 1 else None)
    s = live_configs(L, 70, 1, case)   # 70 samples: several CTAs and a ragged tail
    got = to_complex(gm.log_psi(cfg_of(s)))
    torch.cuda.synchronize()
    want = om.log_psi(s)
    assert_logpsi_close(got, want, TOL[prec])
    gm.status()


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", CASES)
def test_local_energy(case, prec):
    L, K, M, proj, inv, bias, mom, irr, std = case
    om, gm, _ = make_pair(L, K=K, M=M, proj=proj, spin_inv=inv, use_bias=bias, momentum=mom, irrep=irr,
                          std=std, precision=prec, logc_std=0.2 if K > 1 else None)
    n = 40 if L == 4 else 6
    s = live_configs(L, n, 2, case)
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    got = to_complex(gm.local_energy(cfg_of(s), sums=sums))
    want = om.local_energy(s)
    fin = np.isfinite(want)
    scale = np.abs(want[fin]) + 1.0
    assert np.max(np.abs(got[fin] - want[fin]) / scale) <= rtol(prec, std)
    sm = sums.cpu().numpy()
    # the FP64 sums are those of the returned per-sample values
    assert abs(sm[0] - got.real.sum()) <= 1e-12 * np.abs(got.real).sum()
    assert abs(sm[2] - (np.abs(got) ** 2).sum()) <= 1e-12 * (np.abs(got) ** 2).sum()
    assert sm[3] == n
    gm.status()


def test_local_energy_mean_energy_per_site_rel_1e6():
    # E/N over a 6x6 projected batch, FP32 form vs the FP64 oracle.
    om, gm, _ = make_pair(6, K=1, M=72, proj=True, spin_inv=1, std=0.05, precision=FP32)
    s = synth.random_sz0(36, 24, seed=3)
    got = to_complex(gm.local_energy(cfg_of(s)))
    want = om.local_energy(s)
    e_got, e_want = got.real.mean() / 36, want.real.mean() / 36
    assert abs(e_got - e_want) <= 1e-6 * abs(e_want)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[3]])
def test_lanczos_h1_h2_random_configs(case, prec):
    L, K, M, proj, inv, bias, mom, irr, std = case
    om, gm, _ = make_pair(L, K=K, M=M, proj=proj, spin_inv=inv, use_bias=bias, momentum=mom, irrep=irr,
                          std=std, precision=prec, logc_std=0.2 if K > 1 else None)
    s = live_configs(L, 12, 4, case)
    h1, h2, mo, lz = gm.lanczos(cfg_of(s))
    h1, h2 = to_complex(h1), to_complex(h2)
    w1, w2 = om.lanczos_h(s)
    assert np.max(np.abs(h1 - w1) / (np.abs(w1) + 1)) <= rtol(prec, std)
    assert np.max(np.abs(h2 - w2) / (np.abs(w2) + 1)) <= rtol(prec, std) * 10
    # the p = 1 step is the closed form of the moments the GPU returned
    mo = mo.cpu().numpy()
    ref_l = oracle.lanczos_step(mo[:4])
    lz = lz.cpu().numpy()
    np.testing.assert_allclose(lz, [ref_l["E"], ref_l["v"], ref_l["alpha"]], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("prec,L,K,M,proj,inv,std", [
    (FP32, 4, 1, 16, False, 0, 0.05), (FP32, 4, 2, 12, True, 1, 0.05), (FP32, 6, 1, 24, True, 1, 0.05),
    (FP64, 4, 1, 16, False, 0, 0.3), (FP64, 4, 2, 12, True, 1, 0.2), (FP64, 6, 1, 24, True, 1, 0.05)])
def test_lanczos_moments_on_sampled_configs(prec, L, K, M, proj, inv, std):
    # <H^n>, n <= 3, over configurations drawn from |psi|^2 by the GPU
    # sampler: relative error <= 1e-6 against the oracle on the same samples
    # (FP32 at the workloads' weight scales; FP64 also at the 0.3 stress scale,
    # where FP32 ratios near zeros of cosh(theta) lose about 1e-5).
    om, gm, _ = make_pair(L, K=K, M=M, proj=proj, spin_inv=inv, std=std, precision=prec,
                          logc_std=0.2 if K > 1 else None)
    n_chains, n_per = (64, 2) if L == 4 else (8, 1)
    cfg, _ = gm.sample(31, n_chains, n_per, 5, 50)
    s = synth.unpack(cfg.cpu().numpy().view(np.uint64), L * L)
    h1, h2, mo, lz = gm.lanczos(cfg)
    w1, w2 = om.lanczos_h(s)
    ref = oracle.moments(w1, w2)
    mo = mo.cpu().numpy()
    np.testing.assert_allclose(mo[:4], ref["m"], rtol=1e-6 if prec == FP32 else 1e-10)
    assert mo[4] == len(s)
    ref_l = oracle.lanczos_step(ref["m"])
    # E_p1 carries the moment errors through d = (m3 - 3 m1 m2 + 2 m1^3)/(2 v^3):
    # bound = sum_k |dE/dm_k| |m_k| * (moment tolerance), derivatives by central
    # differences of the closed form
    mtol = 1e-6 if prec == FP32 else 1e-10
    bound = 0.0
    for k in (1, 2, 3):
        h = 1e-6 * abs(ref["m"][k])
        up, dn = ref["m"].copy(), ref["m"].copy()
        up[k] += h
        dn[k] -= h
        dE = (oracle.lanczos_step(up)["E"] - oracle.lanczos_step(dn)["E"]) / (2 * h)
        bound += abs(dE) * abs(ref["m"][k]) * mtol
    assert abs(lz.cpu().numpy()[0] - ref_l["E"]) <= 2 * bound + 1e-12


def test_lanczos_6x6_projected_two_samples():
    om, gm, _ = make_pair(6, K=1, M=72, proj=True, spin_inv=1, std=0.05, precision=FP32)
    s = synth.random_sz0(36, 2, seed=5)
    h1, h2, _, _ = gm.lanczos(cfg_of(s))
    w1, w2 = om.lanczos_h(s)
    np.testing.assert_allclose(to_complex(h1), w1, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(to_complex(h2), w2, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("prec", [FP32, FP64, BF16X2, BF16X3])
@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[3], CASES[6]])
def test_grad_logpsi(case, prec):
    # BF16X2 / BF16X3: theta' from the tcgen05 GEMM, read by the gradient
    # kernel; with two bf16 terms per weight (2^-17 relative each) O carries
    # ~1e-5 relative error at weight scales >= 0.1, with three FP32 accuracy
    L, K, M, proj, inv, bias, mom, irr, std = case
    om, gm, _ = make_pair(L, K=K, M=M, proj=proj, spin_inv=inv, use_bias=bias, momentum=mom, irrep=irr,
                          std=std, precision=prec, logc_std=0.2 if K > 1 else None)
    s = live_configs(L, 5, 6, case)
    got = to_complex(gm.grad_logpsi(cfg_of(s)))
    want = om.grad_logpsi(s)
    scale = np.abs(want).max()
    tol = 1e-10 if prec == FP64 else 5e-5 if (prec == BF16X2 and std > 0.05) else 1e-5
    assert np.max(np.abs(got - want)) <= tol * max(scale, 1.0)


def test_energy_grad_and_sr_matvec_fp64():
    om, gm, _ = make_pair(4, K=1, M=6, proj=True, spin_inv=1, std=0.2, precision=FP64)
    s = synth.random_sz0(16, 30, seed=7)
    cfg = cfg_of(s)
    O = gm.grad_logpsi(cfg)
    e = gm.local_energy(cfg)
    F = to_complex(gm.energy_grad(O, e))
    Oc, ec = to_complex(O), to_complex(e)
    Fref = oracle.energy_grad(Oc, ec)
    np.testing.assert_allclose(F, Fref, rtol=1e-9, atol=1e-12)
    lam, dtau = 1e-3, 0.1
    d = oracle.sr_solve(Oc, Fref, lam, dtau)
    x = torch.from_numpy(np.stack([d.real, d.imag], -1)).cuda()
    y = to_complex(gm.sr_matvec(O, x, lam))
    np.testing.assert_allclose(y, -dtau * Fref, rtol=1e-7, atol=1e-10)


def test_fp32_matches_fp64_form():
    _, g32, p = make_pair(6, K=1, M=72, proj=True, spin_inv=1, std=0.05, precision=FP32)
    _, g64, _ = make_pair(6, K=1, M=72, proj=True, spin_inv=1, std=0.05, precision=FP64)
    s = synth.random_sz0(36, 300, seed=8)
    c = cfg_of(s)
    assert_logpsi_close(to_complex(g32.log_psi(c)), to_complex(g64.log_psi(c)), 1e-5)
