"""Form (3): hand-written O_k / energy-gradient kernels behind
torch.autograd, and the FP64 conjugate-gradient SR solve (Eq. 12).

* GPU gradients with exact weights |psi|^2 over the whole 4x4 Sz=0 sector
  equal central finite differences of the exact energy (oracle amplitudes,
  Kronecker-product H) within 1e-5.
* The CG solve equals the oracle's dense solve of the same system.
* autograd's backward equals nnqs_energy_grad; an exact-weight SR step lowers
  the exact energy.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from paper_2206_14307_gb300 import nnqs, synth
from paper_2206_14307_gb300.autograd import VMCEnergy, sr_step
from tests.helpers import make_pair, to_complex
from tests.kron_h import hamiltonian_full, sz0_restrict

pytestmark = pytest.mark.gpu
L, N, M = 4, 16, 4


@functools.lru_cache(maxsize=None)
def _H():
    return sz0_restrict(hamiltonian_full(L, 1.0, 0.5), N)[0]


def _exact_energy(om, params, s_all):
    lp = om.with_params(params).log_psi(s_all)
    psi = np.exp(lp - lp.real.max())
    H = _H()
    return (np.vdot(psi, H @ psi) / np.vdot(psi, psi)).real


def _all_states():
    st = oracle.sz0_basis(N)
    return oracle.states_to_spins(st, N)


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_gradient_matches_fd_of_exact_energy(prec):
    om, gm, p = make_pair(L, M=M, proj=True, spin_inv=1, std=0.2, seed=52, precision=prec)
    s = _all_states()
    cfg = nnqs.cfg_tensor(synth.pack(s))
    lp = to_complex(gm.log_psi(cfg))
    w = np.exp(2 * (lp.real - lp.real.max()))
    keep = w > 1e-20 * w.max()
    cfg_k = nnqs.cfg_tensor(synth.pack(s[keep]))
    wt = torch.from_numpy(w[keep]).cuda()
    O = gm.grad_logpsi(cfg_k)
    e = gm.local_energy(cfg_k)
    F = to_complex(gm.energy_grad(O, e, weights=wt))
    gm.status()
    h = 1e-5
    for q in np.random.default_rng(3).choice(gm.P, 8, replace=False):
        for unit, part in ((1.0, lambda z: 2 * z.real), (1j, lambda z: 2 * z.imag)):
            dp = np.zeros(gm.P, complex)
            dp[q] = unit * h
            fd = (_exact_energy(om, p + dp, s) - _exact_energy(om, p - dp, s)) / (2 * h)
            assert abs(part(F[q]) - fd) <= 1e-5 * max(1.0, abs(fd)), (q, unit, part(F[q]), fd)


def test_sr_solve_equals_dense_oracle_solve():
    om, gm, _ = make_pair(L, M=M, proj=True, spin_inv=1, std=0.2, seed=53, precision=0)
    s = synth.random_sz0(N, 60, seed=7)
    cfg = nnqs.cfg_tensor(synth.pack(s))
    O = gm.grad_logpsi(cfg)
    e = gm.local_energy(cfg)
    F = gm.energy_grad(O, e)
    lam, dtau = 1e-3, 0.05
    delta, info = gm.sr_solve(O, F, lam=lam, dtau=dtau, max_iter=400, tol=1e-13)
    gm.status()
    ref = oracle.sr_solve(to_complex(O), to_complex(F), lam, dtau)
    np.testing.assert_allclose(to_complex(delta), ref, rtol=1e-7, atol=1e-12 * np.abs(ref).max())
    it, res = info.cpu().numpy()
    assert 0 < it <= 400 and res <= 1e-12
    # (S + lam) delta = -dtau F through the matrix-free product
    y = to_complex(gm.sr_matvec(O, delta, lam))
    np.testing.assert_allclose(y, -dtau * to_complex(F), rtol=1e-8, atol=1e-12)


def test_autograd_backward_equals_energy_gradient():
    _, gm, p = make_pair(L, M=M, proj=True, spin_inv=1, std=0.2, seed=54, precision=1)
    cfg, _ = gm.sample(5, 64, 8, 4, 40)
    params = torch.from_numpy(np.stack([p.real, p.imag], -1)).cuda().requires_grad_(True)
    E = VMCEnergy.apply(params, gm, cfg)
    E.backward()
    O = gm.grad_logpsi(cfg)
    e = gm.local_energy(cfg)
    F = gm.energy_grad(O, e)
    torch.testing.assert_close(params.grad, 2.0 * F, rtol=1e-12, atol=1e-14)
    assert abs(E.item() - e[:, 0].mean().item()) <= 1e-12 * abs(E.item())


def test_exact_weight_sr_step_lowers_the_exact_energy():
    om, gm, p = make_pair(L, M=M, proj=True, spin_inv=1, std=0.2, seed=55, precision=0)
    s = _all_states()
    params = torch.from_numpy(np.stack([p.real, p.imag], -1)).cuda()
    e0 = _exact_energy(om, p, s)
    cfg = nnqs.cfg_tensor(synth.pack(s))
    lp = to_complex(gm.log_psi(cfg))
    w = np.exp(2 * (lp.real - lp.real.max()))
    keep = w > 1e-20 * w.max()
    cfg_k = nnqs.cfg_tensor(synth.pack(s[keep]))
    wt = torch.from_numpy(w[keep]).cuda()
    delta, info = sr_step(gm, params, cfg_k, lam=1e-4, dtau=0.02, max_iter=300, tol=1e-12, weights=wt)
    p1 = params[:, 0].cpu().numpy() + 1j * params[:, 1].cpu().numpy()
    e1 = _exact_energy(om, p1, s)
    assert e1 < e0
