"""Checked mode of the boundary (desc.check_inputs): every call that takes
configurations rejects one outside the Sz = 0 sector of the sampled method
(N/2 spins up, no bit set past site N - 1) with NNQS_EINVAL before any
compute, naming the first offending index; valid inputs pass unchanged."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import to_complex

pytestmark = pytest.mark.gpu


def _bad_batch(N, n, bad_rows, seed=11):
    s = synth.random_sz0(N, n, seed=seed)
    w = synth.pack(s)
    for k in bad_rows:
        up = np.flatnonzero(s[k] > 0)[0]
        w[k, up // 64] &= ~np.uint64(1 << (up % 64))     # one spin flipped down: N/2 - 1 up
    return s, w


@pytest.mark.parametrize("L,prec", [(4, nnqs.FP32), (6, nnqs.BF16X2), (10, nnqs.FP64)])
def test_every_cfg_call_rejects_non_sz0(L, prec):
    N = L * L
    m = nnqs.Model(L, 1.0, 0.5, K=1, M=N // 2, proj_t=True, proj_p=True, spin_inv=0, precision=prec,
                   check_inputs=True)
    m.set_params(synth.random_params(N, N // 2, 1, std=0.05, seed=1))
    s, w = _bad_batch(N, 9, [5, 7])
    cfg = nnqs.cfg_tensor(w)
    calls = {
        "log_psi": lambda: m.log_psi(cfg),
        "local_energy": lambda: m.local_energy(cfg),
        "lanczos": lambda: m.lanczos(cfg),
        "grad_logpsi": lambda: m.grad_logpsi(cfg[:6]),
        "structure_factor": lambda: m.structure_factor(cfg),
        "noalloc": lambda: nnqs.nnqs_lanczos_moments_noalloc(
            m.h, cfg.data_ptr(), 9, torch.empty(8, dtype=torch.float64, device="cuda").data_ptr(),
            torch.empty(3, dtype=torch.float64, device="cuda").data_ptr(), nnqs._stream()),
        "lanczos2": lambda: m.lanczos2(cfg),
    }
    for name, call in calls.items():
        with pytest.raises(nnqs.NNQSError) as ei:
            call()
        assert ei.value.code == nnqs.NNQS_EINVAL, name
        assert "configuration 5 " in str(ei.value), (name, str(ei.value))
    # the valid rows pass, and give what the unchecked model gives
    good = nnqs.cfg_tensor(synth.pack(s[:5]))
    ref = nnqs.Model(L, 1.0, 0.5, K=1, M=N // 2, proj_t=True, proj_p=True, spin_inv=0, precision=prec)
    ref.set_params(synth.random_params(N, N // 2, 1, std=0.05, seed=1))
    np.testing.assert_array_equal(m.log_psi(good).cpu().numpy(), ref.log_psi(good).cpu().numpy())
    np.testing.assert_array_equal(m.local_energy(good).cpu().numpy(), ref.local_energy(good).cpu().numpy())
    m.status()


def test_stray_bits_past_the_last_site_rejected():
    L, N = 6, 36
    m = nnqs.Model(L, 1.0, 0.5, K=1, M=8, precision=nnqs.FP32, check_inputs=True)
    s = synth.random_sz0(N, 4, seed=2)
    w = synth.pack(s)
    w[2, 0] |= np.uint64(1) << np.uint64(40)                  # site 40 does not exist
    up = np.flatnonzero(s[2] > 0)[0]
    w[2, 0] &= ~np.uint64(1 << up)                           # popcount still N/2
    with pytest.raises(nnqs.NNQSError) as ei:
        m.local_energy(nnqs.cfg_tensor(w))
    assert ei.value.code == nnqs.NNQS_EINVAL and "configuration 2 " in str(ei.value)


def test_unchecked_model_does_not_check():
    # the default mode launches no check (results for such inputs are undefined)
    L, N = 4, 16
    m = nnqs.Model(L, 1.0, 0.5, K=1, M=16, precision=nnqs.FP32)
    _, w = _bad_batch(N, 3, [1])
    m.log_psi(nnqs.cfg_tensor(w))
    torch.cuda.synchronize()


def test_batch_instance_checked():
    specs = [dict(L=4, M=16, proj_t=True, proj_p=True, check_inputs=True),
             dict(L=6, M=36, proj_t=True, proj_p=True, check_inputs=True)]
    b = nnqs.Batch(specs)
    for i, sp in enumerate(specs):
        N = sp["L"] ** 2
        b.models[i].set_params(synth.random_params(N, sp["M"], 1, std=0.05, seed=3 + i))
    _, w0 = _bad_batch(16, 4, [])
    _, w1 = _bad_batch(36, 3, [2])
    cfg = torch.cat([nnqs.cfg_tensor(w0).reshape(-1), nnqs.cfg_tensor(w1).reshape(-1)])
    with pytest.raises(nnqs.NNQSError) as ei:
        b.lanczos(cfg, [4, 3])
    assert ei.value.code == nnqs.NNQS_EINVAL and "instance 1" in str(ei.value)
    b.close()
