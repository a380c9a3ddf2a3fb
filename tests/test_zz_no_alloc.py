"""The allocation-free Lanczos-moments entry point.

nnqs_lanczos_moments_noalloc serves callers that cannot allocate device memory
at the point of the call (a framework pool that owns the whole device budget,
or a loop that must not hit the device-wide synchronisation of growing a
workspace): it keeps h1, h2 and the FP64 partial sums in one fixed-size static
device array of the library.  This test drives it through the C ABI and checks
it against nnqs_lanczos_moments, which allocates its workspace, on two calls in
a row of different sizes (so the second call cannot profit from what the
first left in the shared array), and checks the size limit.  It lives in a
file of its own that is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2206_14307_gb300 import nnqs, synth

pytestmark = pytest.mark.gpu


def _model():
    N, M = 36, 24
    m = nnqs.Model(6, 1.0, 0.5, K=1, M=M, proj_t=True, proj_p=True, spin_inv=1, precision=nnqs.FP32)
    m.set_params(synth.random_params(N, M, 1, std=0.05, seed=4242))
    return m


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    m = _model()
    lib = nnqs.lib()
    st = torch.cuda.current_stream().cuda_stream
    cfg_all, _ = m.sample(99, 64, 4, 5, 40)          # 256 configurations from |psi|^2
    for n in (256, 131):                                # second call smaller than the first
        cfg = cfg_all[:n].contiguous()
        ref_m = torch.zeros(8, dtype=torch.float64, device="cuda")
        ref_l = torch.zeros(3, dtype=torch.float64, device="cuda")
        rc = lib.nnqs_lanczos_moments(m.h, ctypes.c_void_p(cfg.data_ptr()), n, None, None,
                                      ctypes.c_void_p(ref_m.data_ptr()), ctypes.c_void_p(ref_l.data_ptr()),
                                      ctypes.c_void_p(st))
        assert rc == 0, lib.nnqs_last_error()
        got_m = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        got_l = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.nnqs_lanczos_moments_noalloc(m.h, ctypes.c_void_p(cfg.data_ptr()), n,
                                              ctypes.c_void_p(got_m.data_ptr()), ctypes.c_void_p(got_l.data_ptr()),
                                              ctypes.c_void_p(st))
        assert rc == 0, lib.nnqs_last_error()
        torch.cuda.synchronize()
        a, b = got_m.cpu().numpy(), ref_m.cpu().numpy()
        assert a[4] == n and b[4] == n
        np.testing.assert_allclose(a[:4], b[:4], rtol=1e-6)     # the moment tolerance of the parity tests
        np.testing.assert_allclose(got_l.cpu().numpy(), ref_l.cpu().numpy(), rtol=1e-6, atol=1e-12)
    m.status()
    m.close()


def test_noalloc_rejects_more_samples_than_its_scratch():
    m = _model()
    lib = nnqs.lib()
    n = nnqs.NOALLOC_MAX_SAMPLES + 1
    rc = lib.nnqs_lanczos_moments_noalloc(m.h, ctypes.c_void_p(16), n, None, None, None)
    assert rc == nnqs.NNQS_EINVAL
    assert b"exceeds" in lib.nnqs_last_error()
    m.close()
