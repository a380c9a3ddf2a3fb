"""Failure detection without a GPU fault.

* A bounded device-side wait that runs out: a test-only switch makes the
  tensor-core kernel arm its first shared-memory barrier without issuing the
  bulk copy, so the barrier never completes.  The wait gives up after its time
  limit, the kernel records NNQS_ETIMEOUT, frees its tensor memory and returns;
  nnqs_status reports it and the next call runs normally.
* A refused allocation, injected on the host (a workspace cap): NNQS_ENOMEM.
* A non-finite amplitude: E_loc at a configuration whose projected amplitude
  vanishes by symmetry (0/0), and the p = 2 step with a neighbour annihilated
  by a B1 projection: NNQS_ERANGE."""
import os

import numpy as np
import pytest
import torch

from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import annihilated, make_pair, to_complex

pytestmark = pytest.mark.gpu


@pytest.fixture
def env():
    saved = {}

    def set_(k, v):
        saved.setdefault(k, os.environ.get(k))
        os.environ[k] = v

    yield set_
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def test_tensor_core_wait_runs_out_then_recovers(env):
    _, g32, p = make_pair(6, K=1, M=72, proj=True, spin_inv=1, std=0.05, precision=nnqs.FP32)
    _, gtc, _ = make_pair(6, K=1, M=72, proj=True, spin_inv=1, std=0.05, precision=nnqs.BF16X2)
    cfg = nnqs.cfg_tensor(synth.pack(synth.random_sz0(36, 64, seed=9)))
    env("NNQS_TEST_SKIP_TC_COPY", "1")
    gtc.log_psi(cfg)                                  # returns; the kernel gives up on the device
    with pytest.raises(nnqs.NNQSError) as ei:
        gtc.status()
    assert ei.value.code == nnqs.NNQS_ETIMEOUT
    os.environ["NNQS_TEST_SKIP_TC_COPY"] = "0"
    got = to_complex(gtc.log_psi(cfg))                # tensor memory was released: this runs
    gtc.status()
    want = to_complex(g32.log_psi(cfg))
    assert np.max(np.abs(got.real - want.real)) < 1e-5


def test_workspace_refusal_is_enomem(env):
    _, gm, _ = make_pair(4, K=1, M=16, proj=True, spin_inv=0, std=0.05, precision=nnqs.FP32)
    cfg = nnqs.cfg_tensor(synth.pack(synth.random_sz0(16, 8, seed=1)))
    env("NNQS_TEST_WORKSPACE_CAP", "1024")
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(nnqs.NNQSError) as ei:
        gm.local_energy(cfg, sums=sums)
    assert ei.value.code == nnqs.NNQS_ENOMEM and "refused" in str(ei.value)
    os.environ["NNQS_TEST_WORKSPACE_CAP"] = ""
    gm.local_energy(cfg, sums=sums)
    gm.status()
    assert sums[3].item() == 8


def test_annihilated_configuration_is_erange():
    L = 4
    _, gm, _ = make_pair(L, K=1, M=16, proj=True, spin_inv=0, irrep=nnqs.B1, std=0.1, precision=nnqs.FP32)
    s = synth.random_sz0(16, 400, seed=3)
    dead = annihilated(L, s, True, irrep=nnqs.B1)
    assert dead.any()
    k = int(np.flatnonzero(dead)[0])
    gm.local_energy(nnqs.cfg_tensor(synth.pack(s[k:k + 1])))
    with pytest.raises(nnqs.NNQSError) as ei:
        gm.status()
    assert ei.value.code == nnqs.NNQS_ERANGE
    gm.local_energy(nnqs.cfg_tensor(synth.pack(s[~dead][:4])))
    gm.status()                                          # cleared, and live inputs are fine


def _bonds(L):
    out = []
    for i in range(L * L):
        x, y = i % L, i // L
        for dx, dy in ((1, 0), (0, 1), (1, 1), (1, -1)):
            out.append((i, (x + dx) % L + L * ((y + dy) % L)))
    return out


def test_p2_neighbour_annihilated_by_b1_is_erange():
    L = 4
    _, gm, _ = make_pair(L, K=1, M=16, proj=True, spin_inv=0, irrep=nnqs.B1, std=0.1, precision=nnqs.FP32)
    s = synth.random_sz0(16, 400, seed=5)
    live = s[~annihilated(L, s, True, irrep=nnqs.B1)]
    pick = None
    for x in live:
        nbrs = []
        for i, j in _bonds(L):
            if x[i] != x[j]:
                y = x.copy()
                y[i], y[j] = x[j], x[i]
                nbrs.append(y)
        if annihilated(L, np.array(nbrs), True, irrep=nnqs.B1).any():
            pick = x
            break
    assert pick is not None
    gm.lanczos2(nnqs.cfg_tensor(synth.pack(pick[None])))
    with pytest.raises(nnqs.NNQSError) as ei:
        gm.status()
    assert ei.value.code == nnqs.NNQS_ERANGE
