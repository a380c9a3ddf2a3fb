"""Edge cases on the GPU against the oracle: empty inputs, ragged batch tails
of the tensor-core tiles, the maximum sizes (L = 16, i.e. four configuration
words; M = 512; K = 8) and the degenerate Lanczos step (an eigenstate-like
sample set: v = 0, E_p1 = m1, alpha = 0)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import assert_logpsi_close, make_pair, to_complex

pytestmark = pytest.mark.gpu


def _cfg(s):
    return nnqs.cfg_tensor(synth.pack(s))


def test_empty_inputs_are_no_ops_and_bad_sizes_rejected():
    _, gm, _ = make_pair(4, M=16)
    cfg = torch.zeros(1, 1, dtype=torch.int64, device="cuda")
    out = torch.full((4, 2), 7.0, dtype=torch.float64, device="cuda")
    big = torch.full((1, gm.P, 2), 7.0, dtype=torch.float64, device="cuda")
    nnqs.nnqs_log_psi(gm.h, cfg.data_ptr(), 0, out.data_ptr())
    nnqs.nnqs_local_energy(gm.h, cfg.data_ptr(), 0, out.data_ptr(), None)
    nnqs.nnqs_lanczos_moments(gm.h, cfg.data_ptr(), 0, out.data_ptr(), out.data_ptr(), None, None)
    nnqs.nnqs_grad_logpsi(gm.h, cfg.data_ptr(), 0, big.data_ptr())
    torch.cuda.synchronize()
    assert torch.all(out == 7.0) and torch.all(big == 7.0)
    for call in (lambda: nnqs.nnqs_log_psi(gm.h, cfg.data_ptr(), -1, out.data_ptr()),
                 lambda: nnqs.nnqs_lanczos2(gm.h, cfg.data_ptr(), 0, None, None, None),
                 lambda: nnqs.nnqs_structure_factor(gm.h, cfg.data_ptr(), 0, None, out.data_ptr()),
                 lambda: nnqs.nnqs_sample(gm.h, 1, 0, 4, 1, 0, cfg.data_ptr(), None)):
        with pytest.raises(nnqs.NNQSError) as ei:
            call()
        assert ei.value.code == nnqs.NNQS_EINVAL


@pytest.mark.parametrize("n", [1, 3, 129, 1000])
def test_ragged_tensor_core_batches(n):
    om, gtc, p = make_pair(6, M=72, proj=True, spin_inv=1, std=0.05, seed=61, precision=nnqs.BF16X2)
    g32 = nnqs.Model(6, 1.0, 0.5, K=1, M=72, proj_t=True, proj_p=True, spin_inv=1, precision=nnqs.FP32)
    g32.set_params(p)
    s = synth.random_sz0(36, n, seed=62 + n)
    c = _cfg(s)
    a, b = to_complex(gtc.log_psi(c)), to_complex(g32.log_psi(c))
    assert_logpsi_close(a, b, 2e-5)
    k = min(n, 3)
    assert_logpsi_close(a[:k], om.log_psi(s[:k]), 1e-5)


def test_maximum_lattice_L16():
    """N = 256 spins, four uint64 words per configuration, 1024 bonds."""
    L, N, M = 16, 256, 16
    om, gm, _ = make_pair(L, M=M, proj=False, std=0.05, seed=63)
    s = synth.random_sz0(N, 3, seed=64)
    c = _cfg(s)
    assert c.shape == (3, 4)
    assert_logpsi_close(to_complex(gm.log_psi(c)), om.log_psi(s), 1e-5)
    e, w = to_complex(gm.local_energy(c)), om.local_energy(s)
    assert np.max(np.abs(e - w) / (np.abs(w) + 1)) <= 1e-5
    h1, h2, _, _ = gm.lanczos(c[:1])
    w1, w2 = om.lanczos_h(s[:1])
    assert np.max(np.abs(to_complex(h1) - w1) / (np.abs(w1) + 1)) <= 1e-5
    assert np.max(np.abs(to_complex(h2) - w2) / (np.abs(w2) + 1)) <= 1e-5
    # the sampler over four words: Sz = 0, and the oracle's chain step for step
    seed, nc, T = 777, 2, 40
    cfg, _ = gm.sample(seed, nc, T, 1, 0)
    got = synth.unpack(cfg.cpu().numpy().view(np.uint64), N)
    assert np.all((got == 1).sum(1) == N // 2)
    for ch in range(nc):
        prev = oracle.init_config(seed, ch, N)
        for t in range(T):
            cur = got[ch * T + t]
            iu, idn, u = oracle.proposal(seed, ch, t, prev)
            prop = prev.copy()
            prop[iu], prop[idn] = -1, 1
            lr = 2 * (om.log_psi(prop)[0] - om.log_psi(prev)[0]).real
            if abs(np.log(max(u, 1e-300)) - lr) > 1e-4:   # not a borderline draw
                assert np.array_equal(cur, prop if u < np.exp(lr) else prev), (ch, t)
            prev = cur


def test_maximum_width_and_number_of_rbms():
    for L, K, M, proj in ((4, 1, 512, False), (4, 8, 16, True)):
        om, gm, _ = make_pair(L, K=K, M=M, proj=proj, std=0.05, seed=65, logc_std=0.2 if K > 1 else None)
        s = synth.random_sz0(L * L, 4, seed=66)
        c = _cfg(s)
        assert_logpsi_close(to_complex(gm.log_psi(c)), om.log_psi(s), 1e-5)
        e, w = to_complex(gm.local_energy(c)), om.local_energy(s)
        assert np.max(np.abs(e - w) / (np.abs(w) + 1)) <= 1e-5
        h1, h2, _, _ = gm.lanczos(c[:2])
        w1, w2 = om.lanczos_h(s[:2])
        assert np.max(np.abs(to_complex(h2) - w2) / (np.abs(w2) + 1)) <= 1e-5


def test_degenerate_lanczos_step():
    """Real parameters without projection give a real psi and real h1; a single
    sample then has v^2 = m2 - m1^2 = (Im h1)^2 = 0: the step returns E = m1,
    v = 0, alpha = 0 instead of dividing by zero."""
    L, N, M = 4, 16, 16
    p = synth.random_params(N, M, 1, std=0.05, seed=67).real.astype(np.complex128)
    gm = nnqs.Model(L, 1.0, 0.5, K=1, M=M, precision=nnqs.FP64)
    gm.set_params(p)
    c = _cfg(synth.random_sz0(N, 1, seed=68))
    h1, h2, mo, lz = gm.lanczos(c)
    m, l = mo.cpu().numpy(), lz.cpu().numpy()
    assert abs(to_complex(h1)[0].imag) < 1e-12
    assert l[0] == m[1] and l[1] < 1e-6 * abs(m[1]) and l[2] == 0.0
    var = nnqs.lanczos_variance(mo, lz).cpu().numpy()
    assert np.all(np.isfinite(var)) and abs(var[1] - m[1]) < 1e-9 * abs(m[1])
