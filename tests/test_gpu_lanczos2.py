"""The p = 2 Lanczos step on the GPU (Sec. 3.3): h3 = (H^3 psi)/psi against
the oracle's triple enumeration, the moments about c and the 3x3 Krylov step
against the oracle on identical inputs."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import make_pair, to_complex

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,proj,inv,M", [(nnqs.FP32, False, 0, 16), (nnqs.FP32, True, 0, 16),
                                             (nnqs.FP32, True, 1, 8), (nnqs.FP64, True, 1, 8)])
def test_h3_matches_triple_enumeration(prec, proj, inv, M):
    om, gm, _ = make_pair(4, M=M, proj=proj, spin_inv=inv, std=0.05, seed=41, precision=prec)
    s = synth.random_sz0(16, 5, seed=42)
    cfg = nnqs.cfg_tensor(synth.pack(s))
    h3, mu, out = gm.lanczos2(cfg)
    gm.status()
    _, _, w3 = om.lanczos_h3(s)
    got = to_complex(h3)
    tol = 1e-5 if prec == nnqs.FP32 else 1e-10
    assert np.max(np.abs(got - w3) / (np.abs(w3) + 1)) <= tol


@pytest.mark.parametrize("L,M", [(4, 16), (6, 36)])
def test_p2_moments_and_step_on_sampled_configurations(L, M):
    om, gm, _ = make_pair(L, M=M, proj=True, std=0.05, seed=43)
    cfg, _ = gm.sample(4343, 32, 4, 5, 50)
    h3, mu, out = gm.lanczos2(cfg)
    h1, h2, mo, lz = gm.lanczos(cfg)
    gm.status()
    H1, H2, H3 = to_complex(h1), to_complex(h2), to_complex(h3)
    mu_h, out_h = mu.cpu().numpy(), out.cpu().numpy()
    c = mu_h[7]
    assert abs(c - mo.cpu().numpy()[1]) <= 1e-12 * abs(c)         # c = <Re h1>
    want_mu, _ = oracle.shifted_moments(H1, H2, H3, c)
    np.testing.assert_allclose(mu_h[:7], want_mu, rtol=1e-9, atol=1e-12 * abs(want_mu[2]))
    k2 = oracle.krylov2(mu_h[:7], c)                               # identical moments
    assert abs(out_h[0] - k2["E"]) <= 1e-10 * abs(k2["E"])
    np.testing.assert_allclose(out_h[1:4], k2["x"], rtol=1e-6, atol=1e-12)
    assert abs(out_h[4] - k2["var"]) <= 1e-6 * abs(k2["var"]) + 1e-9
    # The leading 2x2 block of the pencil is a p = 1 step with the same
    # (shifted, balanced) estimators; when the sampled 3x3 moment matrix B is
    # positive definite, interlacing puts E_p2 at or below it.  (It differs
    # from the closed-form E_p1 of the raw moments by finite-sample terms:
    # its third central moment uses <Re h2> where the closed form uses
    # <|h1|^2>, two estimators of <H^2>.)
    A = np.array([[mu_h[i + j + 1] for j in range(3)] for i in range(3)])
    B = np.array([[mu_h[i + j] for j in range(3)] for i in range(3)])
    e2 = scipy.linalg.eigh(A[:2, :2], B[:2, :2], eigvals_only=True)[0] + c
    if np.linalg.eigvalsh(B).min() > 1e-12 * np.abs(B).max():
        assert out_h[0] <= e2 + 1e-9 * abs(e2)
    # h3 of a subset against the oracle (4x4 only: the triple enumeration is slow)
    if L == 4:
        s = synth.unpack(cfg.cpu().numpy().view(np.uint64), L * L)[:4]
        _, _, w3 = om.lanczos_h3(s)
        assert np.max(np.abs(H3[:4] - w3) / (np.abs(w3) + 1)) <= 1e-5
