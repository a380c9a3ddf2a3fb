"""The distributed form of the Lanczos step on one GPU: the raw sums of
nnqs_lanczos_partial over disjoint parts of a sample set, added as an
all-reduce would add them, give through nnqs_lanczos_finish the moments and
p = 1 energy of nnqs_lanczos_moments on the whole set (Sec. 3.3)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import make_pair, to_complex

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [nnqs.FP32, nnqs.FP64])
def test_partial_sums_of_parts_give_the_union(prec):
    om, gm, _ = make_pair(6, K=1, M=24, proj=True, spin_inv=1, std=0.05, precision=prec)
    cfg, _ = gm.sample(77, 64, 3, 4, 40)
    n = cfg.shape[0]
    h1, h2, mo, lz = gm.lanczos(cfg)
    parts = [cfg[:50], cfg[50:51], cfg[51:]]
    tot = torch.zeros(7, dtype=torch.float64, device="cuda")
    for c in parts:
        a = torch.empty(c.shape[0], 2, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        _, _, s = gm.lanczos_partial(c, a, b)
        # the sums are those of the part's own h1, h2
        ha, hb = to_complex(a), to_complex(b)
        want = [len(ha), ha.real.sum(), (np.abs(ha) ** 2).sum(), (np.conj(ha) * hb).real.sum(), ha.imag.sum(),
                (np.conj(ha) * hb).imag.sum(), (np.abs(hb) ** 2).sum()]
        np.testing.assert_allclose(s.cpu().numpy(), want, rtol=1e-12, atol=1e-12)
        tot += s
    empty = gm.lanczos_partial(cfg[:0])[2]
    assert np.all(empty.cpu().numpy() == 0)
    mo_d, lz_d = nnqs.lanczos_finish(tot)
    mo, lz, mo_d, lz_d = (x.cpu().numpy() for x in (mo, lz, mo_d, lz_d))
    assert mo_d[4] == n
    np.testing.assert_allclose(mo_d, mo, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(lz_d, lz, rtol=1e-9, atol=1e-12)
    # and both are the closed form of the oracle on the same moments
    ref = oracle.lanczos_step(mo_d[:4])
    np.testing.assert_allclose(lz_d, [ref["E"], ref["v"], ref["alpha"]], rtol=1e-12, atol=1e-14)


def test_lanczos_distributed_single_process_is_lanczos_moments():
    _, gm, _ = make_pair(4, K=1, M=16, proj=True, spin_inv=1, std=0.1, precision=nnqs.FP32)
    cfg, _ = gm.sample(5, 32, 4, 4, 40)
    _, _, mo, lz = gm.lanczos(cfg)
    sums, mo_d, lz_d = nnqs.lanczos_distributed(gm, cfg)
    np.testing.assert_allclose(mo_d.cpu().numpy(), mo.cpu().numpy(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(lz_d.cpu().numpy(), lz.cpu().numpy(), rtol=1e-9, atol=1e-12)
