"""GPU Metropolis sampler vs the oracle: Philox proposals bit-exact, accept
decisions equal to the FP64 decisions except at near-ties, and the chain
statistics of |psi|^2."""
import numpy as np
import pytest
import scipy.stats
import torch

import oracle
from paper_2206_14307_gb300 import synth
from tests.helpers import make_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,M,proj,inv,prec", [(4, 8, False, 0, 1), (4, 6, True, 1, 1), (6, 12, True, -1, 1),
                                               (4, 8, False, 0, 0)])
def test_sampler_replays_oracle_proposals(L, M, proj, inv, prec):
    N = L * L
    om, gm, _ = make_pair(L, M=M, proj=proj, spin_inv=inv, std=0.3, precision=prec)
    seed, nc, T = 12345, 3, 150
    cfg, acc = gm.sample(seed, nc, T, 1, 0)
    s = synth.unpack(cfg.cpu().numpy().view(np.uint64), N)
    near = 0
    for c in range(nc):
        prev = oracle.init_config(seed, c, N)
        for t in range(T):
            cur = s[c * T + t]
            iu, idn, u = oracle.proposal(seed, c, t, prev)
            prop = prev.copy(); prop[iu], prop[idn] = -1, 1
            lr = 2 * (om.log_psi(prop)[0] - om.log_psi(prev)[0]).real
            want_acc = u < np.exp(lr)
            got_acc = np.array_equal(cur, prop)
            assert got_acc or np.array_equal(cur, prev), "state is neither the proposal nor the old state"
            if got_acc != want_acc:
                assert abs(np.log(max(u, 1e-300)) - lr) < 1e-4, (c, t)
                near += 1
            prev = cur
    assert near <= 1
    a = acc.cpu().numpy()
    assert np.all((a >= 0) & (a <= 1))


def test_sampler_distribution_4x4():
    N = 16
    om, gm, _ = make_pair(4, M=4, std=0.35, seed=61)
    st = oracle.sz0_basis(N)
    lp = om.log_psi(oracle.states_to_spins(st, N))
    prob = np.exp(2 * (lp.real - lp.real.max())); prob /= prob.sum()
    order = np.argsort(prob)
    cum = np.cumsum(prob[order])
    nb = 16
    bin_of = np.empty(st.size, int)
    bin_of[order] = np.minimum((cum * nb).astype(int), nb - 1)
    pbin = np.bincount(bin_of, weights=prob, minlength=nb)
    n_chains = 20000
    cfg, _ = gm.sample(99, n_chains, 1, 1, 200)
    code = cfg.cpu().numpy().view(np.uint64)[:, 0]
    pos = np.searchsorted(st, code)
    assert np.all(st[pos] == code)
    counts = np.bincount(bin_of[pos], minlength=nb)
    used = pbin > 0          # a state heavier than 1/nb can leave a bin empty
    chi2 = ((counts[used] - n_chains * pbin[used]) ** 2 / (n_chains * pbin[used])).sum()
    assert counts[~used].sum() == 0
    assert scipy.stats.chi2.sf(chi2, used.sum() - 1) > 1e-4


def test_sampler_outputs_sz0_and_is_deterministic():
    om, gm, _ = make_pair(6, M=72, proj=True, spin_inv=1, std=0.05)
    a, acc1 = gm.sample(7, 64, 4, 5, 20)
    b, acc2 = gm.sample(7, 64, 4, 5, 20)
    assert torch.equal(a, b) and torch.equal(acc1, acc2)
    s = synth.unpack(a.cpu().numpy().view(np.uint64), 36)
    assert np.all((s == 1).sum(1) == 18)
