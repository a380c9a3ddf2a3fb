"""The FP32 sampler with each chain's cache in shared memory: one CTA per SM,
the chain's rows (r, g) split over the CTAs of a thread-block cluster when
they do not fit one CTA, the partial sums exchanged through distributed shared
memory.  Proposals are Philox-exact and accept decisions equal the FP64
oracle's except at near-ties, for the cluster sizes the models select (1 at
4x4 and at the 6x6 workload, 8 at 8x8 M = 128) and for forced sizes (test hook
NNQS_TEST_SAMPLER_CLUSTER), including CTAs that own no row, and with
parameters large enough that some cache entries exceed 2^12 in modulus (the
rows' products are then renormalised after every unit pair)."""
import os

import numpy as np
import pytest

import oracle
from paper_2206_14307_gb300 import synth
from tests.helpers import make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture
def cluster_env():
    old = os.environ.get("NNQS_TEST_SAMPLER_CLUSTER")
    yield lambda v: os.environ.__setitem__("NNQS_TEST_SAMPLER_CLUSTER", v)
    if old is None:
        os.environ.pop("NNQS_TEST_SAMPLER_CLUSTER", None)
    else:
        os.environ["NNQS_TEST_SAMPLER_CLUSTER"] = old


def replay(om, gm, N, seed, nc, T):
    cfg, acc = gm.sample(seed, nc, T, 1, 0)
    gm.status()
    s = synth.unpack(cfg.cpu().numpy().view(np.uint64), N)
    near = 0
    for c in range(nc):
        prev = oracle.init_config(seed, c, N)
        for t in range(T):
            cur = s[c * T + t]
            iu, idn, u = oracle.proposal(seed, c, t, prev)
            prop = prev.copy()
            prop[iu], prop[idn] = -1, 1
            lr = 2 * (om.log_psi(prop)[0] - om.log_psi(prev)[0]).real
            want = u < np.exp(lr)
            got = np.array_equal(cur, prop)
            assert got or np.array_equal(cur, prev), "state is neither the proposal nor the old state"
            if got != want:
                assert abs(np.log(max(u, 1e-300)) - lr) < 1e-4, (c, t)
                near += 1
            prev = cur
    a = acc.cpu().numpy()
    assert np.all((a >= 0) & (a <= 1))
    return near


@pytest.mark.parametrize("L,M,proj,inv,std,force,nc,T", [
    (6, 72, True, 1, 0.05, "", 3, 80),      # the 6x6 workload shape: one CTA
    (8, 128, True, 0, 0.05, "", 1, 30),     # 8x8, M = 128: cluster of 8
    (4, 8, False, 0, 0.3, "4", 3, 150),     # one row over a cluster of 4: three CTAs own none
    (4, 6, True, 1, 0.3, "8", 3, 150),      # 128 rows over a cluster of 8
    (6, 12, True, -1, 0.3, "2", 3, 150),
    (4, 8, True, 1, 1.0, "", 3, 120),       # |c| beyond 2^12: rows renormalised after every unit pair
])
def test_cluster_sampler_replays_oracle(cluster_env, L, M, proj, inv, std, force, nc, T):
    cluster_env(force)
    om, gm, _ = make_pair(L, M=M, proj=proj, spin_inv=inv, std=std, precision=1)
    assert replay(om, gm, L * L, 12345, nc, T) <= 1


def test_cluster_sampler_matches_global_cache_sampler(cluster_env):
    """Both FP32 samplers on the 6x6 workload shape: the same chains (they
    compute the same ratios; only the order of the final sums differs)."""
    om, gm, _ = make_pair(6, M=72, proj=True, spin_inv=1, std=0.01, precision=1)
    cluster_env("")
    a, acc_a = gm.sample(2206, 64, 8, 10, 100)
    cluster_env("old")
    b, acc_b = gm.sample(2206, 64, 8, 10, 100)
    gm.status()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    same_chain = [(a[c * 8:(c + 1) * 8] == b[c * 8:(c + 1) * 8]).all() for c in range(64)]
    assert np.mean(same_chain) >= 0.95
    assert abs(acc_a.mean().item() - acc_b.mean().item()) < 0.01
