"""SR training on the GPU (Sec. 3.2 Eq. 12; Sec. 3.4): a fully projected
complex RBM on the 4x4 Heisenberg lattice reaches the exact ground-state
energy (the oracle's ED), checked by exact enumeration of the trained
state's energy; the psi_s -> psi_KL warm start."""
import numpy as np
import pytest

import oracle
from paper_2206_14307_gb300 import nnqs, synth, train

pytestmark = pytest.mark.gpu

L, N, M = 4, 16, 16


def exact_energy(params, J2, proj_p=True):
    om = oracle.Model(L, 1.0, J2, K=1, M=M, proj_t=True, proj_p=proj_p, params=params)
    s = oracle.states_to_spins(oracle.sz0_basis(N), N)
    lp = om.log_psi(s)
    w = np.exp(2 * (lp.real - lp.real.max()))
    keep = w > 1e-14 * w.max()
    return float((w[keep] * om.local_energy(s[keep]).real).sum() / w[keep].sum()) / N


def test_sr_reaches_ed_on_4x4_heisenberg():
    E0 = oracle.ed_ground(L, 1.0, 0.0)[0] / N
    m = nnqs.Model(L, 1.0, 0.0, K=1, M=M, proj_t=True, proj_p=True, use_bias=True, precision=nnqs.FP32)
    tr = train.SRTrainer(m, synth.random_params(N, M, 1, std=0.01, seed=2206), n_chains=256, n_per_chain=8,
                         lr=0.05, seed=5)
    tr.run(150)
    h = tr.history
    assert h[0]["E"] / N > -0.1 and h[-1]["E"] / N < -0.69        # sampled energy falls
    assert all(1 <= x["n_skip"] <= 100 for x in h) and len({x["n_skip"] for x in h}) > 1
    Ex = exact_energy(tr.host_params(), 0.0)
    assert E0 <= Ex + 1e-12
    assert abs(Ex - E0) / abs(E0) < 1e-3


def test_warm_start_from_translation_only_wave_function():
    J2 = 0.0
    ms = nnqs.Model(L, 1.0, J2, K=1, M=M, proj_t=True, proj_p=False, use_bias=True, precision=nnqs.FP32)
    p0 = synth.random_params(N, M, 1, std=0.01, seed=2206)
    ts = train.SRTrainer(ms, p0, n_chains=256, n_per_chain=8, lr=0.05, seed=6)
    ts.run(60)
    E_s = exact_energy(ts.host_params(), J2, proj_p=False)
    mk = nnqs.Model(L, 1.0, J2, K=1, M=M, proj_t=True, proj_p=True, use_bias=True, precision=nnqs.FP32)
    tk = train.SRTrainer(mk, p0, n_chains=256, n_per_chain=8, lr=0.05, seed=7)
    tk.warm_start(ts.params)
    E_warm = exact_energy(tk.host_params(), J2)
    assert E_warm < exact_energy(p0, J2) - 0.3      # far below the random start
    assert E_warm <= E_s + 1e-3                     # projecting on C4v does not undo the training
