"""Host policy of the SR loop (Sec. 3.4) with a stand-in model on the CPU:
N_skip = ceil(5 / r) from the previous step's acceptance, the learning rate
halved when the windowed mean energy stops decreasing, the parameter update
from the solve, and the warm start."""
import numpy as np
import torch

from paper_2206_14307_gb300 import train


class FakeModel:
    """Records the calls; energies follow a given schedule."""

    def __init__(self, energies, acc):
        self.energies, self.acc = list(energies), acc
        self.calls, self.set = [], 0

    def set_params(self, p):
        self.set += 1

    def sample(self, seed, n_chains, n_per_chain, n_skip, n_burn):
        self.calls.append(("sample", seed, n_skip, n_burn))
        return torch.zeros(n_chains * n_per_chain, 1, dtype=torch.int64), torch.full((n_chains,), self.acc)

    def local_energy(self, cfg, sums):
        e = self.energies.pop(0)
        n = cfg.shape[0]
        sums.copy_(torch.tensor([e * n, 0.0, e * e * n + n, float(n)], dtype=torch.float64))
        return torch.zeros(n, 2, dtype=torch.float64)

    def grad_logpsi(self, cfg):
        return torch.zeros(cfg.shape[0], 3, 2, dtype=torch.float64)

    def energy_grad(self, O, eloc):
        return torch.zeros(3, 2, dtype=torch.float64)

    def sr_solve(self, O, F, lam, dtau, max_iter, tol, params_inout):
        params_inout.add_(dtau)      # a visible update of size dtau
        return torch.full((3, 2), dtau, dtype=torch.float64), torch.tensor([7.0, 1e-11], dtype=torch.float64)


def test_n_skip_follows_acceptance_and_lr_halves_on_stall():
    # 20 decreasing energies, then flat ones: the window mean of steps 20-29
    # (-19) is still below that of steps 10-19 (-14.5); steps 30-39 equal
    # steps 20-29, so the lr halves at step 40, and again at step 50
    energies = [-float(k) for k in range(20)] + [-19.0] * 30
    m = FakeModel(energies, acc=0.2)
    tr = train.SRTrainer(m, np.zeros(3, complex), n_chains=4, n_per_chain=2, lr=0.04, n_skip=10, window=10,
                         device="cpu")
    tr.run(30)
    h = tr.history
    assert h[0]["n_skip"] == 10 and all(x["n_skip"] == 25 for x in h[1:])   # ceil(5 / 0.2)
    assert m.calls[1][2] == 25 and m.calls[1][3] == 250                      # burn-in 10 N_skip
    assert tr.lr == 0.04
    tr.run(10)
    assert [x["lr"] for x in h] == [0.04] * 40 and tr.lr == 0.02
    tr.run(10)
    assert tr.lr == 0.01
    # the solve's in-place update accumulates: sum of the lr used at each step
    np.testing.assert_allclose(tr.params.numpy(), 40 * 0.04 + 10 * 0.02)
    assert h[0]["cg_iter"] == 7.0 and h[0]["E"] == 0.0 and abs(h[0]["var"] - 1.0) < 1e-12


def test_lr_floor_and_warm_start():
    m = FakeModel([1.0] * 60, acc=1.0)
    tr = train.SRTrainer(m, np.zeros(3, complex), n_chains=2, n_per_chain=1, lr=0.01, window=5, lr_min=2e-3,
                         device="cpu")
    tr.run(60)
    assert tr.lr == 2e-3 and tr.n_skip == 5
    tr.warm_start(np.array([1 + 2j, 3 - 1j, 0.5j]))
    np.testing.assert_array_equal(tr.host_params(), [1 + 2j, 3 - 1j, 0.5j])
