"""Stochastic-reconfiguration training loop (Sec. 3.2 Eq. 12; Sec. 3.4).

Every step runs on the GPU through the C ABI: Metropolis sampling, E_loc with
its FP64 sums, the hand-written O_k kernel, the energy gradient F and the
FP64 conjugate-gradient solve of (S + lambda) delta = -dtau F, which also
applies alpha += delta to the device parameters.  Only the policy of Sec. 3.4
lives here on the host:

  - N_skip = ceil(5 / r) with r the acceptance rate of the previous step;
  - the learning rate dtau is halved when the windowed mean energy stops
    decreasing (down to a floor);
  - a warm start copies the parameters of a cheaper wave function with the
    same layout (psi_s -> psi_KL: the same RBM, projected on more symmetries).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import nnqs


class SRTrainer:
    """SR on one model; parameters live in ``self.params`` (float64 CUDA
    tensor [P, 2]) and in the model's tables."""

    def __init__(self, model: nnqs.Model, params, n_chains=256, n_per_chain=8, lr=0.02, lam=1e-6, n_skip=10,
                 n_burn=None, seed=1, cg_iter=200, cg_tol=1e-10, window=10, lr_min=5e-4, n_skip_max=100,
                 device="cuda"):
        self.model = model
        self.device = device
        p = np.asarray(params, np.complex128).reshape(-1)
        self.params = torch.tensor(np.stack([p.real, p.imag], -1), dtype=torch.float64, device=device)
        model.set_params(self.params)
        self.n_chains, self.n_per_chain = n_chains, n_per_chain
        self.lr, self.lam, self.n_skip = lr, lam, n_skip
        self.n_burn = n_burn
        self.seed = seed
        self.cg_iter, self.cg_tol = cg_iter, cg_tol
        self.window, self.lr_min, self.n_skip_max = window, lr_min, n_skip_max
        self.history: list[dict] = []
        self._sums = torch.empty(4, dtype=torch.float64, device=device)

    def warm_start(self, params):
        """Start from another wave function's parameters (same K, N, M layout)."""
        if isinstance(params, torch.Tensor):
            self.params.copy_(params)
        else:
            p = np.asarray(params, np.complex128).reshape(-1)
            self.params.copy_(torch.tensor(np.stack([p.real, p.imag], -1), dtype=torch.float64))
        self.model.set_params(self.params)

    def host_params(self) -> np.ndarray:
        a = self.params.cpu().numpy()
        return a[:, 0] + 1j * a[:, 1]

    def step(self) -> dict:
        k = len(self.history)
        m = self.model
        burn = self.n_burn if self.n_burn is not None else 10 * self.n_skip
        cfg, acc = m.sample(self.seed * 1000003 + k, self.n_chains, self.n_per_chain, self.n_skip, burn)
        eloc = m.local_energy(cfg, sums=self._sums)
        O = m.grad_logpsi(cfg)
        F = m.energy_grad(O, eloc)
        _, info = m.sr_solve(O, F, lam=self.lam, dtau=self.lr, max_iter=self.cg_iter, tol=self.cg_tol,
                             params_inout=self.params)
        m.set_params(self.params)
        s = self._sums.cpu().numpy()
        n = s[3]
        E = s[0] / n
        var = max(s[2] / n - E * E, 0.0)
        r = float(acc.mean().item())
        rec = dict(step=k, E=E, var=var, acc=r, n_skip=self.n_skip, lr=self.lr,
                   cg_iter=float(info[0].item()), cg_res=float(info[1].item()))
        self.history.append(rec)
        # Sec. 3.4: N_skip from the acceptance rate of this step
        self.n_skip = int(min(self.n_skip_max, max(1, math.ceil(5.0 / max(r, 1e-3)))))
        # halve the learning rate when the windowed mean energy stops decreasing
        w = self.window
        if len(self.history) >= 2 * w and len(self.history) % w == 0:
            cur = np.mean([h["E"] for h in self.history[-w:]])
            prev = np.mean([h["E"] for h in self.history[-2 * w:-w]])
            if cur >= prev:
                self.lr = max(self.lr_min, 0.5 * self.lr)
        return rec

    def run(self, steps: int) -> list[dict]:
        for _ in range(steps):
            self.step()
        return self.history
