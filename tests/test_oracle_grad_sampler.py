"""Oracle pins for O_k, the energy gradient, SR (Eq. 12) and the Metropolis
pair-exchange sampler (Sec. 3.2)."""
import numpy as np
import pytest
import scipy.stats

import oracle
from paper_2206_14307_gb300 import synth

L, N = 4, 16


@pytest.mark.parametrize("proj,inv,bias,K", [(False, 0, True, 1), (True, 1, True, 2), (True, -1, True, 1), (True, 1, False, 1)])
def test_grad_logpsi_matches_holomorphic_fd(proj, inv, bias, K):
    M = 3
    p = synth.random_params(N, M, K, std=0.2, seed=51, logc_std=0.3)
    m = oracle.Model(L, K=K, M=M, proj_t=proj, proj_p=proj, spin_inv=inv, use_bias=bias, params=p)
    s = synth.random_sz0(N, 2, seed=8)
    O = m.grad_logpsi(s)
    rng = np.random.default_rng(2)
    idx = rng.choice(m.P, 25, replace=False)
    h = 1e-5
    for q in idx:
        dp = np.zeros(m.P, complex); dp[q] = h
        lp = m.with_params(p + dp).log_psi(s)
        lm = m.with_params(p - dp).log_psi(s)
        d = lp - lm
        d = d.real + 1j * ((d.imag + np.pi) % (2 * np.pi) - np.pi)
        fd = d / (2 * h)
        np.testing.assert_allclose(O[:, q], fd, rtol=1e-6, atol=1e-8)


def test_odd_inversion_without_bias_is_rejected():
    p = synth.random_params(N, 3, 1, seed=1)
    with pytest.raises(ValueError):
        oracle.Model(L, K=1, M=3, proj_t=True, proj_p=True, spin_inv=-1, use_bias=False, params=p)


def test_energy_gradient_matches_fd_of_exact_energy():
    # With exact weights |psi|^2 over the whole 4x4 Sz=0 sector,
    # dE/dRe alpha_k = 2 Re F_k and dE/dIm alpha_k = 2 Im F_k, where
    # E(alpha) = <psi|H|psi>/<psi|psi> is formed with the Kronecker-product
    # Hamiltonian.
    from tests.kron_h import hamiltonian_full, sz0_restrict
    M = 3
    p = synth.random_params(N, M, 1, std=0.2, seed=52)
    m = oracle.Model(L, K=1, M=M, proj_t=True, proj_p=True, spin_inv=1, params=p)
    st = oracle.sz0_basis(N)
    s = oracle.states_to_spins(st, N)
    H, _ = sz0_restrict(hamiltonian_full(L, 1.0, 0.5), N)

    def E(par):
        lp = m.with_params(par).log_psi(s)
        psi = np.exp(lp - lp.real.max())
        return (np.vdot(psi, H @ psi) / np.vdot(psi, psi)).real

    lp0 = m.log_psi(s)
    w = np.exp(2 * (lp0.real - lp0.real.max()))
    keep = w > 1e-20 * w.max()
    rng = np.random.default_rng(3)
    qs = rng.choice(m.P, 8, replace=False)
    sub = np.flatnonzero(keep)
    O = m.grad_logpsi(s[sub])
    e = m.local_energy(s[sub])
    F = oracle.energy_grad(O, e, w[sub])
    h = 1e-5
    for q in qs:
        for unit, part in ((1.0, lambda z: 2 * z.real), (1j, lambda z: 2 * z.imag)):
            dp = np.zeros(m.P, complex); dp[q] = unit * h
            fd = (E(p + dp) - E(p - dp)) / (2 * h)
            assert abs(fd - part(F[q])) < 1e-7 * max(1.0, abs(fd))


def test_sr_step_is_regularised_least_squares():
    # Eq. 12 with ridge lambda is the normal equation of
    #   min_d || (O - <O>) d / sqrt(n) + dtau (E_loc - <E>) / sqrt(n) ||^2 + lambda ||d||^2,
    # solved here with a QR least-squares routine on the stacked system.
    rng = np.random.default_rng(4)
    n, P = 40, 12
    O = rng.normal(size=(n, P)) + 1j * rng.normal(size=(n, P))
    e = rng.normal(size=n) + 1j * rng.normal(size=n)
    lam, dtau = 1e-3, 0.05
    F = oracle.energy_grad(O, e)
    d = oracle.sr_solve(O, F, lam, dtau)
    A = np.vstack([(O - O.mean(0)) / np.sqrt(n), np.sqrt(lam) * np.eye(P)])
    b = np.concatenate([-dtau * (e - e.mean()) / np.sqrt(n), np.zeros(P)])
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(d, ref, rtol=1e-9, atol=1e-12)


def test_sampler_matches_exact_distribution():
    # Independent chains (last state of each after a long burn-in) are
    # distributed as |psi|^2 / sum |psi|^2: chi-square over 16 bins of equal
    # exact probability, formed by sorting the 12870 states by |psi|^2.
    M = 4
    p = synth.random_params(N, M, 1, std=0.35, seed=61)
    m = oracle.Model(L, K=1, M=M, params=p)
    st = oracle.sz0_basis(N)
    s_all = oracle.states_to_spins(st, N)
    lp = m.log_psi(s_all)
    prob = np.exp(2 * (lp.real - lp.real.max()))
    prob /= prob.sum()
    order = np.argsort(prob)
    cum = np.cumsum(prob[order])
    nb = 16
    bin_of = np.empty(st.size, int)
    bin_of[order] = np.minimum((cum * nb).astype(int), nb - 1)
    pbin = np.bincount(bin_of, weights=prob, minlength=nb)
    n_chains = 12000
    out, acc = m.sample(seed=2024, n_chains=n_chains, n_per_chain=1, n_skip=1, n_burn=150)
    assert np.all((out == 1).sum(1) == N // 2)
    code = ((out > 0).astype(np.uint64) << np.arange(N, dtype=np.uint64)).sum(1)
    pos = np.searchsorted(st, code)
    assert np.all(st[pos] == code)
    counts = np.bincount(bin_of[pos], minlength=nb)
    chi2 = ((counts - n_chains * pbin) ** 2 / (n_chains * pbin)).sum()
    assert scipy.stats.chi2.sf(chi2, nb - 1) > 1e-4
    # mean local energy of the samples agrees with the exact variational energy
    e = m.local_energy(out)
    psi = np.exp(lp - lp.real.max())
    from tests.kron_h import hamiltonian_full, sz0_restrict
    H, _ = sz0_restrict(hamiltonian_full(L, 1.0, 0.5), N)
    Evar = (np.vdot(psi, H @ psi) / np.vdot(psi, psi)).real
    err = e.real.std() / np.sqrt(n_chains)
    assert abs(e.real.mean() - Evar) < 5 * err


def test_sampler_chain_is_a_metropolis_walk():
    # Consecutive states differ by nothing or by one up/down exchange, the
    # exchanged pair is the Philox proposal of that step, and the decision
    # follows u < |psi'/psi|^2.
    M = 4
    p = synth.random_params(N, M, 1, std=0.3, seed=62)
    m = oracle.Model(L, K=1, M=M, params=p)
    out, acc = m.sample(seed=77, n_chains=2, n_per_chain=120, n_skip=1, n_burn=0)
    for c in range(2):
        prev = oracle.init_config(77, c, N)
        for t in range(120):
            cur = out[c * 120 + t]
            iu, idn, u = oracle.proposal(77, c, t, prev)
            prop = prev.copy(); prop[iu], prop[idn] = -1, 1
            r2 = np.exp(2 * (m.log_psi(prop)[0] - m.log_psi(prev)[0]).real)
            assert np.array_equal(cur, prop if u < r2 else prev)
            prev = cur
