"""Oracle pins for the projected RBM amplitude (Sec. 3.1, Eqs. 2-6)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2206_14307_gb300 import synth


def brute_rbm(params, N, M, s, use_bias=True):
    """Eq. 2 as the marginal of the RBM's Boltzmann weight over hidden units
    h in {-1,+1}^M: sum_h exp(a.s + b.h + h^T W s)."""
    logc = params[0]
    a = params[1:1 + N]
    b = params[1 + N:1 + N + M]
    W = params[1 + N + M:].reshape(M, N)
    if not use_bias:
        a = a * 0
        b = b * 0
    tot = 0
    for h in itertools.product([-1, 1], repeat=M):
        h = np.array(h)
        tot += np.exp(a @ s + b @ h + h @ (W @ s))
    return np.exp(logc) * tot


@pytest.mark.parametrize("use_bias", [True, False])
def test_rbm_equals_hidden_unit_sum(use_bias):
    N, M = 16, 5
    p = synth.random_params(N, M, 1, std=0.3, seed=11)
    m = oracle.Model(4, K=1, M=M, use_bias=use_bias, params=p)
    s = synth.random_sz0(N, 6, seed=3)
    got = m.log_psi(s)
    for k in range(len(s)):
        want = brute_rbm(p, N, M, s[k].astype(float), use_bias)
        assert abs(np.exp(got[k]) - want) <= 1e-11 * abs(want)


def test_sum_of_rbms_equals_sum_of_hidden_sums():
    N, M, K = 16, 4, 3
    p = synth.random_params(N, M, K, std=0.3, seed=12, logc_std=0.5)
    m = oracle.Model(4, K=K, M=M, params=p)
    s = synth.random_sz0(N, 4, seed=4)
    P1 = 1 + N + M + M * N
    got = m.log_psi(s)
    for k in range(len(s)):
        want = sum(brute_rbm(p[r * P1:(r + 1) * P1], N, M, s[k].astype(float)) for r in range(K))
        assert abs(np.exp(got[k]) - want) <= 1e-11 * abs(want)


def _apply(perm_g, s):
    t = np.empty_like(s)
    t[perm_g] = s
    return t


@pytest.mark.parametrize("L,mom,irrep,inv,bias", [(4, 0, 0, 1, True), (4, 0, 2, -1, True), (4, 1, 1, 0, False),
                                                  (4, 2, 3, 1, True), (6, 0, 0, 1, True), (6, 3, 2, 0, False)])
def test_projected_amplitude_transforms_by_character(L, mom, irrep, inv, bias):
    # Eqs. 4-6: psi(h s) = chi(h) psi(s) for every h of the group, and
    # psi(-s) = chi_P psi(s) with spin inversion.
    N = L * L
    M = 6
    p = synth.random_params(N, M, 2, std=0.2, seed=21)
    m = oracle.Model(L, K=2, M=M, proj_t=True, proj_p=True, momentum=mom, irrep=irrep,
                     spin_inv=inv, use_bias=bias, params=p)
    perm, chi = oracle.group(L, True, True, mom, irrep)
    s = synth.random_sz0(N, 3, seed=5)
    base = np.exp(m.log_psi(s))
    rng = np.random.default_rng(0)
    for g in rng.choice(len(perm), 12, replace=False):
        hs = np.stack([_apply(perm[g], x) for x in s])
        # configurations fixed by an element of character -1 have psi = 0
        np.testing.assert_allclose(np.exp(m.log_psi(hs)), chi[g] * base, rtol=1e-11,
                                   atol=1e-11 * np.abs(base).max())
    if inv:
        np.testing.assert_allclose(np.exp(m.log_psi(-s)), inv * base, rtol=1e-11,
                                   atol=1e-11 * np.abs(base).max())


def test_different_irreps_are_orthogonal():
    # Projections onto different one-dimensional irreps are orthogonal over the
    # whole Sz=0 sector of the 4x4 lattice.
    N, M = 16, 4
    p = synth.random_params(N, M, 1, std=0.3, seed=31)
    st = oracle.sz0_basis(N)
    s = oracle.states_to_spins(st, N)
    vecs = []
    for mom, irrep in [(0, 0), (0, 2), (1, 0), (0, 1)]:
        m = oracle.Model(4, K=1, M=M, proj_t=True, proj_p=True, momentum=mom, irrep=irrep, params=p)
        lp = m.log_psi(s)
        v = np.exp(lp - lp.real.max())
        vecs.append(v / np.linalg.norm(v))
    for a in range(len(vecs)):
        for b in range(a + 1, len(vecs)):
            assert abs(np.vdot(vecs[a], vecs[b])) < 1e-12


def test_log_psi_stable_for_large_theta():
    # log 2cosh must not overflow: with W ~ 60 every |theta| is in the hundreds.
    N, M = 16, 3
    p = synth.random_params(N, M, 1, std=60.0, seed=41)
    p[0] = 0
    m = oracle.Model(4, K=1, M=M, use_bias=False, params=p)
    s = synth.random_sz0(N, 3, seed=6)
    lp = m.log_psi(s)
    W = p[1 + N + M:].reshape(M, N)
    for k in range(3):
        th = W @ s[k]
        # for |Re theta| >> 1, log 2cosh(theta) = +-theta up to exp(-2|Re theta|)
        want = np.sum(np.where(th.real >= 0, th, -th))
        assert abs(lp[k].real - want.real) < 1e-9
        d = (lp[k].imag - want.imag) % (2 * np.pi)
        assert min(d, 2 * np.pi - d) < 1e-9
