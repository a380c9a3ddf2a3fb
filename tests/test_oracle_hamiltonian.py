"""Oracle pins for E_loc, (H^2 psi)/psi, moments, Lanczos and ED on 4x4
(Sec. 2.1 Eq. 1, Sec. 3.2 Eq. 10, Sec. 3.3 Eqs. 13-18)."""
import functools

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg as spla

import oracle
from paper_2206_14307_gb300 import synth
from tests.kron_h import hamiltonian_full, sz0_restrict

L, N = 4, 16
J2 = 0.5


@functools.lru_cache(maxsize=None)
def H_sz0(j2=J2):
    H, idx = sz0_restrict(hamiltonian_full(L, 1.0, j2), N)
    return H, idx


@functools.lru_cache(maxsize=None)
def basis():
    st = oracle.sz0_basis(N)
    return st, oracle.states_to_spins(st, N)


def test_basis_matches_kron_ordering():
    st, _ = basis()
    _, idx = H_sz0()
    assert st.size == 12870
    assert np.array_equal(st.astype(np.int64), idx)


def _model(proj=False, **kw):
    M = kw.pop("M", 6)
    K = kw.pop("K", 1)
    p = synth.random_params(N, M, K, std=kw.pop("std", 0.25), seed=kw.pop("seed", 7))
    return oracle.Model(L, 1.0, J2, K=K, M=M, proj_t=proj, proj_p=proj, params=p, **kw)


def _psi_all(m):
    _, s = basis()
    lp = m.log_psi(s)
    return np.exp(lp - lp.real.max())


@pytest.mark.parametrize("proj,inv", [(False, 0), (True, 1)])
def test_local_energy_equals_H_psi_over_psi(proj, inv):
    m = _model(proj, spin_inv=inv, M=4 if proj else 6)
    psi = _psi_all(m)
    H, _ = H_sz0()
    hpsi = H @ psi
    _, s = basis()
    rng = np.random.default_rng(0)
    sel = rng.choice(len(s), 300 if proj else 3000, replace=False)
    sel = sel[np.abs(psi[sel]) > 1e-8 * np.abs(psi).max()]
    e = m.local_energy(s[sel])
    np.testing.assert_allclose(e, hpsi[sel] / psi[sel], rtol=1e-10, atol=1e-10)


def test_h2_equals_H2_psi_over_psi():
    m = _model(False, M=5, seed=8)
    psi = _psi_all(m)
    H, _ = H_sz0()
    hpsi = H @ psi
    h2psi = H @ hpsi
    _, s = basis()
    sel = np.random.default_rng(1).choice(len(s), 60, replace=False)
    h1, h2 = m.lanczos_h(s[sel])
    np.testing.assert_allclose(h1, hpsi[sel] / psi[sel], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(h2, h2psi[sel] / psi[sel], rtol=1e-10, atol=1e-9)


def test_exact_moments_and_lanczos_step():
    # Exact-weight estimators of <H^n> (weights |psi|^2 over the whole sector)
    # equal psi^T H^n psi / psi^T psi from repeated sparse matvecs, and the
    # closed-form p=1 energy equals the lowest generalized eigenvalue of the
    # 2x2 pencil and the Rayleigh-Ritz value in span{psi, H psi}.
    m = _model(False, M=4, seed=9, std=0.3)
    psi = _psi_all(m)
    H, _ = H_sz0()
    _, s = basis()
    h1, h2 = m.lanczos_h(s)
    w = np.abs(psi) ** 2
    mo = oracle.moments(h1, h2, w)
    nrm = np.vdot(psi, psi).real
    v1 = H @ psi
    v2 = H @ v1
    exact = [1.0, np.vdot(psi, v1).real / nrm, np.vdot(v1, v1).real / nrm, np.vdot(v1, v2).real / nrm]
    np.testing.assert_allclose(mo["m"], exact, rtol=1e-12)
    assert abs(mo["im_h1"]) < 1e-12 and abs(mo["im_h1h2"]) < 1e-10
    lz = oracle.lanczos_step(mo["m"])
    mm = mo["m"]
    ev = scipy.linalg.eigh([[mm[1], mm[2]], [mm[2], mm[3]]], [[1, mm[1]], [mm[1], mm[2]]], eigvals_only=True)
    assert abs(lz["E"] - ev[0]) < 1e-10 * abs(ev[0])
    # Rayleigh-Ritz with dense vectors
    B = np.stack([psi, v1], 1)
    Hs = B.conj().T @ (H @ B)
    Ss = B.conj().T @ B
    rr = scipy.linalg.eigh(Hs, Ss, eigvals_only=True)[0]
    assert abs(lz["E"] - rr) < 1e-9 * abs(rr)
    # variational ordering E0 <= E_p1 <= E_var
    E0 = spla.eigsh(H, k=1, which="SA")[0][0]
    assert E0 - 1e-9 <= lz["E"] <= mm[1] + 1e-12
    # eigenvector psi0 + alpha psi1 reproduces the energy
    phi = psi + lz["alpha"] * (v1 - mm[1] * psi) / lz["v"]
    assert abs(np.vdot(phi, H @ phi).real / np.vdot(phi, phi).real - lz["E"]) < 1e-9 * abs(lz["E"])


def test_lanczos_closed_form_on_random_matrices():
    # 2x2 closed form vs the generalized eigensolve for arbitrary spectra.
    rng = np.random.default_rng(3)
    for _ in range(20):
        A = rng.normal(size=(30, 30)); A = A + A.T
        x = rng.normal(size=30); x /= np.linalg.norm(x)
        m = [1.0, x @ A @ x, x @ A @ A @ x, x @ A @ A @ A @ x]
        lz = oracle.lanczos_step(m)
        ev = scipy.linalg.eigh([[m[1], m[2]], [m[2], m[3]]], [[1, m[1]], [m[1], m[2]]], eigvals_only=True)
        assert abs(lz["E"] - ev[0]) < 1e-9 * max(1, abs(ev[0]))


@pytest.mark.parametrize("j2", [0.0, 0.5])
def test_ed_ground_state(j2):
    E, vec = oracle.ed_ground(L, 1.0, j2)
    H, _ = H_sz0(j2)
    E_ref = spla.eigsh(H, k=1, which="SA", tol=1e-12)[0][0]
    assert abs(E - E_ref) < 1e-10 * abs(E_ref)
    assert np.linalg.norm(H @ vec - E * vec) < 1e-8
    if j2 == 0.0:
        # literature value for the 4x4 Heisenberg antiferromagnet, E0/N ~ -0.701780
        assert abs(E / N + 0.70178) < 1e-4
    # the global ground state of the full 2^16 space lies in Sz = 0
    Hf = hamiltonian_full(L, 1.0, j2)
    E_full = spla.eigsh(Hf, k=1, which="SA", tol=1e-10)[0][0]
    assert abs(E_full - E) < 1e-8 * abs(E)


def test_eloc_of_eigenvector_is_constant():
    # Eq. 10 for the exact eigenvector: E_loc(s) = E0 wherever psi(s) != 0;
    # and its moments are those of an eigenstate (v = 0, Lanczos returns E0).
    E, vec = oracle.ed_ground(L, 1.0, J2)
    st, _ = basis()
    hv = oracle.apply_h(L, 1.0, J2, st, vec)
    mask = np.abs(vec) > 1e-6 * np.abs(vec).max()
    np.testing.assert_allclose(hv[mask] / vec[mask], E, rtol=1e-8)
    w = vec ** 2
    h1 = np.where(mask, hv / np.where(mask, vec, 1), E)
    hh = oracle.apply_h(L, 1.0, J2, st, hv)
    h2 = np.where(mask, hh / np.where(mask, vec, 1), E * E)
    mo = oracle.moments(h1, h2, w)
    lz = oracle.lanczos_step(mo["m"])
    assert abs(lz["E"] - E) < 1e-7 * abs(E)


def test_apply_h_matches_kron():
    st, _ = basis()
    H, _ = H_sz0()
    x = np.random.default_rng(4).normal(size=st.size)
    np.testing.assert_allclose(oracle.apply_h(L, 1.0, J2, st, x), H @ x, rtol=1e-12, atol=1e-12)


def test_fourth_moment_and_p1_variance_exact():
    # m4 = <|h2|^2> under exact weights equals psi^T H^4 psi / psi^T psi; the
    # p = 1 state's energy and variance from the moments equal those of the
    # explicit vector phi = psi0 + alpha (H - m1) psi0 / v built with the
    # Kronecker Hamiltonian; E1 equals the closed-form E_p1.
    m = _model(False, M=4, seed=10, std=0.3)
    psi = _psi_all(m)
    H, _ = H_sz0()
    _, s = basis()
    h1, h2 = m.lanczos_h(s)
    mo = oracle.moments(h1, h2, np.abs(psi) ** 2)
    nrm = np.vdot(psi, psi).real
    v2 = H @ (H @ psi)
    np.testing.assert_allclose(mo["m4"], np.vdot(v2, v2).real / nrm, rtol=1e-12)
    m5 = np.concatenate([mo["m"], [mo["m4"]]])
    lz = oracle.lanczos_step(mo["m"])
    var = oracle.lanczos_variance(m5, lz)
    phi = psi + lz["alpha"] * (H @ psi - m5[1] * psi) / lz["v"]
    hphi = H @ phi
    pn = np.vdot(phi, phi).real
    E1 = np.vdot(phi, hphi).real / pn
    var1 = np.vdot(hphi, hphi).real / pn - E1 ** 2
    assert abs(var["E1"] - E1) < 1e-10 * abs(E1)
    assert abs(var["E1"] - lz["E"]) < 1e-10 * abs(E1)
    assert abs(var["var1"] - var1) < 1e-8 * abs(var1)
    assert abs(var["var0"] - (m5[2] - m5[1] ** 2)) < 1e-12 * m5[2]
    assert 0 < var["var1"] < var["var0"]          # a Lanczos step lowers the variance
    # the extrapolated energy lies on the line through both points, at zero variance
    slope = (m5[1] - var["E1"]) / (var["var0"] - var["var1"])
    assert abs(var["E_extrap"] - (var["E1"] - slope * var["var1"])) < 1e-12 * abs(E1)


def test_variance_of_an_eigenstate_vanishes():
    # the ED ground state: zero variance at p = 0 and p = 1, E_extrap = E0
    H, _ = H_sz0(0.0)
    E0, vec = spla.eigsh(H, k=1, which="SA", tol=1e-14)
    v = vec[:, 0] / np.linalg.norm(vec[:, 0])
    # moments of the eigenvector from repeated matvecs
    m, x = [1.0], v
    for _ in range(4):
        y = H @ x
        m.append(np.vdot(v, y).real)
        x = y
    lz = oracle.lanczos_step(m[:4])
    var = oracle.lanczos_variance(m, lz)
    assert lz["alpha"] == 0.0 and abs(var["var0"]) <= 1e-12 * E0[0] ** 2
    assert abs(var["E1"] - E0[0]) < 1e-12 * abs(E0[0]) and abs(var["E_extrap"] - E0[0]) < 1e-9 * abs(E0[0])


def test_h3_equals_H3_psi_over_psi():
    for proj, M, seed in ((False, 5, 11), (True, 4, 12)):
        m = _model(proj, M=M, seed=seed)
        psi = _psi_all(m)
        H, _ = H_sz0()
        v1 = H @ psi
        v2 = H @ v1
        v3 = H @ v2
        _, s = basis()
        sel = np.random.default_rng(2).choice(len(s), 6 if proj else 12, replace=False)
        sel = sel[np.abs(psi[sel]) > 1e-6 * np.abs(psi).max()]
        h1, h2, h3 = m.lanczos_h3(s[sel])
        np.testing.assert_allclose(h1, v1[sel] / psi[sel], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(h2, v2[sel] / psi[sel], rtol=1e-10, atol=1e-9)
        np.testing.assert_allclose(h3, v3[sel] / psi[sel], rtol=1e-10, atol=1e-8)


def test_p2_krylov_step_exact():
    # exact-weight shifted moments = psi^T (H - c)^k psi / psi^T psi (k <= 6);
    # the 3x3 pencil's lowest eigenvalue = scipy's generalized eigensolve =
    # Rayleigh-Ritz in span{psi, H psi, H^2 psi}; E0 <= E_p2 <= E_p1; the
    # variance of the p = 2 state equals that of the explicit vector.
    m = _model(False, M=4, seed=13, std=0.3)
    psi = _psi_all(m)
    H, _ = H_sz0()
    _, s = basis()
    # h3 of the whole sector from dense matvecs would test nothing new; the
    # oracle's triple enumeration is pinned above, so exact weights use it on a
    # subset and the dense vectors for the identities on the full sector
    nrm = np.vdot(psi, psi).real
    c = np.vdot(psi, H @ psi).real / nrm
    Hc = H - c * scipy.sparse.identity(H.shape[0], format="csr")
    vs = [psi]
    for _ in range(3):
        vs.append(Hc @ vs[-1])
    mu_exact = [np.vdot(vs[i], vs[j]).real / nrm for i, j in ((0, 0), (0, 1), (1, 1), (1, 2), (2, 2), (2, 3), (3, 3))]
    h1 = (H @ psi) / psi
    h2 = (H @ (H @ psi)) / psi
    h3 = (H @ (H @ (H @ psi))) / psi
    mu, z = oracle.shifted_moments(h1, h2, h3, c, np.abs(psi) ** 2)
    np.testing.assert_allclose(mu, mu_exact, rtol=1e-9, atol=1e-9 * mu_exact[2])
    k2 = oracle.krylov2(mu, c)
    A = np.array([[mu[i + j + 1] for j in range(3)] for i in range(3)])
    B = np.array([[mu[i + j] for j in range(3)] for i in range(3)])
    ev = scipy.linalg.eigh(A, B, eigvals_only=True)
    assert abs(k2["E"] - (c + ev[0])) < 1e-9 * abs(k2["E"])
    Q, _ = np.linalg.qr(np.stack([psi, H @ psi, H @ (H @ psi)], 1))
    rr = np.linalg.eigvalsh(Q.conj().T @ (H @ Q))[0]
    assert abs(k2["E"] - rr) < 1e-8 * abs(rr)
    E0 = spla.eigsh(H, k=1, which="SA")[0][0]
    m4 = oracle.moments(h1, h2, np.abs(psi) ** 2)
    E1 = oracle.lanczos_step(m4["m"])["E"]
    assert E0 - 1e-9 <= k2["E"] <= E1 + 1e-9
    x = k2["x"]
    assert x[0] == 1.0
    phi = vs[0] + x[1] * vs[1] + x[2] * vs[2]
    hphi = H @ phi
    pn = np.vdot(phi, phi).real
    Ephi = np.vdot(phi, hphi).real / pn
    assert abs(Ephi - k2["E"]) < 1e-9 * abs(Ephi)
    var = np.vdot(hphi, hphi).real / pn - Ephi ** 2
    assert abs(k2["var"] - var) < 1e-6 * abs(var) + 1e-12
    # the shift does not change the step
    mu2, _ = oracle.shifted_moments(h1, h2, h3, c + 0.37, np.abs(psi) ** 2)
    assert abs(oracle.krylov2(mu2, c + 0.37)["E"] - k2["E"]) < 1e-8 * abs(k2["E"])
