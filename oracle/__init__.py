"""FP64 CPU oracle for the projected-RBM VMC path (test infrastructure only).

This package wraps ``nnqs_oracle.c`` -- a plain, slow, double-precision C
implementation of every quantity on the path, evaluated from the paper's
definitions (Sec. 2.1 Eq. 1; Sec. 3.1 Eqs. 2-6; Sec. 3.2 Eqs. 7-12; Sec. 3.3
Eqs. 13-18).  Only the tests, ``__graft_entry__.smoke()`` and the bench's
``cpu_baseline`` / ``--impl reference`` legs may import it.  It shares no code
with the CUDA library.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (brute-force hidden-unit sums, a
Pauli-Kronecker Hamiltonian, ARPACK, finite differences, group invariance,
published Philox answers, exact |psi|^2 statistics); none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nnqs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i, d, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        L.or_model_new.restype = P
        L.or_model_new.argtypes = [i, d, d, i, i, i, i, i, i, i, i, P]
        L.or_model_free.argtypes = [P]
        L.or_model_G.argtypes = [P]
        L.or_model_G.restype = i
        L.or_bonds.argtypes = [i, P, P, P]
        L.or_group.argtypes = [i, i, i, i, i, P, P]
        L.or_params_per_rbm.argtypes = [i, i]
        for fn in ("or_log_psi", "or_local_energy", "or_grad_logpsi"):
            getattr(L, fn).argtypes = [P, P, i, P]
        L.or_lanczos_h.argtypes = [P, P, i, P, P]
        L.or_moments.argtypes = [i, P, P, P, P]
        L.or_lanczos_step.argtypes = [P, P]
        L.or_lanczos_variance.argtypes = [P, P, P]
        L.or_lanczos_h3.argtypes = [P, P, i, P, P, P]
        L.or_shifted_moments.argtypes = [i, P, P, P, d, P, P]
        L.or_krylov2.argtypes = [P, d, P]
        L.or_structure_factor.argtypes = [i, P, i, P, P]
        L.or_energy_grad.argtypes = [i, i, P, P, P, P]
        L.or_sr_solve.argtypes = [i, i, P, P, d, d, P]
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_init_config.argtypes = [u64, i, i, P]
        L.or_proposal.argtypes = [u64, i, ctypes.c_uint32, i, P, P, P, P]
        L.or_sample.argtypes = [P, u64, i, i, i, i, P, P]
        L.or_sz0_basis.argtypes = [i, P]
        L.or_sz0_basis.restype = ctypes.c_long
        L.or_apply_h.argtypes = [i, d, d, P, ctypes.c_long, P, P]
        L.or_ed_ground.argtypes = [i, d, d, i, P]
        L.or_ed_ground.restype = d
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


MOMENTA = {(0, 0): 0, "0,0": 0, (1, 1): 1, "pi,pi": 1, (1, 0): 2, "pi,0": 2, (0, 1): 3, "0,pi": 3}
IRREPS = {"A1": 0, "A2": 1, "B1": 2, "B2": 3}


def bonds(L: int):
    n = 4 * L * L
    bi, bj, bt = (np.zeros(n, np.int32) for _ in range(3))
    lib().or_bonds(L, _p(bi), _p(bj), _p(bt))
    return bi, bj, bt


def group(L: int, proj_t=True, proj_p=True, momentum=0, irrep=0):
    N = L * L
    perm = np.zeros((8 * N, N), np.int32)
    chi = np.zeros(8 * N, np.float64)
    G = lib().or_group(L, int(proj_t), int(proj_p), int(momentum), int(irrep), _p(perm), _p(chi))
    if G < 0:
        raise ValueError("invalid symmetry combination")
    return perm[:G].copy(), chi[:G].copy()


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(o))
    return o


class Model:
    """An oracle model: lattice, projection and complex parameters (FP64).

    params: complex array of K * (1 + N + M + M*N) entries, per RBM
    [log c_r, a[N], b[M], W[M][N] row-major].
    """

    def __init__(self, L, J1=1.0, J2=0.5, K=1, M=None, proj_t=False, proj_p=False, momentum=0,
                 irrep=0, spin_inv=0, use_bias=True, params=None):
        self.L, self.N = L, L * L
        self.K = K
        self.M = M if M is not None else self.N
        self.J1, self.J2 = J1, J2
        self.cfg = dict(proj_t=proj_t, proj_p=proj_p, momentum=momentum, irrep=irrep,
                        spin_inv=spin_inv, use_bias=use_bias)
        self.P1 = 1 + self.N + self.M + self.M * self.N
        self.P = K * self.P1
        params = np.asarray(params, np.complex128).reshape(-1)
        assert params.size == self.P, (params.size, self.P)
        self.params = params
        buf = np.ascontiguousarray(np.stack([params.real, params.imag], -1).reshape(-1))
        self._h = lib().or_model_new(L, J1, J2, K, self.M, int(proj_t), int(proj_p), int(momentum),
                                     int(irrep), int(spin_inv), int(use_bias), _p(buf))
        if not self._h:
            raise ValueError("oracle rejected the model description")
        self.G = lib().or_model_G(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_model_free(self._h)
            self._h = None

    def with_params(self, params):
        return Model(self.L, self.J1, self.J2, self.K, self.M, params=params, **self.cfg)

    @staticmethod
    def _spins(s):
        s = np.ascontiguousarray(np.asarray(s, np.int8))
        if s.ndim == 1:
            s = s[None]
        return s

    def log_psi(self, s):
        s = self._spins(s)
        out = np.zeros((s.shape[0], 2))
        lib().or_log_psi(self._h, _p(s), s.shape[0], _p(out))
        return out[:, 0] + 1j * out[:, 1]

    def local_energy(self, s):
        s = self._spins(s)
        out = np.zeros((s.shape[0], 2))
        lib().or_local_energy(self._h, _p(s), s.shape[0], _p(out))
        return out[:, 0] + 1j * out[:, 1]

    def lanczos_h(self, s):
        s = self._spins(s)
        h1 = np.zeros((s.shape[0], 2))
        h2 = np.zeros((s.shape[0], 2))
        lib().or_lanczos_h(self._h, _p(s), s.shape[0], _p(h1), _p(h2))
        return h1[:, 0] + 1j * h1[:, 1], h2[:, 0] + 1j * h2[:, 1]

    def lanczos_h3(self, s):
        """(h1, h2, h3) with h3 = (H^3 psi)/psi by triple enumeration."""
        s = self._spins(s)
        n = len(s)
        a, b, c = np.zeros((n, 2)), np.zeros((n, 2)), np.zeros((n, 2))
        lib().or_lanczos_h3(self._h, _p(s), n, _p(a), _p(b), _p(c))
        return a[:, 0] + 1j * a[:, 1], b[:, 0] + 1j * b[:, 1], c[:, 0] + 1j * c[:, 1]

    def grad_logpsi(self, s):
        s = self._spins(s)
        out = np.zeros((s.shape[0], self.P, 2))
        lib().or_grad_logpsi(self._h, _p(s), s.shape[0], _p(out))
        return out[..., 0] + 1j * out[..., 1]

    def sample(self, seed, n_chains, n_per_chain, n_skip, n_burn):
        out = np.zeros((n_chains * n_per_chain, self.N), np.int8)
        acc = np.zeros(n_chains)
        lib().or_sample(self._h, ctypes.c_uint64(seed), n_chains, n_per_chain, n_skip, n_burn,
                        _p(out), _p(acc))
        return out, acc


def moments(h1, h2=None, weights=None):
    """Returns dict with m (m0..m3), z (sum of weights), im_h1, im_h1h2."""
    h1 = np.asarray(h1, np.complex128)
    n = h1.size
    a = np.ascontiguousarray(np.stack([h1.real, h1.imag], -1))
    b = None
    if h2 is not None:
        h2 = np.asarray(h2, np.complex128)
        b = np.ascontiguousarray(np.stack([h2.real, h2.imag], -1))
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, np.float64))
    out = np.zeros(8)
    lib().or_moments(n, _p(a), _p(b) if b is not None else None,
                     _p(w) if w is not None else None, _p(out))
    return dict(m=out[:4].copy(), z=out[4], im_h1=out[5], im_h1h2=out[6], m4=out[7])


def lanczos_step(m):
    m = np.ascontiguousarray(np.asarray(m, np.float64))
    out = np.zeros(3)
    lib().or_lanczos_step(_p(m), _p(out))
    return dict(E=out[0], v=out[1], alpha=out[2])


def lanczos_variance(m, lz):
    """m: m0..m4; lz: {E, v, alpha} or [E, v, alpha] -> dict var0, E1, var1, E_extrap."""
    mm = np.ascontiguousarray(np.asarray(m, np.float64)[:5])
    if isinstance(lz, dict):
        lz = [lz["E"], lz["v"], lz["alpha"]]
    ll = np.ascontiguousarray(np.asarray(lz, np.float64))
    out = np.zeros(4)
    lib().or_lanczos_variance(_p(mm), _p(ll), _p(out))
    return dict(var0=out[0], E1=out[1], var1=out[2], E_extrap=out[3])


def shifted_moments(h1, h2, h3, c, weights=None):
    """mu_0..mu_6 of (H - c) from the local h1, h2, h3; returns (mu[7], sum of weights)."""
    cols = [np.ascontiguousarray(np.stack([np.real(x), np.imag(x)], -1).astype(np.float64)) for x in (h1, h2, h3)]
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, np.float64))
    out = np.zeros(8)
    lib().or_shifted_moments(len(cols[0]), _p(cols[0]), _p(cols[1]), _p(cols[2]), float(c),
                             _p(w) if w is not None else None, _p(out))
    return out[:7].copy(), out[7]


def krylov2(mu, c):
    """p = 2 step from mu_0..mu_6 about c: dict E, x (coefficients of (H-c)^i psi0, x0 = 1), var."""
    mu = np.ascontiguousarray(np.asarray(mu, np.float64)[:7])
    out = np.zeros(5)
    lib().or_krylov2(_p(mu), float(c), _p(out))
    return dict(E=out[0], x=out[1:4].copy(), var=out[4])


def structure_factor(L, spins, weights=None):
    """S(q) for q = 2 pi (qx, qy)/L, array [L*L] indexed qx + L qy."""
    s = np.ascontiguousarray(np.asarray(spins, np.int8).reshape(-1, L * L))
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, np.float64))
    out = np.zeros(L * L)
    lib().or_structure_factor(L, _p(s), len(s), _p(w) if w is not None else None, _p(out))
    return out


def energy_grad(O, eloc, weights=None):
    O = np.asarray(O, np.complex128)
    n, P = O.shape
    Ob = np.ascontiguousarray(np.stack([O.real, O.imag], -1))
    e = np.ascontiguousarray(np.stack([np.real(eloc), np.imag(eloc)], -1).astype(np.float64))
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, np.float64))
    F = np.zeros((P, 2))
    lib().or_energy_grad(n, P, _p(Ob), _p(e), _p(w) if w is not None else None, _p(F))
    return F[:, 0] + 1j * F[:, 1]


def sr_solve(O, F, lam=1e-6, dtau=1.0):
    O = np.asarray(O, np.complex128)
    n, P = O.shape
    Ob = np.ascontiguousarray(np.stack([O.real, O.imag], -1))
    Fb = np.ascontiguousarray(np.stack([np.real(F), np.imag(F)], -1).astype(np.float64))
    out = np.zeros((P, 2))
    rc = lib().or_sr_solve(n, P, _p(Ob), _p(Fb), float(lam), float(dtau), _p(out))
    if rc != 0:
        raise np.linalg.LinAlgError("singular SR matrix")
    return out[:, 0] + 1j * out[:, 1]


def init_config(seed, chain, N):
    s = np.zeros(N, np.int8)
    lib().or_init_config(ctypes.c_uint64(seed), chain, N, _p(s))
    return s


def proposal(seed, chain, t, s):
    s = np.ascontiguousarray(np.asarray(s, np.int8))
    iu, idn = ctypes.c_int(), ctypes.c_int()
    u = ctypes.c_double()
    lib().or_proposal(ctypes.c_uint64(seed), chain, ctypes.c_uint32(t), s.size, _p(s),
                      ctypes.byref(iu), ctypes.byref(idn), ctypes.byref(u))
    return iu.value, idn.value, u.value


def sz0_basis(N):
    d = lib().or_sz0_basis(N, None)
    st = np.zeros(d, np.uint64)
    lib().or_sz0_basis(N, _p(st))
    return st


def apply_h(L, J1, J2, states, x):
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    y = np.zeros_like(x)
    lib().or_apply_h(L, J1, J2, _p(states), states.size, _p(x), _p(y))
    return y


def ed_ground(L, J1=1.0, J2=0.5, maxit=300):
    d = lib().or_sz0_basis(L * L, None)
    vec = np.zeros(d)
    E = lib().or_ed_ground(L, J1, J2, maxit, _p(vec))
    return E, vec


def states_to_spins(states, N):
    """Bit i set <=> s_i = +1."""
    st = np.asarray(states, np.uint64)
    bits = (st[:, None] >> np.arange(N, dtype=np.uint64)[None, :]) & np.uint64(1)
    return (2 * bits.astype(np.int8) - 1).astype(np.int8)
