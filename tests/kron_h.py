"""Independent J1-J2 Hamiltonian for the oracle pins (test helper).

Built as a sum of two-site operators S_i.S_j = S^z S^z + (S^+ S^- + S^- S^+)/2,
each a Kronecker product of 2x2 spin matrices (site i <-> bit i, bit set <=> up),
in the full 2^N space, then restricted to the Sz = 0 sector.  It shares nothing
with the oracle's bit-manipulation matrix elements; only the list of bonds
comes from the lattice geometry, which is checked separately.
"""
import numpy as np
import scipy.sparse as sp

SZ = sp.csr_matrix(np.array([[-0.5, 0.0], [0.0, 0.5]]))
SP = sp.csr_matrix(np.array([[0.0, 0.0], [1.0, 0.0]]))  # |up><down|
SM = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))


def site_op(op, i, N):
    return sp.kron(sp.identity(2 ** (N - 1 - i), format="csr"),
                   sp.kron(op, sp.identity(2 ** i, format="csr"), format="csr"), format="csr")


def geometric_bonds(L):
    """Nearest (|dr| = 1) and diagonal next-nearest (|dr| = sqrt 2) pairs of the
    periodic L x L lattice, found by distance rather than by construction."""
    N = L * L
    out = []
    for i in range(N):
        for j in range(i + 1, N):
            dx = min(abs(i % L - j % L), L - abs(i % L - j % L))
            dy = min(abs(i // L - j // L), L - abs(i // L - j // L))
            if dx * dx + dy * dy == 1:
                out.append((i, j, 1))
            elif dx == 1 and dy == 1:
                out.append((i, j, 2))
    return out


def hamiltonian_full(L, J1, J2):
    N = L * L
    H = sp.csr_matrix((2 ** N, 2 ** N))
    ops = {}
    for i in range(N):
        ops[i] = (site_op(SZ, i, N), site_op(SP, i, N), site_op(SM, i, N))
    for i, j, t in geometric_bonds(L):
        J = J1 if t == 1 else J2
        zi, pi, mi = ops[i]
        zj, pj, mj = ops[j]
        H = H + J * (zi @ zj + 0.5 * (pi @ mj + mi @ pj))
    return H.tocsr()


def sz0_restrict(H, N):
    idx = np.array([x for x in range(2 ** N) if bin(x).count("1") == N // 2], dtype=np.int64)
    return H[idx][:, idx].tocsr(), idx
