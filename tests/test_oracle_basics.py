"""Oracle pins: Philox known answers, lattice geometry, symmetry group."""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    # Published Philox4x32-10 answers (tests/golden/philox4x32_10_kat.txt).
    n = 0
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        assert list(oracle.philox4x32_10(v[:4], v[4:6])) == v[6:]
        n += 1
    assert n == 3


@pytest.mark.parametrize("L", [4, 6, 8, 10])
def test_bonds_match_geometry(L):
    # Eq. 1: every nearest and every diagonal next-nearest pair exactly once.
    from tests.kron_h import geometric_bonds
    bi, bj, bt = oracle.bonds(L)
    got = sorted((min(a, b), max(a, b), t) for a, b, t in zip(bi, bj, bt))
    want = sorted(geometric_bonds(L))
    assert got == want
    assert len(got) == 4 * L * L


def _compose(p, q):
    # (p o q)(i) = p[q[i]]
    return p[q]


@pytest.mark.parametrize("L,mom,irrep", [(4, 0, 0), (4, 1, 2), (4, 2, 0), (6, 0, 3), (6, 3, 1)])
def test_group_closure_and_characters(L, mom, irrep):
    perm, chi = oracle.group(L, True, True, mom, irrep)
    G = len(perm)
    assert G == (8 if mom <= 1 else 4) * L * L
    keys = {tuple(p): k for k, p in enumerate(perm)}
    assert len(keys) == G
    for p in perm:
        assert sorted(p) == list(range(L * L))
    rng = np.random.default_rng(1)
    pairs = [(a, b) for a in range(G) for b in range(G)]
    for a, b in (pairs if G <= 64 else [pairs[k] for k in rng.choice(len(pairs), 3000, replace=False)]):
        c = keys[tuple(_compose(perm[a], perm[b]))]
        assert chi[c] == chi[a] * chi[b]          # one-dimensional representation


@pytest.mark.parametrize("L", [4, 6])
def test_group_preserves_bond_types(L):
    bi, bj, bt = oracle.bonds(L)
    bset = {(min(a, b), max(a, b)): t for a, b, t in zip(bi, bj, bt)}
    perm, _ = oracle.group(L, True, True, 0, 0)
    for p in perm:
        for (a, b), t in bset.items():
            assert bset[(min(p[a], p[b]), max(p[a], p[b]))] == t


def test_group_unprojected_is_identity():
    perm, chi = oracle.group(6, False, False, 0, 0)
    assert perm.shape == (1, 36) and list(perm[0]) == list(range(36)) and chi[0] == 1.0


def test_rank_select_and_init():
    N = 16
    s = oracle.init_config(99, 3, N)
    assert (s == 1).sum() == N // 2
    for t in range(200):
        iu, idn, u = oracle.proposal(99, 3, t, s)
        assert s[iu] == 1 and s[idn] == -1 and 0.0 <= u < 1.0
        # the chosen sites are the k-th up and k-th down site for some ranks
        ups = np.flatnonzero(s == 1)
        downs = np.flatnonzero(s == -1)
        assert iu in ups and idn in downs
        s = s.copy(); s[iu], s[idn] = -1, 1
    # ranks are uniform over many draws
    cnt = np.zeros(N // 2)
    s = oracle.init_config(5, 0, N)
    ups = list(np.flatnonzero(s == 1))
    for t in range(8000):
        iu, _, _ = oracle.proposal(5, 0, t, s)
        cnt[ups.index(iu)] += 1
    chi2 = ((cnt - 1000) ** 2 / 1000).sum()
    assert chi2 < 30   # 7 dof; p ~ 1e-4


def test_mixed_batch_instances_are_seeded_and_in_range():
    from paper_2206_14307_gb300 import synth
    a = synth.mixed_batch(64, seed=5)
    assert a == synth.mixed_batch(64, seed=5)
    assert a != synth.mixed_batch(64, seed=6)
    assert len(a) == 64
    for d in a:
        assert d["L"] in (4, 6, 8, 10) and d["alpha"] in (1, 2, 4) and d["K"] in (1, 2)
        assert 0.0 <= d["J2"] <= 0.7 and d["M"] == d["alpha"] * d["L"] ** 2
    assert {d["L"] for d in a} == {4, 6, 8, 10}
