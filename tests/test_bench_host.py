"""Host-side counting of the bench: the number of flip sets a Lanczos step
evaluates per configuration, against a brute-force walk of the rule (every
anti-aligned bond b1; after exchanging it, every other bond b2 anti-aligned in
the new configuration, disjoint pairs counted once)."""
import numpy as np

import bench
from paper_2206_14307_gb300 import synth


def brute(x, b):
    cnt = 0
    for b1, (i1, j1) in enumerate(b):
        if x[i1] == x[j1]:
            continue
        cnt += 1
        y = x.copy()
        y[i1], y[j1] = x[j1], x[i1]
        for b2, (i2, j2) in enumerate(b):
            if b2 == b1:
                continue
            if not {i1, j1} & {i2, j2}:
                cnt += int(b2 > b1 and x[i2] != x[j2])
            else:
                cnt += int(y[i2] != y[j2])
    return cnt


def test_lanczos_flip_set_count_matches_brute_force():
    for L in (4, 6):
        b = bench.bonds(L)
        s = synth.random_sz0(L * L, 8, seed=L)
        got = bench.lanczos_entries(s, L)
        assert [brute(x, b) for x in s] == got.tolist()


def test_neel_state_counts():
    # Neel state on 4x4: all 2N J1 bonds anti-aligned, all 2N J2 bonds aligned
    L = 4
    x = np.array([1 if (i % L + i // L) % 2 == 0 else -1 for i in range(L * L)], np.int8)
    assert bench.lanczos_entries(x[None], L)[0] == brute(x, bench.bonds(L))
    assert ((x[bench.bonds(L)[:, 0]] != x[bench.bonds(L)[:, 1]]).sum()) == 2 * L * L
