"""Writes lanczos_8x8_m128.txt (and, with --std 0.05, lanczos_8x8_m128_std0.05.txt):
the FP64 oracle's Lanczos-step quantities on the 8x8 workload, for the GPU
parity test at full model size.

Workload: L = 8 periodic J1-J2 lattice, J2/J1 = 0.5, one complex RBM with
M = 128 hidden units and biases, projected over the 64 translations x C4v
(|G| = 512), A1, K = (0,0), no spin inversion; parameters N(0, 0.01^2) per
real and imaginary part (seed 2206; --std 0.05 for the stress scale, where the
state is farther from the ferromagnetic eigenstate and the p = 1 step is better
conditioned).  Configurations: 32 independent chains
of the oracle's own Metropolis sampler (seed 14307, burn-in 100 steps, one
sample after 10 more steps per chain), i.e. draws from |psi|^2.

Per configuration the oracle gives h1 = (H psi)/psi and h2 = (H^2 psi)/psi
(Sec. 3.3) by explicit double enumeration, every psi(s'') from scratch.  This
script calls only the oracle and the seeded input generator; nothing here
comes from the CUDA library.  About 15 minutes on 8 cores.

    python tests/golden/make_lanczos_8x8.py [--std 0.05]
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2206_14307_gb300 import synth  # noqa: E402

L, J1, J2, M, STD, PSEED = 8, 1.0, 0.5, 128, 0.01, 2206
SSEED, CHAINS, SKIP, BURN = 14307, 32, 10, 100


def out_path(std):
    return os.path.join(HERE, "lanczos_8x8_m128.txt" if std == 0.01 else f"lanczos_8x8_m128_std{std}.txt")


def params_digest(p):
    """SHA-256 of the parameters as little-endian (re, im) doubles."""
    buf = np.ascontiguousarray(np.stack([p.real, p.imag], -1).astype("<f8"))
    return hashlib.sha256(buf.tobytes()).hexdigest()


def main(std=STD):
    N = L * L
    OUT = out_path(std)
    p = synth.random_params(N, M, 1, std=std, seed=PSEED)
    om = oracle.Model(L, J1, J2, K=1, M=M, proj_t=True, proj_p=True, spin_inv=0, params=p)
    assert om.G == 512
    s, acc = om.sample(SSEED, CHAINS, 1, SKIP, BURN)
    h1, h2 = om.lanczos_h(s)
    words = synth.pack(s)
    with open(OUT, "w") as f:
        f.write("# Oracle (FP64) Lanczos-step quantities, 8x8 J1-J2 (J2/J1=0.5), complex RBM M=128,\n")
        f.write("# translations x C4v (|G|=512), A1, K=(0,0), no inversion, biases on.\n")
        f.write(f"# params: synth.random_params(64, 128, 1, std={std}, seed={PSEED}) sha256 {params_digest(p)}\n")
        f.write(f"# configurations: oracle sampler, seed {SSEED}, {CHAINS} chains x 1, n_skip {SKIP}, "
                f"n_burn {BURN}\n")
        f.write("# written by tests/golden/make_lanczos_8x8.py (calls only oracle/ and synth)\n")
        f.write("# columns: cfg word (hex, bit i <=> s_i = +1)  Re h1  Im h1  Re h2  Im h2\n")
        for k in range(len(s)):
            f.write(f"{int(words[k, 0]):016x} {h1[k].real:.17e} {h1[k].imag:.17e} "
                    f"{h2[k].real:.17e} {h2[k].imag:.17e}\n")
    print(f"wrote {OUT}: {len(s)} configurations, mean acceptance {acc.mean():.3f}")


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--std", type=float, default=STD)
    main(ap.parse_args().std)
