"""Lanczos-step parity at the 8x8 workload's full model size (Sec. 3.3,
Eqs. 13-18): L = 8, J2/J1 = 0.5, one complex RBM with M = 128, translations x
C4v (|G| = 512), against the FP64 oracle's h1, h2 by double enumeration on 32
configurations drawn from |psi|^2 by the oracle's own sampler (stored in
tests/golden/, written by make_lanczos_8x8.py, which calls only the oracle).

Checked: h1 and h2 element by element, the moments <H^n> (n = 1..4) at 1e-6
relative, and E_p1.  The p = 1 closed form amplifies moment errors by its
condition number kappa = sum_k |dE/dm_k| |m_k| / |E| (derivatives by central
differences); at the parameter scale 0.01 the random state is within about 1%
of the ferromagnetic S = N/2 eigenstate (h1 close to 0.75 N on every sample,
v / m1 ~ 1e-3), kappa is ~6e5, and E_p1 of the FP32 engine is held to the
propagated bound 2 kappa x (moment error); the plain FP64 GPU form meets 1e-6
relative on E_p1 there.  At the 0.05 stress scale the step is better
conditioned and both forms are checked the same way."""
import hashlib
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import to_complex

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FILES = ["lanczos_8x8_m128.txt", "lanczos_8x8_m128_std0.05.txt"]


def load(name):
    path = os.path.join(HERE, "golden", name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    std, digest = None, None
    words, h1, h2 = [], [], []
    for line in open(path):
        if line.startswith("# params:"):
            std = float(line.split("std=")[1].split(",")[0])
            digest = line.split("sha256")[1].strip()
        if line.startswith("#"):
            continue
        f = line.split()
        words.append(int(f[0], 16))
        h1.append(float(f[1]) + 1j * float(f[2]))
        h2.append(float(f[3]) + 1j * float(f[4]))
    return std, digest, np.array(words, np.uint64)[:, None], np.array(h1), np.array(h2)


def kappa(m, E):
    """Relative condition number of the p = 1 energy with respect to m1..m3."""
    k = 0.0
    for i in (1, 2, 3):
        h = 1e-6 * abs(m[i])
        up, dn = m.copy(), m.copy()
        up[i] += h
        dn[i] -= h
        dE = (oracle.lanczos_step(up)["E"] - oracle.lanczos_step(dn)["E"]) / (2 * h)
        k += abs(dE) * abs(m[i])
    return k / abs(E)


@pytest.mark.parametrize("name", FILES)
@pytest.mark.parametrize("prec", [nnqs.FP32, nnqs.FP64])
def test_lanczos_step_8x8_M128_G512_vs_oracle(name, prec):
    std, digest, words, w1, w2 = load(name)
    p = synth.random_params(64, 128, 1, std=std, seed=2206)
    buf = np.ascontiguousarray(np.stack([p.real, p.imag], -1).astype("<f8"))
    assert hashlib.sha256(buf.tobytes()).hexdigest() == digest, "seeded parameters differ from the fixture's"
    gm = nnqs.Model(8, 1.0, 0.5, K=1, M=128, proj_t=True, proj_p=True, spin_inv=0, precision=prec)
    gm.set_params(p)
    assert gm.G == 512
    h1, h2, mo, lz = gm.lanczos(nnqs.cfg_tensor(words))
    gm.status()
    h1, h2, mo, lz = to_complex(h1), to_complex(h2), mo.cpu().numpy(), lz.cpu().numpy()
    e1 = np.max(np.abs(h1 - w1) / np.abs(w1))
    e2 = np.max(np.abs(h2 - w2) / np.abs(w2))
    ref = oracle.moments(w1, w2)
    want_m = np.array([ref["m"][1], ref["m"][2], ref["m"][3], ref["m4"]])
    got_m = np.array([mo[1], mo[2], mo[3], mo[7]])
    em = np.max(np.abs(got_m - want_m) / np.abs(want_m))
    step = oracle.lanczos_step(ref["m"])
    kap = kappa(ref["m"], step["E"])
    eE = abs(lz[0] - step["E"]) / abs(step["E"])
    print(f"\n{name} prec={prec}: h1 rel {e1:.2e}, h2 rel {e2:.2e}, moments rel {em:.2e}, "
          f"E_p1/N gpu {lz[0] / 64:.10f} oracle {step['E'] / 64:.10f} rel {eE:.2e}, kappa {kap:.3e}, "
          f"propagated bound {2 * kap * max(em, 1e-16):.2e}")
    assert mo[4] == len(w1)
    tol = 1e-10 if prec == nnqs.FP64 else 1e-5
    assert e1 <= tol and e2 <= tol
    assert em <= 1e-6 if prec == nnqs.FP32 else em <= 1e-10
    # E_p1: 1e-6 relative where the moment errors allow it; otherwise the
    # propagated bound of the closed form
    assert eE <= max(1e-6, 2 * kap * em)
    if prec == nnqs.FP64:
        assert eE <= 1e-6
    # the device's closed form is the oracle's on the device's own moments
    own = oracle.lanczos_step(mo[:4])
    np.testing.assert_allclose(lz, [own["E"], own["v"], own["alpha"]], rtol=1e-9, atol=1e-12)
