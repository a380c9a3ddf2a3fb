"""The two FP32 E_loc engines agree: the shared-memory per-bond-table form
(one CTA per SM, packed FP32x2, factors p (q + U) with q = (1 - p)/p) and the
general connected-configuration engine (forced by the test hook
NNQS_TEST_ELOC_ENGINE=old), on the 6x6 workload shape and on shapes with
several RBMs, no biases, odd inversion and a B1 irrep; the plain factors
1 + p (U - 1) (taken where some |p| < 2^-12; forced by NNQS_TEST_ELOC_PLAIN=1)
are checked the same way; both engines are also checked against the FP64
oracle on a few samples (at std 1.0, within 10x the general engine's own
distance from it)."""
import os

import numpy as np
import pytest

from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import annihilated, make_pair, to_complex

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,K,M,inv,bias,irrep,std,n,plain", [
    (6, 1, 72, 1, True, 0, 0.01, 2000, None),    # the 6x6 workload
    (6, 1, 72, 1, True, 0, 0.01, 500, "1"),      # the plain factors throughout
    (6, 1, 72, 1, True, 0, 0.05, 500, None),
    (6, 2, 20, 0, False, 0, 0.1, 300, None),
    (4, 2, 12, -1, True, 2, 0.2, 300, "1"),
    (4, 1, 16, 0, True, 0, 0.3, 300, None),
    (6, 1, 36, 1, True, 0, 0.05, 300, None),
    (4, 1, 16, 0, True, 0, 1.0, 100, None),     # large parameters: |q| far from 1 both ways
    (4, 1, 16, 1, True, 0, 1.0, 100, None),
])
def test_fast_eloc_matches_general_engine(L, K, M, inv, bias, irrep, std, n, plain):
    N = L * L
    om, gm, _ = make_pair(L, K=K, M=M, proj=True, spin_inv=inv, use_bias=bias, irrep=irrep, std=std,
                          precision=nnqs.FP32, logc_std=0.2 if K > 1 else None)
    s = synth.random_sz0(N, 3 * n, seed=17)
    s = s[~annihilated(L, s, True, 0, irrep, inv, bias)][:n]
    cfg = nnqs.cfg_tensor(synth.pack(s))
    old = os.environ.pop("NNQS_TEST_ELOC_ENGINE", None)
    try:
        if plain:
            os.environ["NNQS_TEST_ELOC_PLAIN"] = plain
        fast = to_complex(gm.local_energy(cfg))
        os.environ.pop("NNQS_TEST_ELOC_PLAIN", None)
        os.environ["NNQS_TEST_ELOC_ENGINE"] = "old"
        gen = to_complex(gm.local_energy(cfg))
    finally:
        os.environ.pop("NNQS_TEST_ELOC_PLAIN", None)
        if old is None:
            os.environ.pop("NNQS_TEST_ELOC_ENGINE", None)
        else:
            os.environ["NNQS_TEST_ELOC_ENGINE"] = old
    gm.status()
    if std <= 0.3:
        tol = 1e-5 if std <= 0.05 else 1e-4
        assert np.max(np.abs(fast - gen) / (np.abs(gen) + 1)) <= tol
        want = om.local_energy(s[:4])
        assert np.max(np.abs(fast[:4] - want) / (np.abs(want) + 1)) <= tol
    else:
        # std 1.0: E_loc reaches 1e6 through cancelling ratios, beyond what FP32
        # holds; on every sample the fast engine is held to the general FP32
        # engine's own distance from the FP64 oracle
        want = om.local_energy(s)
        err = np.abs(fast - want) / (np.abs(want) + 1)
        err_gen = np.abs(gen - want) / (np.abs(want) + 1)
        assert np.all(err <= 10 * err_gen + 1e-5), (np.max(err), np.max(err_gen))
