"""The two FP32 engines of h1 = (H psi)/psi and h2 = (H^2 psi)/psi (Sec. 3.3)
agree: the shared-memory per-site-table form (second-level flip sets as
exchanges in the once-exchanged configuration, one CTA per SM) and the general
connected-configuration engine (forced by the test hook
NNQS_TEST_ELOC_ENGINE=old), on the 8x8 workload shape, on widths up to 256
hidden units, with several RBMs, no biases, odd inversion and a B1 irrep; a
capped flip-set list (test hook NNQS_TEST_LANCZOS_LIST) makes samples take
several passes, and the plain second-level form 1 + p'(U - 1) (taken where some
|p'| < 2^-12; forced by NNQS_TEST_LANCZOS_PLAIN) is checked the same way.  Both are also checked against the FP64 oracle's double
enumeration on a few samples."""
import os

import numpy as np
import pytest

from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import annihilated, make_pair, to_complex

pytestmark = pytest.mark.gpu


def _with_env(name, value, fn):
    old = os.environ.pop(name, None)
    try:
        if value is not None:
            os.environ[name] = value
        return fn()
    finally:
        if old is None:
            os.environ.pop(name, None)
        else:
            os.environ[name] = old


def _h(gm, cfg):
    h1, h2, _, _ = gm.lanczos(cfg)
    return to_complex(h1), to_complex(h2)


@pytest.mark.parametrize("L,K,M,inv,bias,irrep,std,n,cap,plain", [
    (8, 1, 128, 0, True, 0, 0.01, 96, None, None),   # the 8x8 workload shape
    (8, 1, 128, 0, True, 0, 0.01, 24, "300", None),  # several passes per sample
    (8, 1, 128, 0, True, 0, 0.01, 48, None, "1"),    # the plain form throughout
    (4, 1, 16, 0, True, 0, 1.0, 100, None, None),    # some |p'| below 2^-12
    (6, 1, 72, 1, True, 0, 0.05, 200, None, None),
    (6, 1, 144, 1, True, 0, 0.02, 100, None, None),  # 32 lanes per row
    (4, 1, 200, 0, True, 0, 0.02, 100, None, None),
    (6, 2, 20, 0, False, 0, 0.1, 150, None, None),
    (4, 2, 12, -1, True, 2, 0.2, 150, "40", "1"),
    (4, 1, 16, 0, True, 0, 0.3, 150, None, None),
])
def test_fast_lanczos_matches_general_engine(L, K, M, inv, bias, irrep, std, n, cap, plain):
    N = L * L
    om, gm, _ = make_pair(L, K=K, M=M, proj=True, spin_inv=inv, use_bias=bias, irrep=irrep, std=std,
                          precision=nnqs.FP32, logc_std=0.2 if K > 1 else None)
    s = synth.random_sz0(N, 3 * n, seed=19)
    s = s[~annihilated(L, s, True, 0, irrep, inv, bias)][:n]
    cfg = nnqs.cfg_tensor(synth.pack(s))
    f1, f2 = _with_env("NNQS_TEST_ELOC_ENGINE", None, lambda: _with_env(
        "NNQS_TEST_LANCZOS_LIST", cap, lambda: _with_env("NNQS_TEST_LANCZOS_PLAIN", plain, lambda: _h(gm, cfg))))
    g1, g2 = _with_env("NNQS_TEST_ELOC_ENGINE", "old", lambda: _h(gm, cfg))
    gm.status()
    k = len(s) if N <= 16 else 1 if N >= 64 else 3
    w1, w2 = om.lanczos_h(s[:k])

    def err(a, b):
        return np.max(np.abs(a - b) / (np.abs(b) + 1))

    e_fast = max(err(f1[:k], w1), err(f2[:k], w2))
    e_old = max(err(g1[:k], w1), err(g2[:k], w2))
    print(f"\nL={L} M={M} std={std}: fast vs oracle {e_fast:.2e}, general vs oracle {e_old:.2e}, "
          f"fast vs general {max(err(f1, g1), err(f2, g2)):.2e}")
    tol = 1e-5 if std <= 0.05 else 1e-4
    if std <= 0.3:
        assert err(f1, g1) <= tol and err(f2, g2) <= tol
        assert e_fast <= tol
    else:
        # far from the workload's parameter scale FP32 itself is ill-conditioned
        # (|p| near the zeros of cosh): no worse than the general FP32 engine
        assert e_fast <= max(tol, 10 * e_old)
