"""The C ABI library loads and exports every function declared in
include/nnqs.h; argument validation happens on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nnqs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nnqs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_14307_gb300 import build
    build.build()
    from paper_2206_14307_gb300 import nnqs
    return nnqs.lib()


def test_header_declares_the_abi():
    names = declared_functions()
    for want in ("nnqs_create", "nnqs_sample", "nnqs_log_psi", "nnqs_local_energy", "nnqs_lanczos_moments",
                 "nnqs_grad_logpsi"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2206_14307_gb300 import nnqs
    so = nnqs.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (nnqs_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(nnqs.ABI_FUNCTIONS) == set(declared_functions())


@pytest.mark.parametrize("field,value,code", [("L", 5, -5), ("L", 2, -5), ("L", 18, -5), ("K", 0, -5),
                                              ("M", 0, -5), ("M", 513, -5), ("momentum", 4, -1),
                                              ("irrep", 7, -1), ("spin_inversion", 2, -1), ("precision", 9, -1)])
def test_invalid_descriptions_rejected_on_host(lib, field, value, code):
    from paper_2206_14307_gb300 import nnqs
    d = nnqs.nnqs_desc(6, 1.0, 0.5, 1, 36, 1, 1, 0, 0, 1, 1, nnqs.FP32)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    rc = lib.nnqs_create(ctypes.byref(d), ctypes.byref(h))
    assert rc == code
    assert h.value is None
    assert len(lib.nnqs_last_error()) > 0


def test_odd_inversion_without_bias_rejected(lib):
    from paper_2206_14307_gb300 import nnqs
    d = nnqs.nnqs_desc(4, 1.0, 0.5, 1, 16, 1, 1, 0, 0, -1, 0, nnqs.FP32)
    h = ctypes.c_void_p()
    assert lib.nnqs_create(ctypes.byref(d), ctypes.byref(h)) == nnqs.NNQS_EINVAL
    assert b"vanishes" in lib.nnqs_last_error()


def test_null_model_is_einval(lib):
    assert lib.nnqs_log_psi(None, None, 1, None, None) == -1
    assert lib.nnqs_num_params(None) == -1


def test_tile_shape_table(lib):
    from paper_2206_14307_gb300 import nnqs
    n = lib.nnqs_num_tile_shapes()
    assert n == 16
    widths = []
    for v in range(n):
        gl, mpl = nnqs.nnqs_tile_shape(v)
        assert gl in (8, 16, 32) and 1 <= mpl <= 16
        widths.append(gl * mpl)
    assert widths == sorted(widths) and widths[0] == 16 and widths[-1] == 512
    with pytest.raises(nnqs.NNQSError):
        nnqs.nnqs_tile_shape(n)


def test_batch_arguments_rejected_on_host(lib):
    from paper_2206_14307_gb300 import nnqs
    ok = nnqs.nnqs_desc(4, 1.0, 0.5, 1, 16, 0, 0, 0, 0, 0, 1, nnqs.FP32)
    f64 = nnqs.nnqs_desc(4, 1.0, 0.5, 1, 16, 0, 0, 0, 0, 0, 1, nnqs.FP64)
    arr = (nnqs.nnqs_desc * 2)(ok, f64)
    h = ctypes.c_void_p()
    assert lib.nnqs_batch_create(ctypes.cast(arr, ctypes.c_void_p), 2, ctypes.byref(h)) == nnqs.NNQS_EUNSUPPORTED
    assert h.value is None
    assert lib.nnqs_batch_create(ctypes.cast(arr, ctypes.c_void_p), 0, ctypes.byref(h)) == nnqs.NNQS_EINVAL
    assert lib.nnqs_batch_create(None, 1, ctypes.byref(h)) == nnqs.NNQS_EINVAL
    assert lib.nnqs_batch_size(None) == -1
    assert lib.nnqs_batch_get_shape(None, 0) == -1
    assert lib.nnqs_batch_model(None, 0) is None
    assert lib.nnqs_batch_lanczos(None, None, None, None, None, None, None, None) == nnqs.NNQS_EINVAL
    assert lib.nnqs_batch_autotune(None, None, None, 1, None, None, None) == nnqs.NNQS_EINVAL
    assert lib.nnqs_batch_destroy(None) == nnqs.NNQS_OK
