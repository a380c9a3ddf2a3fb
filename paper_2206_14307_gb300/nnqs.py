"""Thin Python binding of the C ABI in include/nnqs.h (argument marshalling only).

Every step of the computation runs in the CUDA library ``libnnqs_gb300.so``;
PyTorch only provides device memory and streams.  Importing this module on a
machine without the built library raises immediately -- there is no fallback.

Functions with the ABI's names (``nnqs_create``, ``nnqs_log_psi``, ...) take
raw pointers as Python ints; the ``Model`` class wraps them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnnqs_gb300.so")

NNQS_OK, NNQS_EINVAL, NNQS_ENOMEM, NNQS_ECUDA, NNQS_ETIMEOUT, NNQS_EUNSUPPORTED, NNQS_ERANGE = 0, -1, -2, -3, -4, -5, -6
FP64, FP32, BF16X2, BF16X3 = 0, 1, 2, 3
A1, A2, B1, B2 = 0, 1, 2, 3
K00, KPIPI, KPI0, K0PI = 0, 1, 2, 3

# exported symbols of include/nnqs.h
ABI_FUNCTIONS = (
    "nnqs_create", "nnqs_destroy", "nnqs_num_params", "nnqs_group_size", "nnqs_set_params",
    "nnqs_set_params_device", "nnqs_sample", "nnqs_log_psi", "nnqs_local_energy",
    "nnqs_lanczos_moments", "nnqs_grad_logpsi", "nnqs_energy_grad", "nnqs_sr_matvec",
    "nnqs_status", "nnqs_last_error", "nnqs_lanczos_moments_noalloc", "nnqs_sr_solve",
    "nnqs_num_tile_shapes", "nnqs_tile_shape", "nnqs_batch_create", "nnqs_batch_destroy", "nnqs_batch_size",
    "nnqs_batch_model", "nnqs_batch_get_shape", "nnqs_batch_set_shape", "nnqs_batch_autotune",
    "nnqs_batch_lanczos", "nnqs_batch_status", "nnqs_lanczos_variance", "nnqs_structure_factor",
    "nnqs_lanczos2", "nnqs_lanczos_partial", "nnqs_lanczos_finish",
)
NOALLOC_MAX_SAMPLES = 65536


class nnqs_desc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("J1", ctypes.c_double), ("J2", ctypes.c_double),
                ("K", ctypes.c_int32), ("M", ctypes.c_int32),
                ("project_translations", ctypes.c_int32), ("project_point_group", ctypes.c_int32),
                ("momentum", ctypes.c_int32), ("irrep", ctypes.c_int32),
                ("spin_inversion", ctypes.c_int32), ("use_bias", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("check_inputs", ctypes.c_int32)]


class NNQSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nnqs error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2206_14307_gb300.build.build() "
                              "(no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "nnqs_create": ([ctypes.POINTER(nnqs_desc), ctypes.POINTER(P)], ctypes.c_int),
            "nnqs_destroy": ([P], ctypes.c_int),
            "nnqs_num_params": ([P], i64),
            "nnqs_group_size": ([P], i32),
            "nnqs_set_params": ([P, P, i64, P], ctypes.c_int),
            "nnqs_set_params_device": ([P, P, i64, P], ctypes.c_int),
            "nnqs_sample": ([P, u64, i32, i32, i32, i32, P, P, P], ctypes.c_int),
            "nnqs_log_psi": ([P, P, i64, P, P], ctypes.c_int),
            "nnqs_local_energy": ([P, P, i64, P, P, P], ctypes.c_int),
            "nnqs_lanczos_moments": ([P, P, i64, P, P, P, P, P], ctypes.c_int),
            "nnqs_grad_logpsi": ([P, P, i64, P, P], ctypes.c_int),
            "nnqs_energy_grad": ([P, P, P, P, i64, P, P], ctypes.c_int),
            "nnqs_sr_matvec": ([P, P, P, i64, P, d, P, P], ctypes.c_int),
            "nnqs_sr_solve": ([P, P, P, i64, P, d, d, i32, d, P, P, P, P], ctypes.c_int),
            "nnqs_status": ([P, P], ctypes.c_int),
            "nnqs_lanczos_moments_noalloc": ([P, P, i64, P, P, P], ctypes.c_int),
            "nnqs_last_error": ([], ctypes.c_char_p),
            "nnqs_lanczos_variance": ([P, P, P, P], ctypes.c_int),
            "nnqs_lanczos2": ([P, P, i64, P, P, P, P], ctypes.c_int),
            "nnqs_lanczos_partial": ([P, P, i64, P, P, P, P], ctypes.c_int),
            "nnqs_lanczos_finish": ([P, P, P, P], ctypes.c_int),
            "nnqs_structure_factor": ([P, P, i64, P, P, P], ctypes.c_int),
            "nnqs_num_tile_shapes": ([], i32),
            "nnqs_tile_shape": ([i32, P, P], ctypes.c_int),
            "nnqs_batch_create": ([P, i32, ctypes.POINTER(P)], ctypes.c_int),
            "nnqs_batch_destroy": ([P], ctypes.c_int),
            "nnqs_batch_size": ([P], i32),
            "nnqs_batch_model": ([P, i32], P),
            "nnqs_batch_get_shape": ([P, i32], i32),
            "nnqs_batch_set_shape": ([P, i32, i32], ctypes.c_int),
            "nnqs_batch_autotune": ([P, P, P, i32, P, P, P], ctypes.c_int),
            "nnqs_batch_lanczos": ([P, P, P, P, P, P, P, P], ctypes.c_int),
            "nnqs_batch_status": ([P, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != NNQS_OK:
        raise NNQSError(rc, lib().nnqs_last_error().decode())
    return rc


# ---- raw ABI (same names; pointers are Python ints) -------------------------------------------
def nnqs_create(desc: nnqs_desc) -> int:
    h = ctypes.c_void_p()
    _check(lib().nnqs_create(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def nnqs_destroy(h): return _check(lib().nnqs_destroy(h))
def nnqs_num_params(h): return lib().nnqs_num_params(h)
def nnqs_group_size(h): return lib().nnqs_group_size(h)
def nnqs_set_params(h, params_host_ptr, P, stream=0): return _check(lib().nnqs_set_params(h, params_host_ptr, P, stream))
def nnqs_set_params_device(h, params_ptr, P, stream=0): return _check(lib().nnqs_set_params_device(h, params_ptr, P, stream))


def nnqs_sample(h, seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out, acc_out, stream=0):
    return _check(lib().nnqs_sample(h, seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out, acc_out, stream))


def nnqs_log_psi(h, cfg, n, out, stream=0): return _check(lib().nnqs_log_psi(h, cfg, n, out, stream))
def nnqs_local_energy(h, cfg, n, eloc, sums, stream=0): return _check(lib().nnqs_local_energy(h, cfg, n, eloc, sums, stream))


def nnqs_lanczos_moments(h, cfg, n, h1, h2, moments, lanczos, stream=0):
    return _check(lib().nnqs_lanczos_moments(h, cfg, n, h1, h2, moments, lanczos, stream))


def nnqs_grad_logpsi(h, cfg, n, O, stream=0): return _check(lib().nnqs_grad_logpsi(h, cfg, n, O, stream))
def nnqs_energy_grad(h, O, eloc, weights, n, F, stream=0):
    return _check(lib().nnqs_energy_grad(h, O, eloc, weights, n, F, stream))


def nnqs_sr_matvec(h, O, weights, n, x, lam, y, stream=0):
    return _check(lib().nnqs_sr_matvec(h, O, weights, n, x, lam, y, stream))


def nnqs_sr_solve(h, O, weights, n, F, lam, dtau, max_iter, tol, delta, info, params_inout, stream=0):
    return _check(lib().nnqs_sr_solve(h, O, weights, n, F, lam, dtau, max_iter, tol, delta, info, params_inout,
                                      stream))
def nnqs_status(h, stream=0): return _check(lib().nnqs_status(h, stream))


def nnqs_lanczos_moments_noalloc(h, cfg, n, moments, lanczos, stream=0):
    return _check(lib().nnqs_lanczos_moments_noalloc(h, cfg, n, moments, lanczos, stream))


def nnqs_lanczos2(h, cfg, n, h3, mu, out, stream=0):
    return _check(lib().nnqs_lanczos2(h, cfg, n, h3, mu, out, stream))


def nnqs_lanczos_partial(h, cfg, n, h1, h2, sums, stream=0):
    return _check(lib().nnqs_lanczos_partial(h, cfg, n, h1, h2, sums, stream))


def nnqs_lanczos_finish(sums, moments, lanczos, stream=0):
    return _check(lib().nnqs_lanczos_finish(sums, moments, lanczos, stream))


def nnqs_lanczos_variance(moments, lanczos, out, stream=0):
    return _check(lib().nnqs_lanczos_variance(moments, lanczos, out, stream))


def nnqs_structure_factor(h, cfg, n, weights, sq_out, stream=0):
    return _check(lib().nnqs_structure_factor(h, cfg, n, weights, sq_out, stream))


def nnqs_num_tile_shapes(): return lib().nnqs_num_tile_shapes()


def nnqs_tile_shape(v):
    gl, mpl = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().nnqs_tile_shape(v, ctypes.byref(gl), ctypes.byref(mpl)))
    return gl.value, mpl.value


def nnqs_batch_create(descs) -> int:
    arr = (nnqs_desc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(lib().nnqs_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(descs), ctypes.byref(h)))
    return h.value


def nnqs_batch_destroy(b): return _check(lib().nnqs_batch_destroy(b))
def nnqs_batch_size(b): return lib().nnqs_batch_size(b)


def nnqs_batch_model(b, i):
    h = lib().nnqs_batch_model(b, i)
    if not h:
        raise NNQSError(NNQS_EINVAL, lib().nnqs_last_error().decode())
    return h


def nnqs_batch_get_shape(b, i): return lib().nnqs_batch_get_shape(b, i)
def nnqs_batch_set_shape(b, i, v): return _check(lib().nnqs_batch_set_shape(b, i, v))


def nnqs_batch_autotune(b, cfg, n_per_model_host, probe, shape_out_host, ms_out_host, stream=0):
    return _check(lib().nnqs_batch_autotune(b, cfg, n_per_model_host, probe, shape_out_host, ms_out_host, stream))


def nnqs_batch_lanczos(b, cfg, n_per_model_host, h1, h2, moments, lanczos, stream=0):
    return _check(lib().nnqs_batch_lanczos(b, cfg, n_per_model_host, h1, h2, moments, lanczos, stream))


def nnqs_batch_status(b, stream=0): return _check(lib().nnqs_batch_status(b, stream))


# ---- torch convenience wrapper ---------------------------------------------------------------
def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Model:
    """A model on the current CUDA device.  Tensors are torch CUDA tensors:
    configurations int64 [n][ceil(N/64)] (the bits of the uint64 words),
    complex results float64 [n][2]."""

    def __init__(self, L, J1=1.0, J2=0.5, K=1, M=None, proj_t=False, proj_p=False, momentum=K00, irrep=A1,
                 spin_inv=0, use_bias=True, precision=FP32, check_inputs=False):
        self.L, self.N = L, L * L
        self.M = M if M is not None else self.N
        self.K = K
        self.desc = nnqs_desc(L, J1, J2, K, self.M, int(proj_t), int(proj_p), momentum, irrep,
                              spin_inv, int(use_bias), precision, int(check_inputs))
        self.h = nnqs_create(self.desc)
        self.P = nnqs_num_params(self.h)
        self.G = nnqs_group_size(self.h)
        self.nwords = (self.N + 63) // 64

    def close(self):
        if getattr(self, "h", None):
            nnqs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        """params: complex numpy array (host) or float64 CUDA tensor [P][2]."""
        import torch
        if isinstance(params, torch.Tensor):
            assert params.is_cuda and params.dtype == torch.float64
            nnqs_set_params_device(self.h, params.data_ptr(), self.P, _stream())
        else:
            p = np.asarray(params, np.complex128).reshape(-1)
            buf = np.ascontiguousarray(np.stack([p.real, p.imag], -1))
            nnqs_set_params(self.h, buf.ctypes.data, self.P, _stream())

    def _out(self, *shape):
        import torch
        return torch.empty(*shape, dtype=torch.float64, device="cuda")

    def log_psi(self, cfg, out=None):
        n = cfg.shape[0]
        out = self._out(n, 2) if out is None else out
        nnqs_log_psi(self.h, cfg.data_ptr(), n, out.data_ptr(), _stream())
        return out

    def local_energy(self, cfg, out=None, sums=None):
        n = cfg.shape[0]
        out = self._out(n, 2) if out is None else out
        nnqs_local_energy(self.h, cfg.data_ptr(), n, out.data_ptr(), _ptr(sums), _stream())
        return out

    def lanczos(self, cfg, h1=None, h2=None, moments=None, lanczos=None):
        n = cfg.shape[0]
        h1 = self._out(n, 2) if h1 is None else h1
        h2 = self._out(n, 2) if h2 is None else h2
        moments = self._out(8) if moments is None else moments
        lanczos = self._out(3) if lanczos is None else lanczos
        nnqs_lanczos_moments(self.h, cfg.data_ptr(), n, h1.data_ptr(), h2.data_ptr(), moments.data_ptr(),
                             lanczos.data_ptr(), _stream())
        return h1, h2, moments, lanczos

    def lanczos_partial(self, cfg, h1=None, h2=None, sums=None):
        """This process's h1, h2 and raw FP64 sums [7] (see lanczos_finish)."""
        n = cfg.shape[0]
        sums = self._out(7) if sums is None else sums
        nnqs_lanczos_partial(self.h, cfg.data_ptr() if n else None, n, _ptr(h1), _ptr(h2), sums.data_ptr(),
                             _stream())
        return h1, h2, sums

    def sample(self, seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out=None, acc_out=None):
        import torch
        if cfg_out is None:
            cfg_out = torch.empty(n_chains * n_per_chain, self.nwords, dtype=torch.int64, device="cuda")
        if acc_out is None:
            acc_out = torch.empty(n_chains, dtype=torch.float32, device="cuda")
        nnqs_sample(self.h, seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out.data_ptr(), acc_out.data_ptr(),
                    _stream())
        return cfg_out, acc_out

    def grad_logpsi(self, cfg, out=None):
        n = cfg.shape[0]
        out = self._out(n, self.P, 2) if out is None else out
        nnqs_grad_logpsi(self.h, cfg.data_ptr(), n, out.data_ptr(), _stream())
        return out

    def energy_grad(self, O, eloc, out=None, weights=None):
        n = O.shape[0]
        out = self._out(self.P, 2) if out is None else out
        nnqs_energy_grad(self.h, O.data_ptr(), eloc.data_ptr(), _ptr(weights), n, out.data_ptr(), _stream())
        return out

    def sr_matvec(self, O, x, lam, out=None, weights=None):
        n = O.shape[0]
        out = self._out(self.P, 2) if out is None else out
        nnqs_sr_matvec(self.h, O.data_ptr(), _ptr(weights), n, x.data_ptr(), float(lam), out.data_ptr(), _stream())
        return out

    def sr_solve(self, O, F, lam=1e-6, dtau=1.0, max_iter=200, tol=1e-10, weights=None, params_inout=None):
        """CG solution of (S + lam) delta = -dtau F; returns (delta, info)."""
        n = O.shape[0]
        delta = self._out(self.P, 2)
        info = self._out(2)
        nnqs_sr_solve(self.h, O.data_ptr(), _ptr(weights), n, F.data_ptr(), float(lam), float(dtau), int(max_iter),
                      float(tol), delta.data_ptr(), info.data_ptr(), _ptr(params_inout), _stream())
        return delta, info

    def lanczos2(self, cfg, h3=None, mu=None, out=None):
        """p = 2 step: (h3 [n][2], mu [8] = mu_0..mu_6 and c, out [5] = E_p2, x0..x2, var_p2)."""
        n = cfg.shape[0]
        h3 = self._out(n, 2) if h3 is None else h3
        mu = self._out(8) if mu is None else mu
        out = self._out(5) if out is None else out
        nnqs_lanczos2(self.h, cfg.data_ptr(), n, h3.data_ptr(), mu.data_ptr(), out.data_ptr(), _stream())
        return h3, mu, out

    def structure_factor(self, cfg, weights=None, out=None):
        """S(q) [N] for q = 2 pi (qx, qy)/L at index qx + L qy."""
        out = self._out(self.N) if out is None else out
        nnqs_structure_factor(self.h, cfg.data_ptr(), cfg.shape[0], _ptr(weights), out.data_ptr(), _stream())
        return out

    def status(self):
        return nnqs_status(self.h, _stream())


def lanczos_finish(sums, moments=None, lanczos=None):
    """Moments [8] and the p = 1 step [3] from raw sums [7] summed over processes."""
    import torch
    moments = torch.empty(8, dtype=torch.float64, device=sums.device) if moments is None else moments
    lanczos = torch.empty(3, dtype=torch.float64, device=sums.device) if lanczos is None else lanczos
    nnqs_lanczos_finish(sums.data_ptr(), moments.data_ptr(), lanczos.data_ptr(), _stream())
    return moments, lanczos


def allreduce_sums(sums, group=None):
    """Element-wise sum of a raw-sum tensor over the processes of a
    torch.distributed group (in place; a no-op without an initialised group
    of more than one process).  This is the one exchange step of the
    distributed Lanczos step: 7 doubles per process."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums


def lanczos_distributed(model, cfg, h1=None, h2=None, group=None):
    """One Lanczos step over the union of every process's samples: the
    partial sums of this process's cfg, their all-reduce, the closed form.
    Returns (sums, moments, lanczos) on this process's device."""
    _, _, sums = model.lanczos_partial(cfg, h1, h2)
    allreduce_sums(sums, group)
    moments, lanczos = lanczos_finish(sums)
    return sums, moments, lanczos


def lanczos_variance(moments, lanczos, out=None):
    """{var0, E1, var1, E_extrap} on the device from the [8] moments and [3] step."""
    import torch
    out = torch.empty(4, dtype=torch.float64, device="cuda") if out is None else out
    nnqs_lanczos_variance(moments.data_ptr(), lanczos.data_ptr(), out.data_ptr(), _stream())
    return out


def cfg_tensor(words: np.ndarray):
    """uint64 numpy words -> int64 CUDA tensor with the same bits."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(words).view(np.int64)).cuda()


class _Borrowed(Model):
    """Model view of a batch instance (owned by the batch)."""

    def __init__(self, h, desc):
        self.h = h
        self.desc = desc
        self.L, self.N, self.M, self.K = desc.L, desc.L * desc.L, desc.M, desc.K
        self.P = nnqs_num_params(h)
        self.G = nnqs_group_size(h)
        self.nwords = (self.N + 63) // 64

    def close(self):
        self.h = None


class Batch:
    """Instances of uneven size run in one persistent, graph-captured launch.
    ``specs`` are dicts of Model's keyword arguments (L, J1, J2, K, M, proj_t,
    proj_p, momentum, irrep, spin_inv, use_bias, precision)."""

    def __init__(self, specs):
        descs = []
        for sp in specs:
            L = sp["L"]
            M = sp.get("M") or L * L
            descs.append(nnqs_desc(L, sp.get("J1", 1.0), sp.get("J2", 0.5), sp.get("K", 1), M,
                                   int(sp.get("proj_t", False)), int(sp.get("proj_p", False)),
                                   sp.get("momentum", K00), sp.get("irrep", A1), sp.get("spin_inv", 0),
                                   int(sp.get("use_bias", True)), sp.get("precision", FP32),
                                   int(sp.get("check_inputs", False))))
        self.h = nnqs_batch_create(descs)
        self.models = [_Borrowed(nnqs_batch_model(self.h, i), d) for i, d in enumerate(descs)]

    def __len__(self):
        return len(self.models)

    def close(self):
        if getattr(self, "h", None):
            for m in self.models:
                m.h = None
            nnqs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _counts(counts):
        return np.ascontiguousarray(np.asarray(counts, np.int64))

    def shape(self, i):
        return nnqs_batch_get_shape(self.h, i)

    def set_shape(self, i, v):
        nnqs_batch_set_shape(self.h, i, v)

    def autotune(self, cfg, counts, probe=64):
        """cfg: int64 CUDA tensor holding every instance's words back to back."""
        n = self._counts(counts)
        shapes = np.zeros(len(self), np.int32)
        ms = np.zeros(len(self), np.float64)
        nnqs_batch_autotune(self.h, cfg.data_ptr(), n.ctypes.data, probe, shapes.ctypes.data, ms.ctypes.data,
                            _stream())
        return shapes, ms

    def lanczos(self, cfg, counts, h1=None, h2=None, moments=None, lanczos=None):
        import torch
        n = self._counts(counts)
        tot = int(n.sum())
        h1 = torch.empty(tot, 2, dtype=torch.float64, device="cuda") if h1 is None else h1
        h2 = torch.empty(tot, 2, dtype=torch.float64, device="cuda") if h2 is None else h2
        moments = torch.empty(len(self), 8, dtype=torch.float64, device="cuda") if moments is None else moments
        lanczos = torch.empty(len(self), 3, dtype=torch.float64, device="cuda") if lanczos is None else lanczos
        nnqs_batch_lanczos(self.h, cfg.data_ptr() if tot else None, n.ctypes.data, h1.data_ptr(), h2.data_ptr(),
                           moments.data_ptr(), lanczos.data_ptr(), _stream())
        return h1, h2, moments, lanczos

    def status(self):
        return nnqs_batch_status(self.h, _stream())
