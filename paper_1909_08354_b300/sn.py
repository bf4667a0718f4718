"""ctypes binding of libsn (include/sn.h), argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
to it; the numerical work happens in the CUDA library.  Arrays may be numpy
arrays or CPU torch tensors (host memory, pinned or not) or CUDA torch tensors
(device memory).  Loading fails loudly if libsn.so has not been built.
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SN_LIB_PATH") or os.path.join(_HERE, "libsn.so")

SN_OK, SN_EINVAL, SN_ENOMEM, SN_ECUDA, SN_ETIMEOUT, SN_ENONFINITE, SN_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
SN_ENGINE_FP32, SN_ENGINE_TC16, SN_ENGINE_UMMA = 0, 1, 2
SN_STAGING_TMA, SN_STAGING_REGISTERS, SN_STAGING_RESIDENT = 0, 1, 2
SN_OBS_FP64, SN_OBS_FP32 = 0, 1
SN_BATCH_PERSISTENT, SN_BATCH_GRAPH, SN_BATCH_CLASSES = 0, 1, 2
SN_FNO_LAYER_GEMMS, SN_FNO_LAYER_UMMA = 0, 1
SN_FLOOR_MAX, SN_FLOOR_SMOOTH = 0, 1
SN_C64, SN_C128 = 0, 1
SN_KERNEL_NMC, SN_KERNEL_POISSON = 0, 1
_STATUS = {0: "SN_OK", -1: "SN_EINVAL", -2: "SN_ENOMEM", -3: "SN_ECUDA", -4: "SN_ETIMEOUT",
           -5: "SN_ENONFINITE", -6: "SN_ENOTSUP"}


class SnKernel(ctypes.Structure):
    _fields_ = [("coeff_lap", ctypes.c_double), ("G", ctypes.c_double),
                ("alpha_Y", ctypes.c_double), ("lambda_Y", ctypes.c_double),
                ("g_local", ctypes.c_double), ("zero_k0", ctypes.c_int),
                ("v_ext", ctypes.c_void_p), ("v_ext_on_device", ctypes.c_int),
                ("kind", ctypes.c_int), ("B", ctypes.c_double), ("C", ctypes.c_double),
                ("D", ctypes.c_double)]


def _kernel(coeff_lap=-0.5, G=1.0, alpha_Y=0.0, lambda_Y=1.0, g_local=0.0, zero_k0=1,
            kind=SN_KERNEL_NMC, B=1.0, C=0.0, D=0.0) -> SnKernel:
    """An sn_kernel without V_ext: SN_KERNEL_NMC uses G, alpha_Y, lambda_Y;
    SN_KERNEL_POISSON uses B, C, D (see sn_kernel in include/sn.h)."""
    return SnKernel(float(coeff_lap), float(G), float(alpha_Y), float(lambda_Y), float(g_local),
                    int(zero_k0), None, 0, int(kind), float(B), float(C), float(D))


SN_GRAVITY_GR, SN_GRAVITY_NMC = 0, 1
SN_MAX_FIELDS = 16  # include/sn.h
SN_SCHED_KINDS, SN_SCHED_MAX_CTAS = 6, 64  # include/sn.h
SN_SCHED_VALUES = 6 * SN_SCHED_KINDS  # CTAs per SM, then the staging, of each kind and axis


class SnFluid(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("w", ctypes.c_double), ("n_poly", ctypes.c_double),
                ("model", ctypes.c_int), ("lambda_", ctypes.c_double), ("M", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("floor_mode", ctypes.c_int)]


class SnObs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("e_kin", ctypes.c_double),
                ("e_pot", ctypes.c_double), ("e_nl", ctypes.c_double),
                ("e_total", ctypes.c_double), ("centroid", ctypes.c_double * 3),
                ("momentum", ctypes.c_double * 3), ("step", ctypes.c_longlong)]


class SNError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None

# (name, restype, argtypes) of every entry point declared in include/sn.h
_SIGNATURES = [
    ("sn_create_grid", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_int, ctypes.c_void_p]),
    ("sn_set_kernel", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SnKernel)]),
    ("sn_set_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("sn_get_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("sn_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]),
    ("sn_observables", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SnObs)]),
    ("sn_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("sn_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("sn_profile_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("sn_kind_name", ctypes.c_char_p, [ctypes.c_int]),
    ("sn_set_engine", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sn_set_staging", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sn_set_blocking", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sn_set_obs_mode", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sn_set_fluid", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SnFluid)]),
    ("sn_set_fields", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sn_get_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("sn_set_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("sn_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]),
    ("sn_get_fields", ctypes.c_int, [ctypes.c_void_p]),
    ("sn_test_line_fft_f32", ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("sn_test_dsmem_rates", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("sn_test_line_fft_engines", ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("sn_test_umma_phases", ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong), ctypes.c_void_p]),
    ("sn_step_2d_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(SnKernel), ctypes.c_double, ctypes.c_int,
                                          ctypes.c_void_p]),
    ("sn_create_batch", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_void_p]),
    ("sn_set_kernel_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SnKernel)]),
    ("sn_set_state_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int]),
    ("sn_get_state_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int]),
    ("sn_step_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("sn_observables_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(SnObs)]),
    ("sn_batch_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("sn_set_batch_wait_limit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    ("sn_set_batch_ctas", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sn_set_batch_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sn_get_batch_schedule", ctypes.c_int, [ctypes.c_void_p]),
    ("sn_autotune_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("sn_batch_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("sn_destroy_batch", None, [ctypes.c_void_p]),
    ("sn_fno_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_void_p]),
    ("sn_fno_param_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("sn_fno_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("sn_fno_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("sn_fno_get_grads", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("sn_fno_set_grads", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("sn_fno_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("sn_fno_loss", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double)]),
    ("sn_fno_backward", ctypes.c_int, [ctypes.c_void_p]),
    ("sn_fno_adam", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int]),
    ("sn_fno_set_layer_form", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sn_fno_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("sn_fno_destroy", None, [ctypes.c_void_p]),
    ("sn_fno_pack", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p]),
    ("sn_fno_unpack", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_longlong, ctypes.c_void_p]),
    ("sn_fno_pack2", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                                    ctypes.c_void_p]),
    ("sn_mass_c64", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    ("sn_test_gemm_bf16", ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_longlong] * 3
                                        + [ctypes.c_void_p] + [ctypes.c_longlong] * 3
                                        + [ctypes.c_void_p] + [ctypes.c_longlong] * 3
                                        + [ctypes.c_int] * 4 + [ctypes.c_float] * 2),
    ("sn_destroy_grid", None, [ctypes.c_void_p]),
    ("sn_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
]


def lib() -> ctypes.CDLL:
    """Load libsn.so once; raise if it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -m paper_1909_08354_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(g, status: int):
    if status != SN_OK:
        msg = lib().sn_last_error(g).decode(errors="replace")
        raise SNError(status, msg)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _array_ptr(x, dtype: int, count: int, writable: bool = False):
    """(pointer, on_device, keepalive) for a psi buffer of `count` complex values."""
    want = np.complex64 if dtype == SN_C64 else np.complex128
    if _is_torch(x):
        import torch
        tdt = torch.complex64 if dtype == SN_C64 else torch.complex128
        if x.dtype != tdt or not x.is_contiguous() or x.numel() != count:
            raise ValueError(f"expected a contiguous {tdt} tensor of {count} elements")
        return x.data_ptr(), 1 if x.is_cuda else 0, x
    a = x if writable else np.ascontiguousarray(x, dtype=want)
    if a.dtype != want or not a.flags["C_CONTIGUOUS"] or a.size != count:
        raise ValueError(f"expected a C-contiguous {np.dtype(want)} array of {count} elements")
    return a.ctypes.data, 0, a


# ----------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ----------------------------------------------------------------------------

def sn_create_grid(n: Sequence[int], L: Sequence[float], dtype: int = SN_C64, stream=None):
    """Create a grid; returns the opaque handle (an int).  `stream` is a
    cudaStream_t as an int (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    nd = len(n)
    h = ctypes.c_void_p()
    na = (ctypes.c_int * nd)(*[int(v) for v in n])
    La = (ctypes.c_double * nd)(*[float(v) for v in L])
    st = lib().sn_create_grid(ctypes.byref(h), nd, na, La, int(dtype),
                              ctypes.c_void_p(stream) if stream else None)
    _check(None, st)
    return h.value


def sn_set_kernel(g, coeff_lap=-0.5, G=1.0, alpha_Y=0.0, lambda_Y=1.0, g_local=0.0,
                  v_ext=None, zero_k0=1, kind=SN_KERNEL_NMC, B=1.0, C=0.0, D=0.0):
    keep = None
    k = _kernel(coeff_lap, G, alpha_Y, lambda_Y, g_local, zero_k0, kind, B, C, D)
    if v_ext is not None:
        if _is_torch(v_ext):
            import torch
            keep = v_ext.to(torch.float64).contiguous()
            k.v_ext = keep.data_ptr()
            k.v_ext_on_device = 1 if keep.is_cuda else 0
        else:
            keep = np.ascontiguousarray(v_ext, dtype=np.float64)
            k.v_ext = keep.ctypes.data
    _check(g, lib().sn_set_kernel(g, ctypes.byref(k)))
    del keep


def sn_set_state(g, psi, dtype: int, count: int):
    p, dev, keep = _array_ptr(psi, dtype, count)
    _check(g, lib().sn_set_state(g, p, dev))
    del keep


def sn_get_state(g, out, dtype: int, count: int):
    p, dev, keep = _array_ptr(out, dtype, count, writable=True)
    _check(g, lib().sn_get_state(g, p, dev))
    return out


def sn_step(g, dt: float, nsteps: int):
    _check(g, lib().sn_step(g, float(dt), int(nsteps)))


def sn_observables(g) -> dict:
    o = SnObs()
    _check(g, lib().sn_observables(g, ctypes.byref(o)))
    return dict(mass=o.mass, e_kin=o.e_kin, e_pot=o.e_pot, e_nl=o.e_nl, e_total=o.e_total,
                centroid=list(o.centroid), momentum=list(o.momentum), step=o.step)


def sn_sync(g):
    _check(g, lib().sn_sync(g))


def sn_launch_count(g) -> int:
    return int(lib().sn_launch_count(g))


def sn_kind_names():
    names = []
    while True:
        s = lib().sn_kind_name(len(names))
        if s is None:
            return names
        names.append(s.decode())


def sn_profile_step(g, dt: float, nsteps: int) -> dict:
    names = sn_kind_names()
    k = len(names)
    ms = (ctypes.c_double * k)()
    ln = (ctypes.c_longlong * k)()
    by = (ctypes.c_double * k)()
    _check(g, lib().sn_profile_step(g, float(dt), int(nsteps), ms, ln, by, k))
    return {names[i]: dict(ms=ms[i], launches=int(ln[i]), bytes=by[i]) for i in range(k)}


def sn_step_2d_noalloc(psi, L, dt: float, nsteps: int, coeff_lap=-0.5, G=1.0, alpha_Y=0.0,
                       lambda_Y=1.0, g_local=0.0, stream=None, kind=SN_KERNEL_NMC, B=1.0, C=0.0,
                       D=0.0):
    """In-place steps of a 2D complex64 CUDA tensor psi (ny, nx) without device
    allocation (see sn_step_2d_noalloc in include/sn.h)."""
    import torch
    if not (_is_torch(psi) and psi.is_cuda and psi.dtype == torch.complex64 and psi.dim() == 2
            and psi.is_contiguous()):
        raise ValueError("psi must be a contiguous 2D complex64 CUDA tensor")
    k = _kernel(coeff_lap, G, alpha_Y, lambda_Y, g_local, 1, kind, B, C, D)
    st = lib().sn_step_2d_noalloc(psi.data_ptr(), psi.shape[0], psi.shape[1], float(L[0]),
                                  float(L[1]), ctypes.byref(k), float(dt), int(nsteps),
                                  ctypes.c_void_p(stream) if stream else None)
    _check(None, st)


def sn_destroy_grid(g):
    if g:
        lib().sn_destroy_grid(g)


def sn_last_error(g=None) -> str:
    return lib().sn_last_error(g).decode(errors="replace")


def _obs_dict(o):
    return dict(mass=o.mass, e_kin=o.e_kin, e_pot=o.e_pot, e_nl=o.e_nl, e_total=o.e_total,
                centroid=list(o.centroid), momentum=list(o.momentum), step=o.step)


def sn_create_batch(n: Sequence[int], L: Sequence[float], stream=None):
    c = len(n)
    h = ctypes.c_void_p()
    st = lib().sn_create_batch(ctypes.byref(h), c, (ctypes.c_int * c)(*[int(v) for v in n]),
                               (ctypes.c_double * c)(*[float(v) for v in L]),
                               ctypes.c_void_p(stream) if stream else None)
    _check(None, st)
    return h.value


def sn_set_kernel_batch(b, kernels):
    """kernels: sequence of dicts with the keyword arguments of sn_set_kernel."""
    arr = (SnKernel * len(kernels))()
    for i, kw in enumerate(kernels):
        arr[i] = _kernel(kw.get("coeff_lap", -0.5), kw.get("G", 1.0), kw.get("alpha_Y", 0.0),
                         kw.get("lambda_Y", 1.0), kw.get("g_local", 0.0), 1,
                         kw.get("kind", SN_KERNEL_NMC), kw.get("B", 1.0), kw.get("C", 0.0),
                         kw.get("D", 0.0))
    _check(None, lib().sn_set_kernel_batch(b, arr))


def sn_set_state_batch(b, index: int, psi, count: int):
    p, dev, keep = _array_ptr(psi, SN_C64, count)
    _check(None, lib().sn_set_state_batch(b, int(index), p, dev))
    del keep


def sn_get_state_batch(b, index: int, out, count: int):
    p, dev, keep = _array_ptr(out, SN_C64, count, writable=True)
    _check(None, lib().sn_get_state_batch(b, int(index), p, dev))
    return out


def sn_step_batch(b, dt, nsteps: int):
    arr = (ctypes.c_double * len(dt))(*[float(v) for v in dt])
    _check(None, lib().sn_step_batch(b, arr, int(nsteps)))


def sn_observables_batch(b, index: int) -> dict:
    o = SnObs()
    _check(None, lib().sn_observables_batch(b, int(index), ctypes.byref(o)))
    return _obs_dict(o)


def sn_batch_sync(b):
    _check(None, lib().sn_batch_sync(b))


def sn_set_batch_wait_limit(b, cycles: int):
    _check(None, lib().sn_set_batch_wait_limit(b, int(cycles)))


def sn_set_batch_ctas(b, per_sm: int):
    _check(None, lib().sn_set_batch_ctas(b, int(per_sm)))


def sn_set_batch_schedule(b, schedule: int):
    _check(None, lib().sn_set_batch_schedule(b, int(schedule)))


def sn_get_batch_schedule(b) -> int:
    return int(lib().sn_get_batch_schedule(b))


def sn_batch_launch_count(b) -> int:
    return int(lib().sn_batch_launch_count(b))


def sn_destroy_batch(b):
    if b:
        lib().sn_destroy_batch(b)


class Fno:
    """Owns one sn_fno handle (the surrogate network); arrays are CUDA torch tensors."""

    def __init__(self, s=256, c_in=5, width=64, modes=24, layers=4, proj=128, batch_max=8,
                 stream=None):
        self.s, self.c_in, self.width, self.modes, self.layers, self.proj = s, c_in, width, modes, layers, proj
        self.batch_max = batch_max
        h = ctypes.c_void_p()
        _check(None, lib().sn_fno_create(ctypes.byref(h), s, c_in, width, modes, layers, proj,
                                         batch_max, ctypes.c_void_p(stream) if stream else None))
        self.h = h.value
        self.nparams = int(lib().sn_fno_param_count(self.h))

    @staticmethod
    def _dev(t, n):
        import torch
        if not (_is_torch(t) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and t.numel() >= n):
            raise ValueError("expected a contiguous float32 CUDA tensor")
        return t.data_ptr()

    def set_params(self, p):
        if _is_torch(p):
            _check(None, lib().sn_fno_set_params(self.h, self._dev(p, self.nparams), 1))
        else:
            a = np.ascontiguousarray(p, dtype=np.float32)
            _check(None, lib().sn_fno_set_params(self.h, a.ctypes.data, 0))

    def get_params(self):
        out = np.empty(self.nparams, np.float32)
        _check(None, lib().sn_fno_get_params(self.h, out.ctypes.data, 0))
        return out

    def get_grads(self, out=None):
        """Gradients of the last backward: into a float32 CUDA tensor `out`, or a
        new host array."""
        if out is not None and _is_torch(out):
            _check(None, lib().sn_fno_get_grads(self.h, self._dev(out, self.nparams), 1))
            return out
        out = np.empty(self.nparams, np.float32)
        _check(None, lib().sn_fno_get_grads(self.h, out.ctypes.data, 0))
        return out

    def set_grads(self, g):
        """Gradients for the next adam (a float32 CUDA tensor or a host array)."""
        if _is_torch(g):
            _check(None, lib().sn_fno_set_grads(self.h, self._dev(g, self.nparams), 1))
        else:
            a = np.ascontiguousarray(g, dtype=np.float32)
            if a.size != self.nparams:
                raise ValueError(f"expected {self.nparams} gradients")
            _check(None, lib().sn_fno_set_grads(self.h, a.ctypes.data, 0))

    def forward(self, x, out):
        B = x.shape[0]
        _check(None, lib().sn_fno_forward(self.h, self._dev(x, B * self.c_in * self.s ** 2),
                                          self._dev(out, B * 2 * self.s ** 2), B))
        return out

    def loss(self, target, B):
        v = ctypes.c_double()
        _check(None, lib().sn_fno_loss(self.h, self._dev(target, B * 2 * self.s ** 2), B,
                                       ctypes.byref(v)))
        return v.value

    def backward(self):
        _check(None, lib().sn_fno_backward(self.h))

    def adam(self, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(None, lib().sn_fno_adam(self.h, lr, beta1, beta2, eps, t))

    def sync(self):
        _check(None, lib().sn_fno_sync(self.h))

    def set_layer_form(self, form: int):
        """SN_FNO_LAYER_GEMMS or SN_FNO_LAYER_UMMA (the fused tcgen05 layer)."""
        _check(None, lib().sn_fno_set_layer_form(self.h, int(form)))

    def close(self):
        if getattr(self, "h", None):
            lib().sn_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cuda_tensor(t, dtype, name, numel=None):
    """Check a CUDA tensor before its pointer crosses the C-ABI (the library
    cannot check sizes behind a plain pointer)."""
    if not (_is_torch(t) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, {numel} needed")
    return t.data_ptr()


def sn_fno_pack(psi, feats, X, stream=None):
    """psi: (B, s, s) complex64 CUDA; feats: (B, nfeat) float32 CUDA; X: (B, 2+nfeat, s, s)."""
    import torch
    B, cells = psi.shape[0], psi[0].numel()
    nfeat = feats.shape[1] if feats is not None else 0
    pp = _cuda_tensor(psi, torch.complex64, "psi")
    fp = _cuda_tensor(feats, torch.float32, "feats", B * nfeat) if feats is not None else None
    xp = _cuda_tensor(X, torch.float32, "X", B * (2 + nfeat) * cells)
    _check(None, lib().sn_fno_pack(pp, fp, nfeat, xp, B, cells,
                                   ctypes.c_void_p(stream) if stream else None))


def sn_fno_pack2(psi_a, psi_c, feats, X, stream=None):
    """psi_a, psi_c: (B, s, s) complex64 CUDA; feats: (B, nfeat) float32 CUDA;
    X: (B, 4+nfeat, s, s) = (re a, im a, re c, im c, feats...)."""
    import torch
    B, cells = psi_a.shape[0], psi_a[0].numel()
    nfeat = feats.shape[1] if feats is not None else 0
    ap = _cuda_tensor(psi_a, torch.complex64, "psi_a")
    cp = _cuda_tensor(psi_c, torch.complex64, "psi_c", B * cells)
    fp = _cuda_tensor(feats, torch.float32, "feats", B * nfeat) if feats is not None else None
    xp = _cuda_tensor(X, torch.float32, "X", B * (4 + nfeat) * cells)
    _check(None, lib().sn_fno_pack2(ap, cp, fp, nfeat, xp, B, cells,
                                    ctypes.c_void_p(stream) if stream else None))


def sn_fno_unpack(Y, psi, stream=None):
    """Y: (B, 2, s, s) float32 CUDA -> psi: (B, s, s) complex64 CUDA."""
    import torch
    B, cells = psi.shape[0], psi[0].numel()
    pp = _cuda_tensor(psi, torch.complex64, "psi")
    yp = _cuda_tensor(Y, torch.float32, "Y", B * 2 * cells)
    _check(None, lib().sn_fno_unpack(yp, pp, B, cells, ctypes.c_void_p(stream) if stream else None))


def sn_mass_c64(psi, out, stream=None):
    """out: (B,) float64 CUDA tensor receiving sum |psi_b|^2."""
    import torch
    B, cells = psi.shape[0], psi[0].numel()
    pp = _cuda_tensor(psi, torch.complex64, "psi")
    op = _cuda_tensor(out, torch.float64, "out", B)
    _check(None, lib().sn_mass_c64(pp, B, cells, op, ctypes.c_void_p(stream) if stream else None))


def sn_test_line_fft_f32(data, n: int, sign: int, engine: int = SN_ENGINE_FP32, stream=None):
    """Test hook: in-place unnormalised DFTs of the contiguous complex64 lines of
    length n in a CUDA tensor (see sn_test_line_fft_f32 in include/sn.h)."""
    import torch
    if not (_is_torch(data) and data.is_cuda and data.dtype == torch.complex64
            and data.is_contiguous() and data.numel() % n == 0):
        raise ValueError("data must be a contiguous complex64 CUDA tensor of whole lines")
    _check(None, lib().sn_test_line_fft_f32(data.data_ptr(), data.numel() // n, n, sign, engine,
                                            ctypes.c_void_p(stream) if stream else None))


def sn_test_dsmem_rates(cluster_size: int) -> dict:
    """Distributed-shared-memory rates of clusters of cluster_size CTAs (see
    sn_test_dsmem_rates in include/sn.h): aggregate GB/s."""
    out = (ctypes.c_double * 3)()
    _check(None, lib().sn_test_dsmem_rates(int(cluster_size), out))
    return {"remote_read_gbs": out[0], "local_read_gbs": out[1], "push_gbs": out[2]}


def sn_test_line_fft_engines(data, n: int, sign: int, engine: int, reps: int = 1, stream=None) -> float:
    """reps in-place unnormalised DFTs of the lines of length n in a contiguous
    complex64 CUDA tensor on one line engine (SN_ENGINE_UMMA: the tcgen05 form,
    n = 256); returns the CUDA-event time of one launch in ms."""
    import torch
    if not (_is_torch(data) and data.is_cuda and data.dtype == torch.complex64 and data.is_contiguous()):
        raise ValueError("data must be a contiguous complex64 CUDA tensor")
    ms = ctypes.c_double(0.0)
    _check(None, lib().sn_test_line_fft_engines(data.data_ptr(), data.numel() // n, n, sign, engine,
                                                int(reps), ctypes.byref(ms),
                                                ctypes.c_void_p(stream) if stream else None))
    return ms.value


UMMA_PHASES = ("stage A operands", "stage A products", "stage B operands", "stage B products",
               "output")


def sn_test_umma_phases(data, sign: int, stream=None):
    """One launch of the tcgen05 line engine on the 256-point lines of a
    contiguous complex64 CUDA tensor, timed by phase; returns
    ({phase: clock cycles per tile of 8 lines}, tiles)."""
    import torch
    if not (_is_torch(data) and data.is_cuda and data.dtype == torch.complex64 and data.is_contiguous()):
        raise ValueError("data must be a contiguous complex64 CUDA tensor")
    cyc = (ctypes.c_double * 5)()
    tiles = ctypes.c_longlong(0)
    _check(None, lib().sn_test_umma_phases(data.data_ptr(), data.numel() // 256, sign, cyc,
                                           ctypes.byref(tiles),
                                           ctypes.c_void_p(stream) if stream else None))
    return dict(zip(UMMA_PHASES, list(cyc))), tiles.value


def sn_test_gemm_bf16(A, sA, B, sB, C, sC, M, N, K, Z, alpha=1.0, beta=0.0):
    """Test hook: strided batched BF16 GEMM on CUDA float32 tensors; s* = (sz, s_row, s_col)."""
    import torch

    def extent(s, rows, cols):  # one past the largest element offset the GEMM touches
        return (Z - 1) * s[0] + (rows - 1) * s[1] + (cols - 1) * s[2] + 1

    ap = _cuda_tensor(A, torch.float32, "A", extent(sA, M, K))
    bp = _cuda_tensor(B, torch.float32, "B", extent(sB, K, N))
    cp = _cuda_tensor(C, torch.float32, "C", extent(sC, M, N))
    _check(None, lib().sn_test_gemm_bf16(ap, *sA, bp, *sB, cp, *sC, M, N, K, Z, alpha, beta))


class Batch:
    """Owns one sn_batch handle: count square 2D complex64 instances."""

    def __init__(self, n: Sequence[int], L: Sequence[float], stream=None):
        self.n = [int(v) for v in n]
        self.L = [float(v) for v in L]
        self.h = sn_create_batch(self.n, self.L, stream)

    def set_kernels(self, kernels):
        sn_set_kernel_batch(self.h, kernels)

    def set_state(self, i: int, psi):
        sn_set_state_batch(self.h, i, psi, self.n[i] ** 2)

    def get_state(self, i: int, out=None):
        if out is None:
            out = np.empty((self.n[i], self.n[i]), np.complex64)
        return sn_get_state_batch(self.h, i, out, self.n[i] ** 2)

    def step(self, dt, nsteps: int):
        if np.isscalar(dt):
            dt = [dt] * len(self.n)
        sn_step_batch(self.h, dt, nsteps)

    def sync(self):
        sn_batch_sync(self.h)

    def observables(self, i: int) -> dict:
        return sn_observables_batch(self.h, i)

    def set_wait_limit(self, cycles: int):
        sn_set_batch_wait_limit(self.h, cycles)

    def set_ctas(self, per_sm: int):
        """Register budget of the launch: 3 (default), 2 or 1 resident CTAs per SM."""
        sn_set_batch_ctas(self.h, per_sm)

    def set_schedule(self, schedule: int):
        """SN_BATCH_PERSISTENT (one cooperative launch a call, the default),
        SN_BATCH_CLASSES (one cooperative launch per size class) or
        SN_BATCH_GRAPH (a graph per round, an instance per branch)."""
        sn_set_batch_schedule(self.h, schedule)

    def schedule(self) -> int:
        return sn_get_batch_schedule(self.h)

    def autotune(self, dt, steps: int = 50) -> int:
        """Time `steps` steps on the persistent and per-class schedules at each
        register budget and on the graph schedule, keep the fastest, restore the
        states; returns the budget kept (CTAs per SM); schedule() gives the
        schedule kept."""
        dts = [float(dt)] * len(self.n) if np.isscalar(dt) else [float(x) for x in dt]
        arr = (ctypes.c_double * len(dts))(*dts)
        out = ctypes.c_int(0)
        _check(None, lib().sn_autotune_batch(self.h, arr, int(steps), ctypes.byref(out)))
        return out.value

    def launch_count(self) -> int:
        return sn_batch_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            sn_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# Schedule cache (JSON): {key: [SN_SCHED_VALUES values: 3 * SN_SCHED_KINDS CTAs per SM,
# then 3 * SN_SCHED_KINDS stagings]}
# ----------------------------------------------------------------------------

def schedule_key(device: str, n: Sequence[int], engine: int, fields: int) -> str:
    return f"{device}|{'x'.join(str(int(v)) for v in n)}|c64|engine{int(engine)}|fields{int(fields)}"


def load_schedule(path: str, key: str):
    """The cached schedule of key, or None (no file, no entry, or a malformed one)."""
    try:
        with open(path) as f:
            vals = json.load(f).get(key)
    except (OSError, ValueError, AttributeError):
        return None
    m = 3 * SN_SCHED_KINDS
    if (not isinstance(vals, list) or len(vals) != SN_SCHED_VALUES
            or not all(isinstance(v, int) for v in vals)
            or not all(-1 <= v <= SN_SCHED_MAX_CTAS for v in vals[:m])
            or not all(-1 <= v <= SN_STAGING_REGISTERS for v in vals[m:])):
        return None
    return vals


def store_schedule(path: str, key: str, vals) -> None:
    try:
        with open(path) as f:
            table = json.load(f)
        if not isinstance(table, dict):
            table = {}
    except (OSError, ValueError):
        table = {}
    table[key] = [int(v) for v in vals]
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:  # no torch or no device: one shared key
        return "unknown-device"


# ----------------------------------------------------------------------------
# Convenience object over the same calls
# ----------------------------------------------------------------------------

class Grid:
    """Owns one sn_grid handle."""

    def __init__(self, n: Sequence[int], L: Sequence[float], dtype: str = "c64", stream=None):
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.dtype = SN_C64 if dtype in ("c64", "complex64", SN_C64) else SN_C128
        self.cells = int(np.prod(self.n))
        self.fields = 1
        self.engine = SN_ENGINE_FP32
        self.h = sn_create_grid(self.n, self.L, self.dtype, stream)

    @property
    def np_dtype(self):
        return np.complex64 if self.dtype == SN_C64 else np.complex128

    def set_kernel(self, **kw):
        sn_set_kernel(self.h, **kw)

    def set_fields(self, count: int):
        """Several coupled fields sharing one potential (see sn_set_fields in
        include/sn.h); the state is then an array of shape (count, *n)."""
        _check(self.h, lib().sn_set_fields(self.h, int(count)))
        self.fields = int(count)

    @property
    def state_shape(self):
        return self.n if self.fields == 1 else (self.fields,) + self.n

    def set_state(self, psi):
        sn_set_state(self.h, psi, self.dtype, self.fields * self.cells)

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.state_shape, dtype=self.np_dtype)
        return sn_get_state(self.h, out, self.dtype, self.fields * self.cells)

    def step(self, dt: float, nsteps: int = 1):
        sn_step(self.h, dt, nsteps)

    def observables(self) -> dict:
        return sn_observables(self.h)

    def set_fluid(self, nu=1.0, w=1.02, n_poly=1.0, model=SN_GRAVITY_NMC, lam=1.0, M=25.0,
                  rho_floor=1e-12, off=False, floor_mode=0):
        """Eq. 16 (self-gravitating fluid, GR or NMC) on a complex128 grid; off=True
        returns to Eqs. 1-2 (see sn_set_fluid in include/sn.h)."""
        if off:
            _check(self.h, lib().sn_set_fluid(self.h, None))
            return
        f = SnFluid(float(nu), float(w), float(n_poly), int(model), float(lam), float(M),
                    float(rho_floor), int(floor_mode))
        _check(self.h, lib().sn_set_fluid(self.h, ctypes.byref(f)))

    def schedule(self) -> list:
        """CTAs per SM of each fused pass kind and axis, [3 k + a], then the staging of
        each, [3 SN_SCHED_KINDS + 3 k + a] (sn_get_schedule)."""
        buf = (ctypes.c_int * SN_SCHED_VALUES)()
        _check(self.h, lib().sn_get_schedule(self.h, buf, len(buf)))
        return list(buf)

    def set_schedule(self, values):
        vals = [int(v) for v in values]
        buf = (ctypes.c_int * len(vals))(*vals)
        _check(self.h, lib().sn_set_schedule(self.h, buf, len(vals)))

    def autotune(self, dt: float, steps: int = 10, cache: Optional[str] = None,
                 device: Optional[str] = None) -> list:
        """Pick the schedule of the fused passes by timing them (sn_autotune),
        or take it from the JSON file `cache` when it holds one for this device,
        shape, engine and field count; a new result is added to the file."""
        key = schedule_key(device if device is not None else _device_name(), self.n,
                           self.engine, self.fields)
        if cache:
            got = load_schedule(cache, key)
            if got is not None:
                self.set_schedule(got)
                return got
        _check(self.h, lib().sn_autotune(self.h, float(dt), int(steps)))
        vals = self.schedule()
        if cache:
            store_schedule(cache, key, vals)
        return vals

    def set_engine(self, engine: int):
        """SN_ENGINE_FP32 or SN_ENGINE_TC16 (tensor cores on 256-point axes)."""
        _check(self.h, lib().sn_set_engine(self.h, int(engine)))
        self.engine = int(engine)

    def set_staging(self, mode: int):
        """SN_STAGING_TMA (tiles moved by bulk tensor copies) or SN_STAGING_REGISTERS;
        the results are the same bit for bit."""
        _check(self.h, lib().sn_set_staging(self.h, int(mode)))

    def set_obs_mode(self, mode: int):
        """SN_OBS_FP64 (FP64 transforms) or SN_OBS_FP32 (the step's FP32 line
        transforms with FP64 sums, complex64 grids)."""
        _check(self.h, lib().sn_set_obs_mode(self.h, int(mode)))

    def set_blocking(self, planes: int):
        """Run the y/x pass pair of each 3D round in slabs of `planes` z-planes
        (0: off); the results are the same bit for bit."""
        _check(self.h, lib().sn_set_blocking(self.h, int(planes)))

    def sync(self):
        sn_sync(self.h)

    def launch_count(self) -> int:
        return sn_launch_count(self.h)

    def profile_step(self, dt: float, nsteps: int) -> dict:
        return sn_profile_step(self.h, dt, nsteps)

    def close(self):
        if getattr(self, "h", None):
            sn_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
