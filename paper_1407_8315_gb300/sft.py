"""Thin Python binding of the C ABI in include/sft.h.

Argument marshalling only: every step of the transform runs in the CUDA
library (libsft.so); PyTorch supplies device memory and streams.  The names
mirror the C entry points (sft_params_default, sft_plan_create, sft_exact,
sft_exact_host, ...); `Plan` is a small convenience wrapper around them.

There is no CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from collections import namedtuple

import numpy as np

from . import _build_lib

SFT_OK, SFT_EINVAL, SFT_ENOMEM, SFT_ECUDA, SFT_ETIMEOUT, SFT_EUNSUPPORTED = range(6)
SFT_EXACT_ITER, SFT_EXACT_FIXED, SFT_GENERAL, SFT_GENERAL_UNPRUNED = 0, 1, 2, 3
SFT_FP64, SFT_MIXED = 0, 1

_MODES = {"iter": SFT_EXACT_ITER, "fixed": SFT_EXACT_FIXED, "general": SFT_GENERAL,
          "general-unpruned": SFT_GENERAL_UNPRUNED}
_PRECS = {"fp64": SFT_FP64, "mixed": SFT_MIXED}


class sft_params(C.Structure):
    _fields_ = [("N", C.c_int64), ("K", C.c_int64), ("d", C.c_int64), ("a_max", C.c_int32),
                ("max_iters", C.c_int32), ("mode", C.c_int32), ("precision", C.c_int32),
                ("n_cs_shifts", C.c_int32), ("reserved_", C.c_int32), ("seed", C.c_uint64),
                ("zero_tol", C.c_double), ("root_tol", C.c_double), ("res_tol", C.c_double)]


class sft_mlp_config(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_hidden", C.c_int32), ("n_sup", C.c_int32),
                ("n_cls", C.c_int32), ("seed", C.c_uint64), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class sft_result(C.Structure):
    _fields_ = [("cap", C.c_int64), ("idx", C.c_void_p), ("val", C.c_void_p),
                ("count", C.c_void_p), ("unresolved", C.c_void_p), ("overflow", C.c_void_p)]


EXPORTS = ["sft_params_default", "sft_plan_create", "sft_plan_destroy", "sft_plan_get_params",
           "sft_plan_workspace_bytes",
           "sft_exact", "sft_exact_host", "sft_plan_launches_per_call", "sft_strerror",
           "sft_last_cuda_error", "sft_plan_set_profiling", "sft_plan_stage_times",
           "sft_exact_noalloc", "sft_general", "sft_general_host", "sft_plan_cs_shifts",
           "sft_batch_create", "sft_batch_destroy", "sft_batch_set_options", "sft_batch",
           "sft_batch_info", "sft_batch_set_persistent", "sft_batch_persistent_info",
           "sft_mlp_config_for", "sft_mlp_create", "sft_mlp_destroy",
           "sft_mlp_param_count", "sft_mlp_get_params", "sft_mlp_set_params", "sft_mlp_features",
           "sft_mlp_forward", "sft_mlp_grad", "sft_mlp_train", "sft_plan_attach_mlp",
           "sft_exact_auto", "sft_alias_histogram", "sft_plan_set_sub_batches",
           "sft_plan_sub_batches", "sft_plan_set_quad_decoders", "sft_plan_queue_lengths",
           "sft_plan_stage_timeline", "sft_device_math_check"]

_lib = None


class SftError(RuntimeError):
    def __init__(self, status: int, what: str):
        lib = load()
        msg = lib.sft_strerror(status).decode()
        detail = lib.sft_last_cuda_error().decode()
        if detail:
            msg += " (" + detail + ")"
        super().__init__(f"{what}: {msg}")
        self.status = status


def library_path() -> str:
    return _build_lib.LIB


def load(build_if_missing: bool = False):
    """Load libsft.so (raises if it was not built and build_if_missing is False)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build_lib.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is missing; build it with "
                               "paper_1407_8315_gb300.build() (there is no CPU fallback)")
        _build_lib.build()
    lib = C.CDLL(path)
    P = C.POINTER
    lib.sft_params_default.argtypes = [P(sft_params), C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                       C.c_int32]
    lib.sft_plan_create.argtypes = [P(sft_params), C.c_int64, P(C.c_void_p)]
    lib.sft_plan_destroy.argtypes = [C.c_void_p]
    lib.sft_plan_destroy.restype = None
    lib.sft_plan_get_params.argtypes = [C.c_void_p, P(sft_params)]
    lib.sft_plan_queue_lengths.argtypes = [C.c_void_p, P(C.c_int64), C.c_int32]
    lib.sft_plan_queue_lengths.restype = C.c_int32
    lib.sft_plan_workspace_bytes.argtypes = [C.c_void_p]
    lib.sft_plan_workspace_bytes.restype = C.c_size_t
    lib.sft_exact.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, P(sft_result),
                              C.c_void_p]
    lib.sft_exact_host.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, P(sft_result),
                                   C.c_void_p]
    lib.sft_plan_launches_per_call.argtypes = [C.c_void_p]
    lib.sft_plan_launches_per_call.restype = C.c_int32
    lib.sft_plan_set_profiling.argtypes = [C.c_void_p, C.c_int32]
    lib.sft_plan_stage_times.argtypes = [C.c_void_p, C.c_int32, P(C.c_char_p), P(C.c_double),
                                         P(C.c_int64), P(C.c_int32)]
    lib.sft_device_math_check.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                                          C.c_void_p]
    lib.sft_plan_stage_timeline.argtypes = [C.c_void_p, C.c_int32, P(C.c_char_p), P(C.c_int32),
                                            P(C.c_double), P(C.c_double), P(C.c_int32)]
    lib.sft_exact_noalloc.argtypes = [P(sft_params), C.c_int64, C.c_void_p, C.c_int64,
                                      P(sft_result), C.c_void_p]
    lib.sft_general.argtypes = lib.sft_exact.argtypes
    lib.sft_general_host.argtypes = lib.sft_exact_host.argtypes
    lib.sft_plan_cs_shifts.argtypes = [C.c_void_p, P(C.c_int64), C.c_int32]
    lib.sft_plan_cs_shifts.restype = C.c_int32
    lib.sft_batch_create.argtypes = [P(C.c_void_p)]
    lib.sft_batch_destroy.argtypes = [C.c_void_p]
    lib.sft_batch_destroy.restype = None
    lib.sft_batch_set_options.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    lib.sft_batch.argtypes = [C.c_void_p, C.c_int64, P(sft_params), P(C.c_void_p), P(sft_result),
                              C.c_void_p]
    lib.sft_batch_info.argtypes = [C.c_void_p, P(C.c_int32), P(C.c_int64), P(C.c_int32)]
    lib.sft_batch_info.restype = C.c_int32
    lib.sft_batch_set_persistent.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    lib.sft_batch_persistent_info.argtypes = [C.c_void_p, P(C.c_int64), P(C.c_int32)]
    lib.sft_batch_persistent_info.restype = C.c_int32
    lib.sft_mlp_config_for.argtypes = [P(sft_params), P(sft_mlp_config)]
    lib.sft_mlp_create.argtypes = [P(sft_mlp_config), P(C.c_void_p)]
    lib.sft_mlp_destroy.argtypes = [C.c_void_p]
    lib.sft_mlp_destroy.restype = None
    lib.sft_mlp_param_count.argtypes = [C.c_void_p]
    lib.sft_mlp_param_count.restype = C.c_int64
    lib.sft_mlp_get_params.argtypes = [C.c_void_p, C.c_void_p]
    lib.sft_mlp_set_params.argtypes = [C.c_void_p, C.c_void_p]
    lib.sft_mlp_features.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                     C.c_void_p, C.c_int64, P(C.c_int64), C.c_void_p]
    lib.sft_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    lib.sft_mlp_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_void_p, C.c_void_p, C.c_void_p]
    lib.sft_mlp_train.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                  C.c_int32, C.c_int32, C.c_uint64, C.c_void_p, C.c_void_p]
    lib.sft_plan_attach_mlp.argtypes = [C.c_void_p, C.c_void_p]
    lib.sft_exact_auto.argtypes = [P(sft_params), C.c_int64, C.c_void_p, C.c_int64, C.c_int64,
                                   C.c_int64, P(sft_result), C.c_void_p, C.c_void_p]
    lib.sft_plan_set_sub_batches.argtypes = [C.c_void_p, C.c_int32]
    lib.sft_plan_sub_batches.argtypes = [C.c_void_p, C.c_int64]
    lib.sft_plan_sub_batches.restype = C.c_int32
    lib.sft_plan_set_quad_decoders.argtypes = [C.c_void_p, C.c_int32]
    lib.sft_alias_histogram.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                        C.c_void_p, C.c_void_p]
    lib.sft_strerror.argtypes = [C.c_int]
    lib.sft_strerror.restype = C.c_char_p
    lib.sft_last_cuda_error.argtypes = []
    lib.sft_last_cuda_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != SFT_OK:
        raise SftError(status, what)


def sft_params_default(N, K, d, mode="iter", precision="mixed") -> sft_params:
    p = sft_params()
    _check(load().sft_params_default(C.byref(p), int(N), int(K), int(d),
                                     _MODES.get(mode, mode), _PRECS.get(precision, precision)),
           "sft_params_default")
    return p


def sft_plan_create(params: sft_params, max_signals: int = 1) -> int:
    h = C.c_void_p()
    _check(load().sft_plan_create(C.byref(params), int(max_signals), C.byref(h)), "sft_plan_create")
    return h.value


def sft_plan_destroy(handle: int):
    load().sft_plan_destroy(C.c_void_p(handle))


def sft_plan_get_params(handle: int) -> sft_params:
    """The plan's parameters with every default filled in."""
    p = sft_params()
    _check(load().sft_plan_get_params(C.c_void_p(handle), C.byref(p)), "sft_plan_get_params")
    return p


def _check_signals(x, params: sft_params, what: str, host: bool = False):
    """Element type and row length of x against the parameters, before the
    library reads it: complex128 rows for SFT_FP64, complex64 for SFT_MIXED,
    at least N elements each."""
    if host:
        want = np.complex128 if params.precision == SFT_FP64 else np.complex64
        ok = x.dtype == want
    else:
        import torch
        want = torch.complex128 if params.precision == SFT_FP64 else torch.complex64
        ok = x.dtype == want
    if not ok:
        raise ValueError(f"{what}: signals of dtype {x.dtype}, the plan's precision needs {want}")
    if x.shape[1] < params.N:
        raise ValueError(f"{what}: rows of {x.shape[1]} samples, N = {params.N}")


def _check_result(out, B: int, cap: int, what: str, device=None):
    """Shapes (and, for device results, the device) of caller-supplied result
    arrays: idx and val [B, cap] (or [cap] when B is 1), count, unresolved and
    overflow [B]; int64 / complex128 / int64 / int32 / int32."""
    rows = [(out.idx, (B, cap), "int64"), (out.val, (B, cap), "complex128"),
            (out.count, (B,), "int64"), (out.unresolved, (B,), "int32"),
            (out.overflow, (B,), "int32")]
    for t, shape, dt in rows:
        n = 1
        for v in t.shape:
            n *= int(v)
        if n != shape[0] * (shape[1] if len(shape) > 1 else 1) or not str(t.dtype).endswith(dt):
            raise ValueError(f"{what}: result array of shape {tuple(t.shape)} / {t.dtype}, "
                             f"expected {shape} / {dt}")
        if device is not None and t.device != device:
            raise ValueError(f"{what}: result array on {t.device}, signals on {device}")
        if device is not None and not t.is_contiguous():
            raise ValueError(f"{what}: result arrays must be contiguous")


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


Result = namedtuple("Result", "idx val count unresolved overflow")


def sft_exact(handle: int, x, cap: int, out: Result | None = None, stream=None,
              _entry: str = "sft_exact") -> Result:
    """x: torch tensor [B, N] (complex128 for fp64 plans, complex64 for mixed)
    on the current CUDA device.  Returns device tensors (idx int64 [B, cap],
    val complex128 [B, cap], count int64 [B], unresolved int32 [B],
    overflow int32 [B])."""
    import torch
    if x.dim() == 1:
        x = x.unsqueeze(0)
    if not x.is_cuda:
        raise ValueError("sft_exact needs a CUDA tensor (use sft_exact_host for host data)")
    if x.stride(1) != 1:
        raise ValueError("signals must be contiguous along N")
    _check_signals(x, sft_plan_get_params(handle), _entry)
    B = x.shape[0]
    if out is None:
        dev = x.device
        out = Result(torch.empty((B, cap), dtype=torch.int64, device=dev),
                     torch.empty((B, cap), dtype=torch.complex128, device=dev),
                     torch.empty(B, dtype=torch.int64, device=dev),
                     torch.empty(B, dtype=torch.int32, device=dev),
                     torch.empty(B, dtype=torch.int32, device=dev))
    else:
        _check_result(out, B, cap, _entry, x.device)
    r = sft_result(cap, out.idx.data_ptr(), out.val.data_ptr(), out.count.data_ptr(),
                   out.unresolved.data_ptr(), out.overflow.data_ptr())
    # a single row has no meaningful pitch (numpy/torch may report 0 for it)
    pitch = x.stride(0) if B > 1 else x.shape[1]
    _check(getattr(load(), _entry)(C.c_void_p(handle), B, C.c_void_p(x.data_ptr()), pitch,
                                   C.byref(r), C.c_void_p(_stream_ptr(stream))), _entry)
    return out


def sft_general(handle: int, x, cap: int, out: Result | None = None, stream=None) -> Result:
    """Generally K-sparse transform (Algorithm 2) through the C entry point
    sft_general; arguments as sft_exact."""
    return sft_exact(handle, x, cap, out, stream, _entry="sft_general")


def sft_exact_host(handle: int, x: np.ndarray, cap: int, out: Result | None = None,
                   stream=None, _entry: str = "sft_exact_host") -> Result:
    """Host-memory variant: x is a numpy array [B, N]; results come back as
    numpy arrays.  The library copies in, computes and copies out."""
    if x.ndim == 1:
        x = x[None, :]
    if x.strides[1] != x.itemsize:
        raise ValueError("signals must be contiguous along N")
    _check_signals(x, sft_plan_get_params(handle), _entry, host=True)
    B = x.shape[0]
    if out is None:
        out = Result(np.empty((B, cap), np.int64), np.empty((B, cap), np.complex128),
                     np.empty(B, np.int64), np.empty(B, np.int32), np.empty(B, np.int32))
    else:
        _check_result(out, B, cap, _entry)
    r = sft_result(cap, out.idx.ctypes.data, out.val.ctypes.data, out.count.ctypes.data,
                   out.unresolved.ctypes.data, out.overflow.ctypes.data)
    pitch = x.strides[0] // x.itemsize if B > 1 else x.shape[1]
    _check(getattr(load(), _entry)(C.c_void_p(handle), B, C.c_void_p(x.ctypes.data),
                                   pitch, C.byref(r), C.c_void_p(_stream_ptr(stream))), _entry)
    return out


def sft_general_host(handle: int, x: np.ndarray, cap: int, out: Result | None = None,
                     stream=None) -> Result:
    return sft_exact_host(handle, x, cap, out, stream, _entry="sft_general_host")


def sft_plan_cs_shifts(handle: int) -> np.ndarray:
    lib = load()
    n = lib.sft_plan_cs_shifts(C.c_void_p(handle), None, 0)
    out = np.zeros(max(n, 0), dtype=np.int64)
    if n > 0:
        lib.sft_plan_cs_shifts(C.c_void_p(handle), out.ctypes.data_as(C.POINTER(C.c_int64)), n)
    return out


def _device_result(B, cap, dev):
    import torch
    return Result(torch.empty((B, cap), dtype=torch.int64, device=dev),
                  torch.empty((B, cap), dtype=torch.complex128, device=dev),
                  torch.empty(B, dtype=torch.int64, device=dev),
                  torch.empty(B, dtype=torch.int32, device=dev),
                  torch.empty(B, dtype=torch.int32, device=dev))


def sft_exact_noalloc(params: sft_params, x, cap: int, out: Result | None = None,
                      stream=None) -> Result:
    """Allocation-free entry point (no plan): the library keeps its tables and
    workspace in a static device array.  `x` and `out` are device tensors the
    caller provides (`out` is created here with torch if omitted)."""
    if x.dim() == 1:
        x = x.unsqueeze(0)
    if not x.is_cuda or x.stride(1) != 1:
        raise ValueError("sft_exact_noalloc needs a CUDA tensor contiguous along N")
    _check_signals(x, params, "sft_exact_noalloc")
    B = x.shape[0]
    if out is None:
        out = _device_result(B, cap, x.device)
    else:
        _check_result(out, B, cap, "sft_exact_noalloc", x.device)
    r = sft_result(cap, out.idx.data_ptr(), out.val.data_ptr(), out.count.data_ptr(),
                   out.unresolved.data_ptr(), out.overflow.data_ptr())
    pitch = x.stride(0) if B > 1 else x.shape[1]
    _check(load().sft_exact_noalloc(C.byref(params), B, C.c_void_p(x.data_ptr()), pitch,
                                    C.byref(r), C.c_void_p(_stream_ptr(stream))),
           "sft_exact_noalloc")
    return out


def sft_plan_queue_lengths(handle: int) -> list:
    """Bins queued per level (ITER) or per round (FIXED) in the plan's last
    call, summed over its signals."""
    out = (C.c_int64 * 16)()
    n = load().sft_plan_queue_lengths(C.c_void_p(handle), out, 16)
    if n < 0:
        raise SftError(SFT_ECUDA, "sft_plan_queue_lengths")
    return [int(out[i]) for i in range(n)]


def sft_plan_set_profiling(handle: int, enable: bool):
    _check(load().sft_plan_set_profiling(C.c_void_p(handle), int(bool(enable))),
           "sft_plan_set_profiling")


def sft_plan_stage_times(handle: int) -> dict:
    """{stage name: (total ms, launches)} since the previous read; resets."""
    cap = 32
    names = (C.c_char_p * cap)()
    ms = (C.c_double * cap)()
    cnt = (C.c_int64 * cap)()
    n = C.c_int32(0)
    _check(load().sft_plan_stage_times(C.c_void_p(handle), cap, names, ms, cnt, C.byref(n)),
           "sft_plan_stage_times")
    return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(min(n.value, cap))}


def sft_device_math_check(x_ptr: int, n: int, out_ptr: int, which: int, stream: int = 0):
    """The decoders' device arithmetic on n elements (device pointers; see
    the header): 0 the reciprocal, 1 the float-to-double widening, 2 the
    complex square root (n complex values)."""
    _check(load().sft_device_math_check(C.c_void_p(x_ptr), int(n), C.c_void_p(out_ptr),
                                        int(which), C.c_void_p(stream)),
           "sft_device_math_check")


def sft_plan_stage_timeline(handle: int, cap: int = 4096) -> list:
    """[(stage, sub-batch, start ms, end ms)] per profiled launch since the
    previous read, relative to the first launch's start; resets."""
    names = (C.c_char_p * cap)()
    sub = (C.c_int32 * cap)()
    t0 = (C.c_double * cap)()
    t1 = (C.c_double * cap)()
    n = C.c_int32(0)
    _check(load().sft_plan_stage_timeline(C.c_void_p(handle), cap, names, sub, t0, t1,
                                          C.byref(n)), "sft_plan_stage_timeline")
    return [(names[i].decode(), int(sub[i]), t0[i], t1[i]) for i in range(min(n.value, cap))]


class Plan:
    """Convenience owner of one sft plan."""

    def __init__(self, N, K, d, mode="iter", precision="mixed", max_signals=1, a_max=0,
                 max_iters=0, zero_tol=0.0, root_tol=0.0, res_tol=0.0, seed=0, n_cs_shifts=0):
        p = sft_params_default(N, K, d, mode, precision)
        if a_max:
            p.a_max = int(a_max)
            if mode in ("general", "general-unpruned") and not n_cs_shifts:
                p.n_cs_shifts = 3 * int(a_max)
        p.max_iters = int(max_iters) if max_iters else int(p.a_max)
        p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        if n_cs_shifts:
            p.n_cs_shifts = int(n_cs_shifts)
        if zero_tol:
            p.zero_tol = float(zero_tol)
        if root_tol:
            p.root_tol = float(root_tol)
        if res_tol:
            p.res_tol = float(res_tol)
        self.params = p
        self.N, self.K, self.d = int(N), int(K), int(d)
        self.M = self.N // self.d
        self.precision = precision
        self.max_signals = int(max_signals)
        self.handle = None
        self.handle = sft_plan_create(p, max_signals)

    @property
    def dtype_np(self):
        return np.complex128 if self.precision in ("fp64", SFT_FP64) else np.complex64

    @property
    def workspace_bytes(self) -> int:
        return int(load().sft_plan_workspace_bytes(C.c_void_p(self.handle)))

    @property
    def launches_per_call(self) -> int:
        return int(load().sft_plan_launches_per_call(C.c_void_p(self.handle)))

    def exact(self, x, cap=None, out=None, stream=None) -> Result:
        return sft_exact(self.handle, x, cap or max(self.K, 1), out, stream)

    def exact_host(self, x, cap=None, out=None, stream=None) -> Result:
        return sft_exact_host(self.handle, x, cap or max(self.K, 1), out, stream)

    def general(self, x, cap=None, out=None, stream=None) -> Result:
        return sft_general(self.handle, x, cap or max(self.K, 1), out, stream)

    def general_host(self, x, cap=None, out=None, stream=None) -> Result:
        return sft_general_host(self.handle, x, cap or max(self.K, 1), out, stream)

    @property
    def cs_shifts(self) -> np.ndarray:
        return sft_plan_cs_shifts(self.handle)

    def set_sub_batches(self, n: int):
        """Sub-batches per call: 0 chooses from the call's size, 1..4 fixes it."""
        _check(load().sft_plan_set_sub_batches(C.c_void_p(self.handle), int(n)),
               "sft_plan_set_sub_batches")

    def sub_batches(self, n_signals: int) -> int:
        return int(load().sft_plan_sub_batches(C.c_void_p(self.handle), int(n_signals)))

    def set_quad_decoders(self, enable: bool = True):
        """Four lanes per bin for three and four aliases on calls that run as
        one sub-batch (short queues only; values to ~1e-13, not bitwise)."""
        _check(load().sft_plan_set_quad_decoders(C.c_void_p(self.handle), int(bool(enable))),
               "sft_plan_set_quad_decoders")

    def set_profiling(self, enable: bool = True):
        sft_plan_set_profiling(self.handle, enable)

    def attach_mlp(self, mlp):
        """Attach a learned proposal (Mlp) to this SFT_GENERAL plan; None detaches."""
        _check(load().sft_plan_attach_mlp(C.c_void_p(self.handle),
                                          C.c_void_p(mlp.handle if mlp is not None else None)),
               "sft_plan_attach_mlp")
        self._mlp = mlp

    def stage_timeline(self) -> list:
        return sft_plan_stage_timeline(self.handle)

    def stage_times(self) -> dict:
        return sft_plan_stage_times(self.handle)

    def queue_lengths(self) -> list:
        return sft_plan_queue_lengths(self.handle)

    def close(self):
        if self.handle:
            sft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A heterogeneous batch context (sft_batch_create / sft_batch)."""

    def __init__(self, use_graph: bool = True, autotune: bool = True, persistent: bool = True,
                 persistent_ctas: int = 0):
        h = C.c_void_p()
        _check(load().sft_batch_create(C.byref(h)), "sft_batch_create")
        self.handle = h.value
        _check(load().sft_batch_set_options(C.c_void_p(self.handle), int(use_graph), int(autotune)),
               "sft_batch_set_options")
        self.set_persistent(persistent, persistent_ctas)
        self._keep = None

    def set_persistent(self, enable: bool = True, ctas: int = 0):
        """Run the batch's exactly sparse signals that fit one CTA in the
        persistent kernel (sft_batch_set_persistent); ctas 0: autotuned."""
        _check(load().sft_batch_set_persistent(C.c_void_p(self.handle), int(bool(enable)),
                                               int(ctas)), "sft_batch_set_persistent")

    def persistent_info(self):
        n, c = C.c_int64(), C.c_int32()
        load().sft_batch_persistent_info(C.c_void_p(self.handle), C.byref(n), C.byref(c))
        return {"signals": n.value, "ctas": c.value}

    @staticmethod
    def _ptr(a) -> int:
        if hasattr(a, "data_ptr"):
            return int(a.data_ptr())
        if isinstance(a, np.ndarray):
            return int(a.ctypes.data)
        return int(a)

    @staticmethod
    def _size(a) -> int:
        return int(a.numel()) if hasattr(a, "numel") else int(np.size(a))

    def prepare(self, params, xs, outs):
        """Marshal one call: params (sft_params list), xs (device tensors,
        page-locked host arrays or raw addresses, one signal each), outs
        (Result of per-signal buffers).  Returns the argument arrays for
        launch(), reusable while the buffers stay alive."""
        n = len(params)
        pa = (sft_params * n)(*params)
        xa = (C.c_void_p * n)(*[self._ptr(x) for x in xs])
        ra = (sft_result * n)(*[sft_result(self._size(o.idx), self._ptr(o.idx), self._ptr(o.val),
                                           self._ptr(o.count), self._ptr(o.unresolved),
                                           self._ptr(o.overflow)) for o in outs])
        return n, pa, xa, ra

    def launch(self, prepared, stream=None):
        n, pa, xa, ra = prepared
        _check(load().sft_batch(C.c_void_p(self.handle), n, pa, xa, ra,
                                C.c_void_p(_stream_ptr(stream))), "sft_batch")

    def run(self, params, xs, outs, stream=None):
        """params: list of sft_params; xs: one signal each (device tensors or
        page-locked host memory); outs: list of Result with per-signal
        buffers."""
        self._keep = self.prepare(params, xs, outs)
        self.launch(self._keep, stream)

    def info(self):
        g, t = C.c_int32(), C.c_int32()
        nodes = C.c_int64()
        load().sft_batch_info(C.c_void_p(self.handle), C.byref(g), C.byref(nodes), C.byref(t))
        return {"groups": g.value, "graph_nodes": nodes.value, "tuned": t.value}

    def close(self):
        if self.handle:
            load().sft_batch_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sft_exact_auto(params: sft_params, x, cap: int, M_start: int = 1, M_max: int = 0,
                   stream=None):
    """Unknown K (Sec. II-E): x torch CUDA tensor [B, N].  Returns (Result of
    device tensors, numpy int64 [B] of the M each signal stopped at)."""
    import torch
    if x.dim() == 1:
        x = x.unsqueeze(0)
    B = x.shape[0]
    out = _device_result(B, cap, x.device)
    r = sft_result(cap, out.idx.data_ptr(), out.val.data_ptr(), out.count.data_ptr(),
                   out.unresolved.data_ptr(), out.overflow.data_ptr())
    m = np.zeros(B, np.int64)
    pitch = x.stride(0) if B > 1 else x.shape[1]
    _check(load().sft_exact_auto(C.byref(params), B, C.c_void_p(x.data_ptr()), pitch, int(M_start),
                                 int(M_max), C.byref(r), m.ctypes.data,
                                 C.c_void_p(_stream_ptr(stream))), "sft_exact_auto")
    return out, m


# ------------------------------------------------------- learned proposal
def support_bits(supports, d: int) -> np.ndarray:
    """Support labels as the C ABI takes them: uint32 [rows][4], bit t of
    word t // 32 set for every t in the row's support (t < d <= 128)."""
    out = np.zeros((len(supports), 4), np.uint32)
    for i, ts in enumerate(supports):
        for t in ts:
            if not 0 <= t < d:
                raise ValueError("support index outside [0, d)")
            out[i, t >> 5] |= np.uint32(1) << np.uint32(t & 31)
    return out


class Mlp:
    """The learned support proposal (sft_mlp_*): a network sized for a
    SFT_GENERAL plan's (a_max, n_cs_shifts, d)."""

    def __init__(self, plan: "Plan" = None, seed: int = 0, lr: float = 0.0, config=None):
        cfg = sft_mlp_config()
        if config is not None:
            cfg = config
        else:
            _check(load().sft_mlp_config_for(C.byref(plan.params), C.byref(cfg)),
                   "sft_mlp_config_for")
            cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
            if lr:
                cfg.lr = float(lr)
        self.config = cfg
        self.n_in, self.n_sup, self.n_cls = cfg.n_in, cfg.n_sup, cfg.n_cls
        self.n_out = cfg.n_sup + cfg.n_cls
        h = C.c_void_p()
        _check(load().sft_mlp_create(C.byref(cfg), C.byref(h)), "sft_mlp_create")
        self.handle = h.value

    @property
    def param_count(self) -> int:
        return int(load().sft_mlp_param_count(C.c_void_p(self.handle)))

    @property
    def params(self) -> np.ndarray:
        out = np.empty(self.param_count, np.float32)
        _check(load().sft_mlp_get_params(C.c_void_p(self.handle), out.ctypes.data),
               "sft_mlp_get_params")
        return out

    @params.setter
    def params(self, v):
        v = np.ascontiguousarray(v, dtype=np.float32)
        if v.size != self.param_count:
            raise ValueError("wrong parameter count")
        _check(load().sft_mlp_set_params(C.c_void_p(self.handle), v.ctypes.data),
               "sft_mlp_set_params")

    def features(self, plan: "Plan", x, cap_rows: int):
        """Features of the bins the plan votes on x [B, N] (CUDA tensor):
        (feat [rows, n_in] float32, rows [rows, 3] int32: signal, bin, a_k)."""
        import torch
        if x.dim() == 1:
            x = x.unsqueeze(0)
        B = x.shape[0]
        feat = torch.empty((cap_rows, self.n_in), dtype=torch.float32, device=x.device)
        rows = torch.empty((cap_rows, 3), dtype=torch.int32, device=x.device)
        n = C.c_int64()
        pitch = x.stride(0) if B > 1 else x.shape[1]
        _check(load().sft_mlp_features(C.c_void_p(plan.handle), B, C.c_void_p(x.data_ptr()), pitch,
                                       C.c_void_p(feat.data_ptr()), C.c_void_p(rows.data_ptr()),
                                       cap_rows, C.byref(n), C.c_void_p(_stream_ptr(None))),
               "sft_mlp_features")
        k = min(int(n.value), cap_rows)
        return feat[:k], rows[:k], int(n.value)

    def forward(self, feat):
        import torch
        logits = torch.empty((feat.shape[0], self.n_out), dtype=torch.float32, device=feat.device)
        _check(load().sft_mlp_forward(C.c_void_p(self.handle), C.c_void_p(feat.data_ptr()),
                                      feat.shape[0], C.c_void_p(logits.data_ptr()),
                                      C.c_void_p(_stream_ptr(None))), "sft_mlp_forward")
        return logits

    def grad(self, feat, cls, sup):
        """(gradient [param_count] float32 tensor, mean loss tensor [1])."""
        import torch
        g = torch.empty(self.param_count, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        _check(load().sft_mlp_grad(C.c_void_p(self.handle), C.c_void_p(feat.data_ptr()),
                                   C.c_void_p(cls.data_ptr()), C.c_void_p(sup.data_ptr()),
                                   feat.shape[0], C.c_void_p(g.data_ptr()),
                                   C.c_void_p(loss.data_ptr()), C.c_void_p(_stream_ptr(None))),
               "sft_mlp_grad")
        return g, loss

    def train(self, feat, cls, sup, epochs: int, batch: int = 4096, seed: int = 0) -> np.ndarray:
        losses = np.zeros(epochs, np.float32)
        _check(load().sft_mlp_train(C.c_void_p(self.handle), C.c_void_p(feat.data_ptr()),
                                    C.c_void_p(cls.data_ptr()), C.c_void_p(sup.data_ptr()),
                                    feat.shape[0], int(epochs), int(batch),
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, losses.ctypes.data,
                                    C.c_void_p(_stream_ptr(None))), "sft_mlp_train")
        return losses

    def close(self):
        if self.handle:
            load().sft_mlp_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alias_histogram(supports, M: int, n_cells: int = 9, stream=None):
    """Collision counts of Sec. II-C: supports is a device int64 tensor
    [n_sets, K]; returns a device int64 tensor hist[n_cells] with hist[a] the
    number of (set, bin) pairs whose bin k < M holds exactly a locations
    (the last cell: n_cells - 1 or more)."""
    import torch
    if supports.dtype != torch.int64 or not supports.is_cuda or supports.dim() != 2:
        raise ValueError("supports must be a 2-D int64 CUDA tensor")
    s = supports.contiguous()
    hist = torch.empty(int(n_cells), dtype=torch.int64, device=s.device)
    _check(load().sft_alias_histogram(C.c_void_p(s.data_ptr()), s.shape[0], s.shape[1], int(M),
                                      int(n_cells), C.c_void_p(hist.data_ptr()),
                                      C.c_void_p(_stream_ptr(stream))), "sft_alias_histogram")
    return hist
