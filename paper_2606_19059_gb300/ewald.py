"""Python binding of the C ABI in include/ewald_gb300.h.

Argument marshalling only: every step of the apply runs in the CUDA library
``libewald_gb300.so``.  Functions keep the C names.  Device arrays are passed
as raw pointers (e.g. ``tensor.data_ptr()`` of contiguous float64 CUDA
tensors) and streams as ``torch.cuda.Stream.cuda_stream`` integers.  If the
library is missing the import-time loader raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LIB_PATH = _build.LIB


class EwaldError(RuntimeError):
    """A library call returned a status other than EWALD_OK."""

    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {ewald_status_string(status)} (status {status})")


EWALD_OK, EWALD_EINVAL, EWALD_ENOMEM, EWALD_ECUDA, EWALD_ECUFFT, EWALD_ETIMEOUT, EWALD_EUNSUPPORTED = range(7)
EWALD_F64, EWALD_F32_BULK = 0, 1


class ewald_params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("xi", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("cell", ctypes.c_double),
        ("h", ctypes.c_double),
        ("est_err", ctypes.c_double),
        ("n_c", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("P", ctypes.c_int32),
        ("poly_deg", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("p2p_block", ctypes.c_int32),
        ("near_f64", ctypes.c_int32),
        ("fft_f64", ctypes.c_int32),
        ("footprint_bytes", ctypes.c_int64),
        ("near_ds", ctypes.c_int32),
        ("reserved_", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ewald_stage_timing(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("bin_ms", "p2p_ms", "p2g_ms", "fft_ms", "scale_ms", "ifft_ms", "g2p_ms", "sum_ms",
                 "total_ms")]

    def as_dict(self):
        return {name: float(getattr(self, name)) for name, _ in self._fields_}


_lib = None

# (name, restype, argtypes)
_P = ctypes.c_void_p
_SIGS = [
    ("ewald_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("ewald_choose_params", ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(ewald_params), ctypes.POINTER(ewald_params)]),
    ("ewald_plan", ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(_P)]),
    ("ewald_plan_ex", ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(ewald_params), ctypes.POINTER(_P)]),
    ("ewald_destroy", None, [_P]),
    ("ewald_get_params", ctypes.c_int, [_P, ctypes.POINTER(ewald_params)]),
    ("ewald_apply", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("ewald_set_positions", ctypes.c_int, [_P, _P, _P]),
    ("ewald_apply_forces", ctypes.c_int, [_P, _P, _P, _P]),
    ("ewald_apply_combined", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("ewald_apply_host", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("ewald_near_field", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("ewald_far_field", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("ewald_spread", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("ewald_interp", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("ewald_fourier_convolve", ctypes.c_int, [_P, _P, _P, _P]),
    ("ewald_set_timing", ctypes.c_int, [_P, ctypes.c_int]),
    ("ewald_stage_times", ctypes.c_int, [_P, ctypes.POINTER(ewald_stage_timing)]),
    ("ewald_sync_status", ctypes.c_int, [_P, _P]),
    ("ewald_debug_fail_alloc", ctypes.c_int, [ctypes.c_int32]),
    ("ewald_launch_counts", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    ("ewald_window_eval", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P,
                                         ctypes.POINTER(ctypes.c_double)]),
    ("ewald_window_hat", ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_int64, _P, _P]),
    ("ewald_near_field_noalloc", ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ewald_params), _P, _P, _P, _P]),
    ("ewald_probe_fma_peaks", ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double)]),
    ("ewald_autotune_candidates", ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                 ctypes.c_int32, ctypes.POINTER(ewald_params),
                                                 ctypes.POINTER(ctypes.c_int32)]),
    ("ewald_autotune", ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int32,
                                      ctypes.POINTER(ewald_params), ctypes.POINTER(ctypes.c_double)]),
    ("ewald_autotune_clear", None, []),
    ("ewald_batch_create", ctypes.c_int, [ctypes.c_int32, _P, _P, _P, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(_P)]),
    ("ewald_batch_buffers", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                           ctypes.POINTER(_P)]),
    ("ewald_batch_get_params", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ewald_params)]),
    ("ewald_batch_plan", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    ("ewald_batch_apply", ctypes.c_int, [_P, _P]),
    ("ewald_batch_launch_counts", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    ("ewald_batch_destroy", None, [_P]),
    ("ewald_server_create", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]),
    ("ewald_server_submit", ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64)]),
    ("ewald_server_poll", ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double)]),
    ("ewald_server_wait", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double]),
    ("ewald_server_cancel", ctypes.c_int, [_P, ctypes.c_int64]),
    ("ewald_server_resume", ctypes.c_int, [_P]),
    ("ewald_server_stats", ctypes.c_int, [_P, _P]),
    ("ewald_server_destroy", None, [_P]),
]
EXPORTED = [name for name, _, _ in _SIGS]


def load(build_if_missing: bool = True):
    """Load libewald_gb300.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH}")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st: int, where: str):
    if st != EWALD_OK:
        raise EwaldError(st, where)


def ewald_status_string(status: int) -> str:
    return load().ewald_status_string(int(status)).decode()


def ewald_choose_params(N: int, L: float, tol: float, dtype: int = EWALD_F32_BULK, override=None):
    out = ewald_params()
    st = load().ewald_choose_params(int(N), float(L), float(tol), int(dtype),
                                    ctypes.byref(override) if override is not None else None,
                                    ctypes.byref(out))
    _check(st, "ewald_choose_params")
    return out


def ewald_plan_ex(N: int, L: float, tol: float, dtype: int = EWALD_F32_BULK, override=None) -> int:
    h = _P()
    st = load().ewald_plan_ex(int(N), float(L), float(tol), int(dtype),
                              ctypes.byref(override) if override is not None else None, ctypes.byref(h))
    _check(st, "ewald_plan_ex")
    return h.value


def ewald_plan(N: int, L: float, tol: float, dtype: int = EWALD_F32_BULK) -> int:
    return ewald_plan_ex(N, L, tol, dtype, None)


def ewald_destroy(plan: int) -> None:
    load().ewald_destroy(plan)


def ewald_get_params(plan: int) -> ewald_params:
    out = ewald_params()
    _check(load().ewald_get_params(plan, ctypes.byref(out)), "ewald_get_params")
    return out


def _call(name: str, *args):
    _check(getattr(load(), name)(*args), name)


def ewald_apply(plan, x_ptr, f_ptr, u_ptr, stream=0):
    _call("ewald_apply", plan, x_ptr, f_ptr, u_ptr, stream)


def ewald_set_positions(plan, x_ptr, stream=0):
    _call("ewald_set_positions", plan, x_ptr, stream)


def ewald_apply_forces(plan, f_ptr, u_ptr, stream=0):
    _call("ewald_apply_forces", plan, f_ptr, u_ptr, stream)


def ewald_apply_combined(plan, x_ptr, f_ptr, q_ptr, n_ptr, u_ptr, stream=0):
    _call("ewald_apply_combined", plan, x_ptr, f_ptr, q_ptr, n_ptr, u_ptr, stream)


def ewald_apply_host(plan, x_ptr, f_ptr, u_ptr, stream=0):
    _call("ewald_apply_host", plan, x_ptr, f_ptr, u_ptr, stream)


def ewald_near_field(plan, x_ptr, f_ptr, u_ptr, stream=0):
    _call("ewald_near_field", plan, x_ptr, f_ptr, u_ptr, stream)


def ewald_far_field(plan, x_ptr, f_ptr, u_ptr, stream=0):
    _call("ewald_far_field", plan, x_ptr, f_ptr, u_ptr, stream)


def ewald_spread(plan, x_ptr, f_ptr, grid_ptr, stream=0):
    _call("ewald_spread", plan, x_ptr, f_ptr, grid_ptr, stream)


def ewald_interp(plan, x_ptr, grid_ptr, u_ptr, stream=0):
    _call("ewald_interp", plan, x_ptr, grid_ptr, u_ptr, stream)


def ewald_fourier_convolve(plan, grid_in_ptr, grid_out_ptr, stream=0):
    _call("ewald_fourier_convolve", plan, grid_in_ptr, grid_out_ptr, stream)


def ewald_set_timing(plan, enable: int = 1):
    _call("ewald_set_timing", plan, int(enable))


def ewald_stage_times(plan) -> dict:
    out = ewald_stage_timing()
    _check(load().ewald_stage_times(plan, ctypes.byref(out)), "ewald_stage_times")
    return out.as_dict()


def ewald_sync_status(plan, stream=0) -> int:
    """Synchronise and return the device error status (EWALD_OK or EWALD_EINVAL)."""
    return int(load().ewald_sync_status(plan, stream))


def ewald_debug_fail_alloc(nth: int) -> None:
    """Make the nth next device allocation of any plan fail (0 disarms)."""
    _check(load().ewald_debug_fail_alloc(int(nth)), "ewald_debug_fail_alloc")


def ewald_launch_counts(plan):
    k, f = ctypes.c_int32(), ctypes.c_int32()
    _check(load().ewald_launch_counts(plan, ctypes.byref(k), ctypes.byref(f)), "ewald_launch_counts")
    return k.value, f.value


def ewald_window_eval(P: int, nu: int, t):
    import numpy as np

    t = np.ascontiguousarray(t, dtype=np.float64)
    w = np.empty_like(t)
    err = ctypes.c_double()
    _check(load().ewald_window_eval(int(P), int(nu), t.size, t.ctypes.data, w.ctypes.data,
                                    ctypes.byref(err)), "ewald_window_eval")
    return w, err.value


def ewald_window_hat(P: int, h: float, k):
    import numpy as np

    k = np.ascontiguousarray(k, dtype=np.float64)
    w = np.empty_like(k)
    _check(load().ewald_window_hat(int(P), float(h), k.size, k.ctypes.data, w.ctypes.data),
           "ewald_window_hat")
    return w


def ewald_probe_fma_peaks(device: int = 0):
    """Measured (FP32, FP64) FMA-pipe peaks of `device` in TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().ewald_probe_fma_peaks(int(device), ctypes.byref(a), ctypes.byref(b)), "ewald_probe_fma_peaks")
    return a.value, b.value


def ewald_near_field_noalloc(N: int, params: ewald_params, x_ptr, f_ptr, u_ptr, stream=0):
    """Near field with no device allocation (fixed in-library workspace, N <= 32768);
    for callers that cannot allocate device memory themselves."""
    _check(load().ewald_near_field_noalloc(int(N), ctypes.byref(params), x_ptr, f_ptr, u_ptr, stream),
           "ewald_near_field_noalloc")


EWALD_TUNE_MODEL, EWALD_TUNE_MEASURE = 0, 1


def ewald_autotune_candidates(N: int, L: float, tol: float, dtype: int = EWALD_F32_BULK, cap: int = 32):
    arr = (ewald_params * int(cap))()
    n = ctypes.c_int32(0)
    _check(load().ewald_autotune_candidates(int(N), float(L), float(tol), int(dtype), int(cap), arr,
                                            ctypes.byref(n)), "ewald_autotune_candidates")
    return [arr[i] for i in range(n.value)]


def ewald_autotune(N: int, L: float, tol: float, dtype: int = EWALD_F32_BULK, mode: int = EWALD_TUNE_MEASURE):
    out = ewald_params()
    ms = ctypes.c_double(0.0)
    _check(load().ewald_autotune(int(N), float(L), float(tol), int(dtype), int(mode), ctypes.byref(out),
                                 ctypes.byref(ms)), "ewald_autotune")
    return out, ms.value


def ewald_autotune_clear():
    load().ewald_autotune_clear()


class Batch:
    """Owner of one ewald_batch_t: many independent boxes applied with one
    graph launch.  Per box, x/f/u are views (torch, CUDA, float64, N x 3) of
    the batch's own device buffers (marshalling only)."""

    def __init__(self, N, L, tol, dtype: int = EWALD_F32_BULK, tune: int = EWALD_TUNE_MEASURE, nstreams: int = 16):
        import numpy as np

        self.N = np.ascontiguousarray(N, dtype=np.int64)
        Ls = np.ascontiguousarray(np.broadcast_to(np.asarray(L, dtype=np.float64), self.N.shape))
        tols = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, dtype=np.float64), self.N.shape))
        h = _P()
        _check(load().ewald_batch_create(len(self.N), self.N.ctypes.data, Ls.ctypes.data, tols.ctypes.data,
                                         int(dtype), int(tune), int(nstreams), ctypes.byref(h)),
               "ewald_batch_create")
        self.handle = h.value
        self._views = None

    def close(self):
        if getattr(self, "handle", None):
            load().ewald_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.N)

    def params(self, box: int) -> ewald_params:
        out = ewald_params()
        _check(load().ewald_batch_get_params(self.handle, int(box), ctypes.byref(out)), "ewald_batch_get_params")
        return out

    def buffers(self, box: int):
        """(x, f, u) torch views of box `box`'s device buffers."""
        import torch

        if self._views is None:
            self._views = {}
        if box not in self._views:
            px, pf, pu = _P(), _P(), _P()
            _check(load().ewald_batch_buffers(self.handle, int(box), ctypes.byref(px), ctypes.byref(pf),
                                              ctypes.byref(pu)), "ewald_batch_buffers")
            n = int(self.N[box])
            self._views[box] = tuple(_device_view(p.value, (n, 3)) for p in (px, pf, pu))
        return self._views[box]

    def apply(self, stream=None):
        import torch

        s = stream if stream is not None else torch.cuda.current_stream()
        _check(load().ewald_batch_apply(self.handle, s.cuda_stream), "ewald_batch_apply")

    def launch_counts(self):
        k, f = ctypes.c_int32(), ctypes.c_int32()
        _check(load().ewald_batch_launch_counts(self.handle, ctypes.byref(k), ctypes.byref(f)),
               "ewald_batch_launch_counts")
        return k.value, f.value


def _device_view(ptr: int, shape):
    """A torch float64 CUDA tensor over memory the library owns (no copy)."""
    import torch

    n = 1
    for d in shape:
        n *= d

    class _Arr:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (ptr, False),
                                    "version": 3, "strides": None}

    t = torch.as_tensor(_Arr(), device="cuda")
    assert t.data_ptr() == ptr and t.numel() == n
    return t


class ewald_request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("L", ctypes.c_double), ("tol", ctypes.c_double),
                ("dtype", ctypes.c_int32), ("napplies", ctypes.c_int32), ("perturb", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("x_host", _P), ("f_host", _P), ("u_host", _P)]


class ewald_server_summary(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("queued", ctypes.c_int64), ("active", ctypes.c_int64),
                ("peak_footprint_bytes", ctypes.c_int64), ("particle_applies", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("throughput", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


EWALD_REQ_QUEUED, EWALD_REQ_RUNNING, EWALD_REQ_DONE, EWALD_REQ_FAILED, EWALD_REQ_CANCELLED = range(5)


class Server:
    """Owner of one ewald_server_t (marshalling only).  submit() takes host
    numpy arrays and returns a ticket; the arrays are kept alive here until
    the request is finished and result(ticket) hands back u."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 8, start_paused: bool = False):
        h = _P()
        _check(load().ewald_server_create(int(hbm_budget_bytes), int(max_active), int(bool(start_paused)),
                                          ctypes.byref(h)), "ewald_server_create")
        self.handle = h.value
        self._keep = {}

    def submit(self, x, f, tol: float, L: float = 1.0, dtype: int = EWALD_F32_BULK, napplies: int = 20,
               perturb: float = 0.1, seed: int = 0) -> int:
        import numpy as np

        x = np.ascontiguousarray(x, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        if x.ndim != 2 or x.shape[1] != 3 or f.shape != x.shape:
            raise ValueError("x and f must be N x 3")
        u = np.empty_like(x)
        r = ewald_request(N=x.shape[0], L=float(L), tol=float(tol), dtype=int(dtype), napplies=int(napplies),
                          perturb=float(perturb), seed=int(seed), x_host=x.ctypes.data, f_host=f.ctypes.data,
                          u_host=u.ctypes.data)
        t = ctypes.c_int64(0)
        _check(load().ewald_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "ewald_server_submit")
        self._keep[t.value] = (x, f, u)
        return t.value

    def poll(self, ticket: int):
        st = ctypes.c_int32(0)
        lat = ctypes.c_double(0.0)
        code = load().ewald_server_poll(self.handle, int(ticket), ctypes.byref(st), ctypes.byref(lat))
        return st.value, lat.value, code

    def wait(self, ticket: int, timeout_s: float = 3600.0) -> int:
        """Status code: EWALD_OK, EWALD_ETIMEOUT, or the request's failure."""
        return load().ewald_server_wait(self.handle, int(ticket), float(timeout_s))

    def result(self, ticket: int):
        _check(self.wait(ticket), "ewald_server_wait")
        return self._keep.pop(ticket)[2]

    def cancel(self, ticket: int) -> int:
        return load().ewald_server_cancel(self.handle, int(ticket))

    def resume(self):
        _check(load().ewald_server_resume(self.handle), "ewald_server_resume")

    def stats(self) -> dict:
        out = ewald_server_summary()
        _check(load().ewald_server_stats(self.handle, ctypes.byref(out)), "ewald_server_stats")
        return out.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            load().ewald_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owner of one ewald_plan_t working on torch CUDA tensors (marshalling only)."""

    def __init__(self, N: int, L: float, tol: float, dtype: int = EWALD_F32_BULK, **override):
        ov = None
        if override:
            ov = ewald_params()
            for k, v in override.items():
                setattr(ov, k, v)
        self.N, self.L = int(N), float(L)
        self.handle = ewald_plan_ex(N, L, tol, dtype, ov)
        self.params = ewald_get_params(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            ewald_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        import torch

        s = stream if stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    def _check_arr(self, a, shape):
        import torch

        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous() and tuple(a.shape) == shape):
            raise ValueError(f"expected a contiguous float64 CUDA tensor of shape {shape}")

    def apply(self, x, f, out=None, stream=None):
        import torch

        self._check_arr(x, (self.N, 3))
        self._check_arr(f, (self.N, 3))
        u = out if out is not None else torch.empty_like(x)
        ewald_apply(self.handle, x.data_ptr(), f.data_ptr(), u.data_ptr(), self._stream(stream))
        return u

    def apply_combined(self, x, f, q, n, out=None, stream=None):
        """Stokeslet sum of f plus the double-layer sum of q (x) n (Sec. 2.3)."""
        import torch

        for a in (x, f, q, n):
            self._check_arr(a, (self.N, 3))
        u = out if out is not None else torch.empty_like(x)
        ewald_apply_combined(self.handle, x.data_ptr(), f.data_ptr(), q.data_ptr(), n.data_ptr(),
                             u.data_ptr(), self._stream(stream))
        return u

    def set_positions(self, x, stream=None):
        self._check_arr(x, (self.N, 3))
        ewald_set_positions(self.handle, x.data_ptr(), self._stream(stream))

    def apply_forces(self, f, out=None, stream=None):
        import torch

        self._check_arr(f, (self.N, 3))
        u = out if out is not None else torch.empty_like(f)
        ewald_apply_forces(self.handle, f.data_ptr(), u.data_ptr(), self._stream(stream))
        return u

    def near_field(self, x, f, stream=None):
        import torch

        u = torch.empty_like(x)
        ewald_near_field(self.handle, x.data_ptr(), f.data_ptr(), u.data_ptr(), self._stream(stream))
        return u

    def far_field(self, x, f, stream=None):
        import torch

        u = torch.empty_like(x)
        ewald_far_field(self.handle, x.data_ptr(), f.data_ptr(), u.data_ptr(), self._stream(stream))
        return u

    def spread(self, x, f, stream=None):
        import torch

        M = self.params.M
        g = torch.empty((3, M, M, M), dtype=torch.float64, device=x.device)
        ewald_spread(self.handle, x.data_ptr(), f.data_ptr(), g.data_ptr(), self._stream(stream))
        return g

    def interp(self, x, grid, stream=None):
        import torch

        u = torch.empty_like(x)
        ewald_interp(self.handle, x.data_ptr(), grid.data_ptr(), u.data_ptr(), self._stream(stream))
        return u

    def fourier_convolve(self, grid, stream=None):
        import torch

        out = torch.empty_like(grid)
        ewald_fourier_convolve(self.handle, grid.data_ptr(), out.data_ptr(), self._stream(stream))
        return out

    def sync_status(self, stream=None) -> int:
        return ewald_sync_status(self.handle, self._stream(stream))
