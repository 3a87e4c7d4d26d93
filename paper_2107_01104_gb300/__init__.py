"""GB300 tracer advection: Python binding of the C ABI in ``include/tracker.h``.

Argument marshalling only.  Every computation runs in the CUDA kernels of
``_build/libtracker.so``; there is no CPU fallback, and importing a function
that needs the library fails loudly if it has not been built
(``__graft_entry__.build()`` or ``python -m paper_2107_01104_gb300.build``).

Two layers:

* ``tracker_*`` functions with the same names and arguments as the C ABI
  (handles are ``ctypes.c_void_p``; array arguments are torch tensors);
* :class:`Tracker`, a small owner object over one handle.

Array conventions (see the header): positions ``pos[3][np]`` float64 on the
GPU, fields ``f[C][N][N][N]`` (x1 fastest), outputs ``out[C][np]``.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtracker.so")

TRK_OK, TRK_EINVAL, TRK_ENOMEM, TRK_ECUDA, TRK_ENONFINITE, TRK_ENOFIELD, TRK_ECFL, TRK_EIO = 0, -1, -2, -3, -4, -6, -7, -8
TRK_LAGRANGE, TRK_SPLINE = 0, 1
TRK_F64, TRK_F32, TRK_BF16X2 = 0, 1, 2
TRK_RK2, TRK_AB2, TRK_AB3, TRK_AB4 = 0, 1, 2, 3
TRK_DTYPE_F64, TRK_DTYPE_F32 = 0, 1
TRK_STEP_AUTO, TRK_STEP_BLOCK, TRK_STEP_COLUMN, TRK_STEP_DIRECT = 0, 1, 2, 3
TRK_HALO_AUTO, TRK_HALO_ASYNC, TRK_HALO_TMA = 0, 1, 2
TRK_TUNE_DEFAULT, TRK_TUNE_TIMED, TRK_TUNE_CACHED, TRK_TUNE_FIXED = 0, 1, 2, 3

_STATUS = {TRK_EINVAL: "EINVAL", TRK_ENOMEM: "ENOMEM", TRK_ECUDA: "ECUDA", TRK_ENONFINITE: "ENONFINITE",
           TRK_ENOFIELD: "ENOFIELD", TRK_ECFL: "ECFL", TRK_EIO: "EIO"}

# Every exported symbol of the ABI (checked against include/tracker.h by the tests).
ABI_FUNCTIONS = (
    "tracker_create", "tracker_destroy", "tracker_last_error", "tracker_set_stream", "tracker_sync",
    "tracker_set_field", "tracker_set_block", "tracker_num_blocks", "tracker_bin", "tracker_interpolate",
    "tracker_advance", "tracker_advance_batched", "tracker_adjoint", "tracker_launch_count",
    "tracker_profile", "tracker_profile_read", "tracker_bin_static", "tracker_set_step_kernel",
    "tracker_step_kernel_for", "tracker_state_write", "tracker_state_read_info", "tracker_state_read",
    "tracker_last_step_kernel",
    "tracker_field_texture", "tracker_probe_fma", "tracker_set_halo_copy", "tracker_halo_copy",
    "tracker_set_tuning", "tracker_get_tuning",
)


class TrackerError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class trk_state_info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("L", ctypes.c_double), ("family", ctypes.c_int32), ("I", ctypes.c_int32),
        ("m", ctypes.c_int32), ("np", ctypes.c_int64), ("scheme", ctypes.c_int32),
        ("history_valid", ctypes.c_int32), ("step", ctypes.c_int64), ("time", ctypes.c_double),
        ("dt", ctypes.c_double),
    ]


class trk_tuning(ctypes.Structure):
    _fields_ = [("step_kernel", ctypes.c_int), ("direct_block", ctypes.c_int), ("column_segment", ctypes.c_int),
                ("halo_copy", ctypes.c_int), ("direct_particles", ctypes.c_int), ("source", ctypes.c_int)]


class trk_set(ctypes.Structure):
    _fields_ = [
        ("np", ctypes.c_int64), ("pos", ctypes.c_void_p), ("rhs", ctypes.c_void_p), ("out", ctypes.c_void_p),
        ("family", ctypes.c_int), ("I", ctypes.c_int), ("m", ctypes.c_int), ("deriv", ctypes.c_int),
    ]


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtracker.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        c_int, c_i64, c_d, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        sig = {
            "tracker_create": (c_int, [ctypes.POINTER(vp), c_int, c_d, c_int, c_int, c_int, c_int, vp]),
            "tracker_destroy": (c_int, [vp]),
            "tracker_last_error": (ctypes.c_char_p, []),
            "tracker_set_stream": (c_int, [vp, vp]),
            "tracker_sync": (c_int, [vp]),
            "tracker_set_field": (c_int, [vp, vp, c_int, c_int, c_int]),
            "tracker_set_block": (c_int, [vp, c_int, c_int, c_int]),
            "tracker_num_blocks": (c_i64, [vp]),
            "tracker_bin": (c_int, [vp, c_i64, vp, vp, vp, vp]),
            "tracker_interpolate": (c_int, [vp, c_i64, vp, vp, c_int, c_int]),
            "tracker_advance": (c_int, [vp, c_i64, vp, vp, c_d, c_int, c_int, c_int]),
            "tracker_advance_batched": (c_int, [vp, c_int, vp, c_d, c_int, c_int]),
            "tracker_adjoint": (c_int, [vp, c_i64, vp, vp, c_d, c_int, c_int, vp, vp]),
            "tracker_launch_count": (c_i64, [vp]),
            "tracker_profile": (c_int, [vp, c_int]),
            "tracker_profile_read": (c_int, [vp, vp, vp]),
            "tracker_bin_static": (c_int, [c_i64, vp, c_int, c_d, c_int, c_int, c_int, vp, vp, vp, vp, vp]),
            "tracker_set_step_kernel": (c_int, [vp, c_int]),
            "tracker_step_kernel_for": (c_int, [vp, c_i64]),
            "tracker_last_step_kernel": (c_int, [vp]),
            "tracker_field_texture": (c_int, [vp]),
            "tracker_probe_fma": (c_int, [c_int, vp]),
            "tracker_set_halo_copy": (c_int, [vp, c_int]),
            "tracker_set_tuning": (c_int, [vp, vp]),
            "tracker_get_tuning": (c_int, [vp, vp]),
            "tracker_halo_copy": (c_int, [vp, c_int]),
            "tracker_state_write": (c_int, [ctypes.c_char_p, vp, vp, vp]),
            "tracker_state_read_info": (c_int, [ctypes.c_char_p, vp]),
            "tracker_state_read": (c_int, [ctypes.c_char_p, c_i64, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def tracker_last_error() -> str:
    return load_library().tracker_last_error().decode()


def _check(rc: int):
    if rc != TRK_OK:
        raise TrackerError(rc, tracker_last_error())


def _ptr(x):
    if x is None:
        return None
    return ctypes.c_void_p(x.data_ptr())


def _stream_ptr(device=None):
    if not torch.cuda.is_available():
        return ctypes.c_void_p(None)
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev(x, dtype, name, shape0=None, device=None, numel=None, min_numel=None):
    """Checks a device array argument: dtype, on the GPU (on `device` if given),
    contiguous, and optionally its leading dimension or element count."""
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_cuda:
        raise ValueError(f"{name} must be on the GPU")
    if device is not None and x.device != device:
        raise ValueError(f"{name} must be on {device}, got {x.device}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape0 is not None and (x.dim() != 2 or x.shape[0] != shape0):
        raise ValueError(f"{name} must have shape ({shape0}, n), got {tuple(x.shape)}")
    if numel is not None and x.numel() != numel:
        raise ValueError(f"{name} must hold {numel} values, got {x.numel()}")
    if min_numel is not None and x.numel() < min_numel:
        raise ValueError(f"{name} must hold at least {min_numel} values, got {x.numel()}")
    return x


# --------------------------------------------------------------------------
# Same-name functions (one per C entry point)
# --------------------------------------------------------------------------
def tracker_create(N, L=2 * math.pi, family=TRK_SPLINE, I=6, m=2, storage=TRK_F32, stream=None):
    h = ctypes.c_void_p()
    st = ctypes.c_void_p(stream) if stream is not None else _stream_ptr()
    _check(load_library().tracker_create(ctypes.byref(h), int(N), float(L), int(family), int(I), int(m),
                                         int(storage), st))
    return h


def tracker_destroy(h):
    _check(load_library().tracker_destroy(h))


def tracker_set_stream(h, stream=None):
    st = ctypes.c_void_p(stream) if stream is not None else _stream_ptr()
    _check(load_library().tracker_set_stream(h, st))


def tracker_sync(h):
    _check(load_library().tracker_sync(h))


def tracker_set_field(h, field: torch.Tensor):
    if field.dtype not in (torch.float64, torch.float32):
        raise TypeError("field must be float32 or float64")
    if not field.is_contiguous() or field.dim() != 4:
        raise ValueError("field must be a contiguous [C][N][N][N] tensor")
    dt = TRK_DTYPE_F64 if field.dtype == torch.float64 else TRK_DTYPE_F32
    on_host = 0 if field.is_cuda else 1
    _check(load_library().tracker_set_field(h, _ptr(field), int(field.shape[0]), dt, on_host))


def tracker_set_block(h, bx, by, bz):
    _check(load_library().tracker_set_block(h, int(bx), int(by), int(bz)))


def tracker_set_step_kernel(h, kind):
    _check(load_library().tracker_set_step_kernel(h, int(kind)))


def tracker_step_kernel_for(h, np_) -> int:
    """The step kernel (TRK_STEP_COLUMN / BLOCK / DIRECT) tracker_advance uses for np_ particles."""
    r = int(load_library().tracker_step_kernel_for(h, int(np_)))
    _check(min(r, 0))
    return r


def _host_copy(x, dtype, rows, np_, name):
    """A contiguous host copy of a [rows][np] (or [k][3][np]) array."""
    if x is None:
        raise ValueError(f"{name} is required")
    t = torch.as_tensor(x)
    if t.dtype != dtype or t.numel() != rows * np_:
        raise ValueError(f"{name} must be {dtype} with {rows} x {np_} values")
    return t.detach().to("cpu").contiguous()


def tracker_state_write(path, pos, rhs=None, scheme=TRK_RK2, history_valid=0, step=0, time=0.0, dt=0.0,
                        N=0, L=0.0, family=0, I=0, m=0):
    """Write a tracer set (pos [3][np] float64, rhs [k-1][3][np] float32 for ABk) to a state file."""
    np_ = int(torch.as_tensor(pos).shape[-1])
    rows = 3 * int(scheme) if scheme in (TRK_AB2, TRK_AB3, TRK_AB4) else 0   # other values: the library rejects them
    hp = _host_copy(pos, torch.float64, 3, np_, "pos")
    hr = _host_copy(rhs, torch.float32, rows, np_, "rhs") if rows else None
    info = trk_state_info(N=int(N), L=float(L), family=int(family), I=int(I), m=int(m), np=np_,
                          scheme=int(scheme), history_valid=int(history_valid), step=int(step), time=float(time),
                          dt=float(dt))
    _check(load_library().tracker_state_write(os.fsencode(path), ctypes.byref(info), _ptr(hp), _ptr(hr)))


def tracker_state_read_info(path) -> dict:
    info = trk_state_info()
    _check(load_library().tracker_state_read_info(os.fsencode(path), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in trk_state_info._fields_}


def tracker_state_read(path, device=None):
    """(pos [3][np] float64, rhs [k-1][3][np] float32 or None, info dict) from a state file."""
    meta = tracker_state_read_info(path)
    np_, scheme = meta["np"], meta["scheme"]
    pos = torch.empty((3, np_), dtype=torch.float64)
    rhs = torch.empty((scheme, 3, np_), dtype=torch.float32) if scheme != TRK_RK2 else None
    info = trk_state_info()
    _check(load_library().tracker_state_read(os.fsencode(path), np_, _ptr(pos), _ptr(rhs), ctypes.byref(info)))
    meta = {f: getattr(info, f) for f, _ in trk_state_info._fields_}
    if device is not None:
        pos = pos.to(device)
        rhs = rhs.to(device) if rhs is not None else None
    return pos, rhs, meta


def tracker_num_blocks(h) -> int:
    return int(load_library().tracker_num_blocks(h))


def tracker_launch_count(h) -> int:
    return int(load_library().tracker_launch_count(h))


def tracker_profile(h, enable: bool):
    _check(load_library().tracker_profile(h, int(bool(enable))))


def tracker_profile_read(h):
    """{'step': (ms, launches), 'bin': (...), 'other': (...)} of device time since tracker_profile(h, True)."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 3)()
    _check(load_library().tracker_profile_read(h, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(n, ctypes.c_void_p)))
    return {"step": (ms[0], n[0]), "bin": (ms[1], n[1]), "other": (ms[2], n[2])}


def _bin_outputs(dev, n, nb, keys, perm, offsets):
    """Caller-given (or new) int32 outputs of a binning call, checked against the
    sizes the kernels write: keys and perm n entries, offsets nb + 1."""
    keys = torch.empty(n, dtype=torch.int32, device=dev) if keys is None else keys
    perm = torch.empty(n, dtype=torch.int32, device=dev) if perm is None else perm
    offsets = torch.empty(nb + 1, dtype=torch.int32, device=dev) if offsets is None else offsets
    _dev(keys, torch.int32, "keys", device=dev, numel=n)
    _dev(perm, torch.int32, "perm", device=dev, numel=n)
    _dev(offsets, torch.int32, "offsets", device=dev, numel=nb + 1)
    return keys, perm, offsets


def tracker_probe_fma(dtype=TRK_DTYPE_F32) -> float:
    """Measured fused multiply-adds per second of the current GPU (float32 or float64)."""
    r = ctypes.c_double(0.0)
    _check(load_library().tracker_probe_fma(int(dtype), ctypes.byref(r)))
    return r.value


def tracker_bin(h, pos, keys=None, perm=None, offsets=None):
    pos = _dev(pos, torch.float64, "pos", 3)
    n = pos.shape[1]
    keys, perm, offsets = _bin_outputs(pos.device, n, tracker_num_blocks(h), keys, perm, offsets)
    with torch.cuda.device(pos.device):
        _check(load_library().tracker_bin(h, n, _ptr(pos), _ptr(keys), _ptr(perm), _ptr(offsets)))
    return keys, perm, offsets


def tracker_bin_static(pos, N, L=2 * math.pi, block=(8, 8, 8), keys=None, perm=None, offsets=None,
                       nonfinite=None, stream=None):
    """Allocation-free binning (see include/tracker.h); outputs are caller tensors."""
    pos = _dev(pos, torch.float64, "pos", 3)
    n = pos.shape[1]
    dev = pos.device
    if any(int(b) <= 0 or int(N) % int(b) for b in block):
        raise ValueError(f"block edges {tuple(block)} must divide N={N}")
    nb = (N // block[0]) * (N // block[1]) * (N // block[2])
    keys, perm, offsets = _bin_outputs(dev, n, nb, keys, perm, offsets)
    if nonfinite is not None:
        _dev(nonfinite, torch.int32, "nonfinite", device=dev, min_numel=1)
    with torch.cuda.device(dev):
        st = ctypes.c_void_p(stream) if stream is not None else _stream_ptr(dev)
        _check(load_library().tracker_bin_static(n, _ptr(pos), int(N), float(L), int(block[0]), int(block[1]),
                                                 int(block[2]), _ptr(keys), _ptr(perm), _ptr(offsets),
                                                 _ptr(nonfinite), st))
    return keys, perm, offsets


def tracker_interpolate(h, pos, C, out=None, out_dtype=torch.float32, deriv=False):
    pos = _dev(pos, torch.float64, "pos", 3)
    n = pos.shape[1]
    rows = 3 * C if deriv else C
    if out is None:
        out = torch.empty((rows, n), dtype=out_dtype, device=pos.device)
    _dev(out, out.dtype, "out", rows)
    code = TRK_DTYPE_F64 if out.dtype == torch.float64 else TRK_DTYPE_F32
    _check(load_library().tracker_interpolate(h, n, _ptr(pos), _ptr(out), code, int(bool(deriv))))
    return out


def tracker_advance(h, pos, dt, steps, scheme=TRK_RK2, rhs=None, history_valid=0):
    """RK2 or ABk (k = scheme + 1).  rhs: AB history, [k-1][3][np] float32 on the
    device (AB2 also [3][np]); history_valid: valid entries on entry (True = 1)."""
    pos = _dev(pos, torch.float64, "pos", 3)
    if rhs is not None:
        k = scheme + 1
        if rhs.dtype != torch.float32 or not rhs.is_cuda or not rhs.is_contiguous():
            raise ValueError("rhs must be a contiguous float32 CUDA tensor")
        if rhs.numel() != (k - 1) * 3 * pos.shape[1]:
            raise ValueError(f"rhs must hold {k - 1} x 3 x np values for AB{k}")
    _check(load_library().tracker_advance(h, pos.shape[1], _ptr(pos), _ptr(rhs), float(dt), int(steps),
                                          int(scheme), int(history_valid)))
    return pos


def tracker_advance_batched(h, sets, dt, steps, history_valid=False):
    arr = (trk_set * len(sets))()
    for i, s in enumerate(sets):
        pos = _dev(s["pos"], torch.float64, "pos", 3)
        rhs = _dev(s["rhs"], torch.float32, "rhs", 3)
        out = s.get("out")
        arr[i].np = pos.shape[1]
        arr[i].pos = pos.data_ptr()
        arr[i].rhs = rhs.data_ptr()
        arr[i].out = out.data_ptr() if out is not None else None
        arr[i].family = int(s.get("family", TRK_SPLINE))
        arr[i].I = int(s["I"])
        arr[i].m = int(s.get("m", s["I"] // 2 - 1))
        arr[i].deriv = int(bool(s.get("deriv", False)))
    _check(load_library().tracker_advance_batched(h, len(sets), ctypes.cast(arr, ctypes.c_void_p), float(dt),
                                                  int(steps), int(bool(history_valid))))


def tracker_adjoint(h, pos0, lambdaT, dt, steps, ckpt_every=5, grad_pos0=None, grad_field=None):
    pos0 = _dev(pos0, torch.float64, "pos0", 3)
    lambdaT = _dev(lambdaT, torch.float64, "lambdaT", 3)
    if grad_pos0 is None:
        grad_pos0 = torch.empty_like(pos0)
    if grad_field is not None:
        _dev(grad_field, torch.float64, "grad_field")
    _check(load_library().tracker_adjoint(h, pos0.shape[1], _ptr(pos0), _ptr(lambdaT), float(dt), int(steps),
                                          int(ckpt_every), _ptr(grad_pos0), _ptr(grad_field)))
    return grad_pos0, grad_field


# --------------------------------------------------------------------------
# Owner object
# --------------------------------------------------------------------------
class Tracker:
    """One tracker handle: an N^3 periodic grid with a kernel (family, I, m) and a field."""

    def __init__(self, N, L=2 * math.pi, family=TRK_SPLINE, I=6, m=None, storage=TRK_F32, device=None):
        if m is None:
            m = I // 2 - 1 if family == TRK_SPLINE else 0
        self.N, self.L, self.family, self.I, self.m, self.storage = N, L, family, I, m, storage
        self.C = 0
        # every call runs with this device current (the library checks it)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.field_generation = 0     # bumped by every set_field (autograd checks it)
        self.h = None
        with torch.cuda.device(self.device):
            self.h = tracker_create(N, L, family, I, m, storage, stream=_stream_ptr(self.device).value)

    def close(self):
        if self.h is not None:
            tracker_destroy(self.h)   # the library switches to the tracker's device itself
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

    def _stream(self):
        tracker_set_stream(self.h, _stream_ptr(self.device).value)

    def _on_device(self):
        return torch.cuda.device(self.device)

    def set_field(self, field):
        with self._on_device():
            self._stream()
            tracker_set_field(self.h, field)
        self.C = int(field.shape[0])
        self.field_generation += 1

    def set_step_kernel(self, kind):
        """TRK_STEP_AUTO, _BLOCK, _COLUMN or _DIRECT (see tracker_set_step_kernel)."""
        tracker_set_step_kernel(self.h, kind)

    def step_kernel_for(self, np_):
        return tracker_step_kernel_for(self.h, np_)

    def last_step_kernel(self):
        """The kernel the latest advance or interpolate used (after AUTO's timing)."""
        r = int(load_library().tracker_last_step_kernel(self.h))
        _check(min(r, 0))
        return r

    def set_tuning(self, step_kernel=None, direct_block=8, column_segment=8, halo_copy=TRK_HALO_TMA,
                   direct_particles=256):
        """Fix the time-step launch shape (see tracker_set_tuning); no arguments: automatic tuning."""
        if step_kernel is None:
            _check(load_library().tracker_set_tuning(self.h, None))
            return
        p = trk_tuning(step_kernel=int(step_kernel), direct_block=int(direct_block),
                       column_segment=int(column_segment), halo_copy=int(halo_copy),
                       direct_particles=int(direct_particles), source=0)
        _check(load_library().tracker_set_tuning(self.h, ctypes.byref(p)))

    def tuning(self):
        """The launch shape the latest advance ran with and how it was chosen (a dict)."""
        p = trk_tuning()
        _check(load_library().tracker_get_tuning(self.h, ctypes.byref(p)))
        return {f: getattr(p, f) for f, _ in trk_tuning._fields_}

    def set_halo_copy(self, kind):
        """TRK_HALO_AUTO, _ASYNC or _TMA: how the block kernel stages its field halos."""
        _check(load_library().tracker_set_halo_copy(self.h, int(kind)))

    def halo_copy(self, rk2=False):
        """The halo copy the block kernel uses now (TRK_HALO_ASYNC or TRK_HALO_TMA)."""
        r = int(load_library().tracker_halo_copy(self.h, int(bool(rk2))))
        _check(min(r, 0))
        return r

    def field_texture(self):
        """True if the direct kernel reads the node-major field copy through a texture object."""
        r = int(load_library().tracker_field_texture(self.h))
        _check(min(r, 0))
        return bool(r)

    def save_state(self, path, pos, rhs=None, scheme=TRK_RK2, history_valid=0, step=0, time=0.0, dt=0.0):
        """Checkpoint a tracer set with this tracker's grid and kernel in the header."""
        tracker_state_write(path, pos, rhs, scheme, history_valid, step, time, dt, self.N, self.L, self.family,
                            self.I, self.m)

    def load_state(self, path, device="cuda"):
        """Read a checkpoint written for the same grid and kernel: (pos, rhs, info)."""
        pos, rhs, info = tracker_state_read(path, device)
        mine = (self.N, self.family, self.I, self.m)
        theirs = (info["N"], info["family"], info["I"], info["m"])
        if mine != theirs or abs(info["L"] - self.L) > 0:
            raise ValueError(f"state file was written for (N, family, I, m, L) = {theirs + (info['L'],)}")
        return pos, rhs, info

    def bin(self, pos):
        with self._on_device():
            self._stream()
            return tracker_bin(self.h, pos)

    def interpolate(self, pos, out_dtype=torch.float32, deriv=False, out=None):
        with self._on_device():
            self._stream()
            return tracker_interpolate(self.h, pos, self.C, out=out, out_dtype=out_dtype, deriv=deriv)

    def advance(self, pos, dt, steps, scheme=TRK_RK2, rhs=None, history_valid=False):
        with self._on_device():
            self._stream()
            return tracker_advance(self.h, pos, dt, steps, scheme, rhs, history_valid)

    def advance_batched(self, sets, dt, steps, history_valid=False):
        with self._on_device():
            self._stream()
            tracker_advance_batched(self.h, sets, dt, steps, history_valid)

    def adjoint(self, pos0, lambdaT, dt, steps, ckpt_every=5, grad_field=None):
        with self._on_device():
            self._stream()
            return tracker_adjoint(self.h, pos0, lambdaT, dt, steps, ckpt_every, grad_field=grad_field)

    def sync(self):
        with self._on_device():
            tracker_sync(self.h)

    @property
    def launch_count(self):
        return tracker_launch_count(self.h)

    @property
    def num_blocks(self):
        return tracker_num_blocks(self.h)
