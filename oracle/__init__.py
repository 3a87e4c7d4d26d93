"""FP64 CPU oracle for the tracer-advection hot path (test infrastructure).

This package is the slow, obviously-correct reference against which the CUDA
library is checked.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product path never does.  It
shares no code with the CUDA library: it has its own C source
(``oracle.c``), built with plain gcc, and the numpy glue below.

Functions and the passage of arXiv:2107.01104 each one follows:

* :func:`split`        -- Sec. 2.2, interpolation steps 1-3 (X mod 2pi, cell, offset)
* :func:`weights`      -- Sec. 2.2 kernels beta_i: Lagrange (product form) and the
                          spline family of [lalescu2010jcp] (read as a C^m Hermite
                          construction, built procedurally)
* :func:`bin_particles`-- Sec. 3.3.1, slice/block ordering with an ``offset`` array
* :func:`interp`       -- Sec. 2.2 step 4, Eq. (triple_sum), direct quadruple loop
* :func:`advance`      -- Eq. (tracers) with RK2 (Heun) or AB2/AB3/AB4 (Sec. 2.2, 3.3.1)
* :func:`adjoint_rk2`  -- discrete adjoint of the RK2 map (no counterpart in the paper)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

LAGRANGE, SPLINE = 0, 1
RK2, AB2, AB3, AB4 = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (OpenMP, no FP contraction) into ``_build/``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            p = ctypes.c_void_p
            lib.orc_split.argtypes = [i64, p, i, d, p, p]
            lib.orc_weights.argtypes = [i, i, i, d, p, p]
            lib.orc_check_kernel.argtypes = [i, i, i]
            lib.orc_bin.argtypes = [i64, p, i, d, i, i, i, p, p, p]
            lib.orc_interp.argtypes = [i, i, i, i, d, p, i, i64, p, p, i]
            lib.orc_interp_stencil.argtypes = [i, i, i, i, i64, p, p, p]
            lib.orc_advance.argtypes = [i, i, i, i, d, p, i64, p, p, d, i, i, i]
            lib.orc_adjoint_rk2.argtypes = [i, i, i, i, d, p, i64, p, p, d, i, p, p]
            lib.orc_inv_delta.argtypes = [i, d]
            lib.orc_inv_delta.restype = d
            lib.orc_num_threads.restype = i
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc == -4:
        raise FloatingPointError(f"oracle {what}: non-finite position")
    if rc != 0:
        raise ValueError(f"oracle {what}: error {rc}")


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().orc_num_threads())


def inv_delta(N: int, L: float = 2 * np.pi) -> float:
    return float(_load().orc_inv_delta(N, L))


def split(pos, N: int, L: float = 2 * np.pi):
    """Cell index c[3][np] (int32, in [0,N)) and offset t[3][np] in [0,1] (Sec. 2.2 steps 1-3)."""
    pos = _f64(pos)
    np_ = pos.shape[1]
    cell = np.empty((3, np_), np.int32)
    frac = np.empty((3, np_), np.float64)
    _check(_load().orc_split(np_, _ptr(pos), N, L, _ptr(cell), _ptr(frac)), "split")
    return cell, frac


def weights(family: int, I: int, m: int, t: float, deriv: bool = False):
    """beta_i(t) (and beta_i'(t)) for nodes i = 1-I/2 .. I/2."""
    b = np.empty(I, np.float64)
    db = np.empty(I, np.float64)
    rc = _load().orc_weights(family, I, m, float(t), _ptr(b), _ptr(db))
    _check(rc, "weights")
    return (b, db) if deriv else b


def bin_particles(pos, N: int, B=(8, 8, 8), L: float = 2 * np.pi):
    """Stable counting sort by block key (Sec. 3.3.1).  Returns keys, perm, offsets."""
    pos = _f64(pos)
    np_ = pos.shape[1]
    B1, B2, B3 = B
    nblocks = (N // B1) * (N // B2) * (N // B3)
    keys = np.empty(np_, np.int32)
    perm = np.empty(np_, np.int64)
    offsets = np.empty(nblocks + 1, np.int64)
    rc = _load().orc_bin(np_, _ptr(pos), N, L, B1, B2, B3, _ptr(keys), _ptr(perm), _ptr(offsets))
    _check(rc, "bin")
    return keys, perm, offsets


def interp(field, pos, family: int, I: int, m: int = 0, L: float = 2 * np.pi, deriv: bool = False):
    """Eq. (triple_sum) at every particle.  field[C][N][N][N], pos[3][np].

    Returns out[C][np], or out[C][3][np] (d u_k / d X_j) when ``deriv``.
    """
    field = _f64(field)
    pos = _f64(pos)
    C, N = field.shape[0], field.shape[-1]
    np_ = pos.shape[1]
    out = np.empty((C * 3 if deriv else C, np_), np.float64)
    rc = _load().orc_interp(family, I, m, N, L, _ptr(field), C, np_, _ptr(pos), _ptr(out), int(deriv))
    _check(rc, "interp")
    return out.reshape(C, 3, np_) if deriv else out


def interp_stencil(frac, stencil, family: int, I: int, m: int = 0):
    """Eq. (triple_sum) from pre-gathered stencils stencil[np][C][I][I][I] and offsets frac[3][np]."""
    frac = _f64(frac)
    stencil = _f64(stencil)
    np_, C = stencil.shape[0], stencil.shape[1]
    out = np.empty((C, np_), np.float64)
    rc = _load().orc_interp_stencil(family, I, m, C, np_, _ptr(frac), _ptr(stencil), _ptr(out))
    _check(rc, "interp_stencil")
    return out


def advance(field, pos, dt: float, steps: int, family: int, I: int, m: int = 0, scheme: int = RK2,
            rhs=None, history_valid=0, L: float = 2 * np.pi):
    """Integrate Eq. (tracers) for ``steps`` steps.

    RK2 returns the new positions.  ABk (AB2, AB3, AB4: k = scheme + 1)
    returns (positions, rhs): rhs holds the k-1 newest u, [k-1][3][np]
    (AB2: [3][np]), u_{n-1} first; ``history_valid`` entries of the given rhs
    are valid on entry (True counts as 1).
    """
    field = _f64(field)
    pos = _f64(pos).copy()
    N = field.shape[-1]
    np_ = pos.shape[1]
    k = 0 if scheme == RK2 else scheme + 1
    if k:
        rhs = np.zeros((k - 1, 3, np_)) if rhs is None else _f64(rhs).reshape(k - 1, 3, np_).copy()
    rc = _load().orc_advance(family, I, m, N, L, _ptr(field), np_, _ptr(pos), _ptr(rhs) if k else None,
                             float(dt), int(steps), int(scheme), int(history_valid))
    _check(rc, "advance")
    if not k:
        return pos
    return pos, (rhs[0] if k == 2 else rhs)


def adjoint_rk2(field, pos0, lambdaT, dt: float, steps: int, family: int, I: int, m: int = 0,
                with_field: bool = True, L: float = 2 * np.pi):
    """Discrete adjoint of ``steps`` RK2 steps: (dLoss/dX0, dLoss/dfield)."""
    field = _f64(field)
    pos0 = _f64(pos0)
    lam = _f64(lambdaT)
    N = field.shape[-1]
    np_ = pos0.shape[1]
    gpos = np.empty((3, np_), np.float64)
    gfield = np.zeros_like(field) if with_field else None
    rc = _load().orc_adjoint_rk2(family, I, m, N, L, _ptr(field), np_, _ptr(pos0), _ptr(lam),
                                 float(dt), int(steps), _ptr(gpos), _ptr(gfield))
    _check(rc, "adjoint")
    return gpos, gfield
