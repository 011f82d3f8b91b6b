"""Seeded synthetic SU(3) gauge fields (input generator only).

The recipe, from the workload description of the method's experiments: links
U_mu(x) = exp(i eps sum_a r_a lambda_a / 2) with r_a ~ N(0, 1), followed by a
Haar-random gauge transformation h(x) U_mu(x) h(x+mu)^dagger.  eps = 0 gives
a pure-gauge field.  Both the FP64 oracle's tests and the CUDA path draw their
inputs from here; this module holds none of the gauge-fixing arithmetic.

Link layout (complex128, shape ``(N_t, N_3, N_2, N_1, 4, 3, 3)``): site index
``x1 + N1*(x2 + N2*(x3 + N3*t))``, direction 0 is t and 1..3 are x1..x3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fieldgen.c")
_LIB = os.path.join(_HERE, "libfieldgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator into an in-tree shared library; returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
             _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.lgtgen_field.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_void_p]
            lib.lgtgen_field.restype = ctypes.c_int
            lib.lgtgen_field_threads.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_double,
                                                 ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
            lib.lgtgen_field_threads.restype = ctypes.c_int
            lib.lgtgen_haar.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            lib.lgtgen_haar.restype = ctypes.c_int
            lib.lgtgen_philox.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            lib.lgtgen_philox.restype = None
            _lib = lib
    return _lib


def field(dims, eps: float, seed: int, threads: int = 0) -> np.ndarray:
    """Synthetic links for ``dims = (N_t, N_3, N_2, N_1)`` as complex128 of shape
    ``(N_t, N_3, N_2, N_1, 4, 3, 3)`` (C-contiguous), generated on ``threads``
    OpenMP threads (0: the default team; the values do not depend on it)."""
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or min(dims) < 1:
        raise ValueError(f"bad dims {dims}")
    out = np.empty(dims + (4, 3, 3), dtype=np.complex128)
    d = (ctypes.c_int32 * 4)(*dims)
    rc = _load().lgtgen_field_threads(d, float(eps), int(seed) & (2**64 - 1), out.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError(f"lgtgen_field failed ({rc})")
    return out


def haar(seed: int, count: int) -> np.ndarray:
    """``count`` Haar-random SU(3) matrices, shape ``(count, 3, 3)``."""
    out = np.empty((int(count), 3, 3), dtype=np.complex128)
    _load().lgtgen_haar(int(seed) & (2**64 - 1), int(count), out.ctypes.data)
    return out


def philox(ctr, key):
    """One Philox4x32-10 block of the generator's own implementation."""
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    _load().lgtgen_philox(c, k, o)
    return tuple(int(v) for v in o)
