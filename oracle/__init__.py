"""CPU oracle for the correlator X stage -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It wraps ``liboracle.so`` (plain C, ``xcorr_oracle.c``), which
computes, per channel c and input pair i <= j,

    V_ij(c) = sum_t x_i(c, t) * conj(x_j(c, t))       (Sec. 2; Sec. 4, Fig. 2)

in int64 for 4/8-bit integer samples and in float64 for float32 samples.  Output is
``[n_sel_chan][P][2]`` with baseline b = i*N - i*(i-1)/2 + (j-i).  The oracle shares no
code with the CUDA library.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests (brute
force, a library special case, Hermitian symmetry, closed forms, additivity and the
int32-overflow edge).  None is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_baseline_index.restype = ctypes.c_int64
        L.oracle_baseline_index.argtypes = [ctypes.c_int64] * 3
        L.oracle_n_baselines.restype = ctypes.c_int64
        L.oracle_n_baselines.argtypes = [ctypes.c_int64]
        L.oracle_unpack.restype = ctypes.c_int
        L.oracle_unpack.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_threads_used.restype = ctypes.c_int
        L.oracle_threads_used.argtypes = [ctypes.c_int]
        L.oracle_xcorr_int.restype = ctypes.c_int
        L.oracle_xcorr_int.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        L.oracle_xcorr_f64.restype = ctypes.c_int
        L.oracle_xcorr_f64.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        _lib = L
    return _lib


def n_baselines(n_inputs: int) -> int:
    return int(lib().oracle_n_baselines(n_inputs))


def baseline_index(n_inputs: int, i: int, j: int) -> int:
    return int(lib().oracle_baseline_index(n_inputs, i, j))


def threads_used(requested: int = 0) -> int:
    return int(lib().oracle_threads_used(requested))


def unpack(packed: np.ndarray, n_inputs: int, n_chan: int, n_time: int, bits: int):
    """Oracle unpack of a packed [T][C][N] block -> (re, im) int32 arrays of shape [T][C][N]."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    re = np.empty((n_time, n_chan, n_inputs), dtype=np.int32)
    im = np.empty_like(re)
    st = lib().oracle_unpack(packed.ctypes.data, n_inputs, n_chan, n_time, bits, re.ctypes.data, im.ctypes.data)
    if st:
        raise ValueError(f"oracle_unpack failed ({st})")
    return re, im


def xcorr_int(packed: np.ndarray, n_inputs: int, n_chan: int, n_time: int, bits: int,
              chans=None, n_threads: int = 0) -> np.ndarray:
    """int64 visibilities ``[n_sel][P][2]`` of a packed 4/8-bit block (chans=None: all channels)."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    need = n_time * n_chan * n_inputs * (1 if bits == 4 else 2)
    if packed.size < need:
        raise ValueError("packed buffer too small")
    P = n_inputs * (n_inputs + 1) // 2
    if chans is None:
        sel = None
        n_sel = n_chan
    else:
        sel = np.ascontiguousarray(chans, dtype=np.int32)
        n_sel = int(sel.size)
    vis = np.zeros((n_sel, P, 2), dtype=np.int64)
    st = lib().oracle_xcorr_int(packed.ctypes.data, n_inputs, n_chan, n_time, bits,
                                None if sel is None else sel.ctypes.data, n_sel, vis.ctypes.data, n_threads)
    if st:
        raise ValueError(f"oracle_xcorr_int failed ({st})")
    return vis


def xcorr_f64(samples: np.ndarray, n_inputs: int, n_chan: int, n_time: int,
              chans=None, n_threads: int = 0) -> np.ndarray:
    """float64 visibilities ``[n_sel][P][2]`` of float32 samples ``[T][C][N][2]``."""
    x = np.ascontiguousarray(samples, dtype=np.float32)
    if x.size < n_time * n_chan * n_inputs * 2:
        raise ValueError("sample buffer too small")
    P = n_inputs * (n_inputs + 1) // 2
    if chans is None:
        sel = None
        n_sel = n_chan
    else:
        sel = np.ascontiguousarray(chans, dtype=np.int32)
        n_sel = int(sel.size)
    vis = np.zeros((n_sel, P, 2), dtype=np.float64)
    st = lib().oracle_xcorr_f64(x.ctypes.data, n_inputs, n_chan, n_time,
                                None if sel is None else sel.ctypes.data, n_sel, vis.ctypes.data, n_threads)
    if st:
        raise ValueError(f"oracle_xcorr_f64 failed ({st})")
    return vis
