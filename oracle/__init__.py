"""X-engine oracle -- TEST INFRASTRUCTURE ONLY.

A plain CPU restatement of the correlator's X-engine (arXiv:1904.07778,
Sec. 2 "System Design" and Sec. 2.2 "X-engine"): for every channel c and
every input pair j <= i, V[c][i][j] = sum_t x_i(c,t) conj(x_j(c,t)) in exact
int64.  The arithmetic lives in ``xcorr_oracle.c``; this module only builds
and marshals.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It imports nothing from the
CUDA package and the CUDA package imports nothing from here.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against
hand-evaluated values, closed forms, invariants and the paper's own
identities (FX == XF, Sec. 2; the delay test, Sec. 3, Eq. 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xcorr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

L_TCI, L_TIC, L_CIT = 0, 1, 2
ERANGE = -4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_correlate.argtypes = [P, I, I, I, I, I, I, P, I, P, I]
            lib.oracle_decode.argtypes = [P, I, I, I, I, I, I, P, P]
            lib.oracle_correlate_cd.argtypes = [P, I, I, I, P]
            lib.oracle_normalise.argtypes = [P, I, I, P, P]
            lib.oracle_projected_power.argtypes = [P, I, I, I, I, I, I, P, I, P, I, P, I]
            for f in (lib.oracle_correlate, lib.oracle_decode, lib.oracle_correlate_cd,
                      lib.oracle_normalise, lib.oracle_projected_power):
                f.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def n_baselines(n_inputs: int) -> int:
    return n_inputs * (n_inputs + 1) // 2


class OracleRangeError(ValueError):
    """An 8-bit sample equal to -128 (outside the symmetric quantiser)."""


def correlate(block, n_inputs, n_chans, n_time, bits=4, layout=L_TCI, hi_is_real=True,
              chans=None, threads=None, out=None, check_range=True):
    """Visibilities of one packed block: int64 array [n_chans or len(chans)][B][2].

    If ``out`` is given it is accumulated into (+=), else a zeroed array is made.
    """
    lib = _load()
    blk = np.ascontiguousarray(np.frombuffer(memoryview(block), dtype=np.uint8)
                               if not isinstance(block, np.ndarray) else block.view(np.uint8).reshape(-1))
    need = n_inputs * n_chans * n_time * (bits // 4)
    if blk.size != need:
        raise ValueError("block has %d bytes, expected %d" % (blk.size, need))
    ch = None
    nch = n_chans
    if chans is not None:
        ch = np.ascontiguousarray(np.asarray(chans, dtype=np.int32))
        nch = ch.size
    nb = n_baselines(n_inputs)
    if out is None:
        out = np.zeros((nch, nb, 2), dtype=np.int64)
    assert out.dtype == np.int64 and out.flags.c_contiguous and out.shape == (nch, nb, 2)
    if threads is None:
        threads = os.cpu_count() or 1
    st = lib.oracle_correlate(_ptr(blk), layout, bits, 1 if hi_is_real else 0, n_inputs, n_chans,
                              n_time, _ptr(ch) if ch is not None else None, nch, _ptr(out),
                              int(threads))
    if st == ERANGE and check_range:
        raise OracleRangeError("8-bit sample equal to -128")
    if st not in (0, ERANGE):
        raise RuntimeError("oracle_correlate failed: %d" % st)
    return out


def decode(block, n_inputs, n_chans, n_time, bits=4, layout=L_TCI, hi_is_real=True):
    """Decoded samples as (re, im) int32 arrays [C][N][T]."""
    lib = _load()
    blk = np.ascontiguousarray(np.asarray(block, dtype=np.uint8).reshape(-1))
    re = np.zeros((n_chans, n_inputs, n_time), dtype=np.int32)
    im = np.zeros_like(re)
    st = lib.oracle_decode(_ptr(blk), layout, bits, 1 if hi_is_real else 0, n_inputs, n_chans,
                           n_time, _ptr(re), _ptr(im))
    if st not in (0, ERANGE):
        raise RuntimeError("oracle_decode failed: %d" % st)
    return re, im


def correlate_complex(x: np.ndarray) -> np.ndarray:
    """Same definition over complex128 samples x[C][N][T]: complex128 [C][B]."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.complex128)
    C, N, T = x.shape
    xv = x.view(np.float64).reshape(C, N, T, 2)
    out = np.zeros((C, n_baselines(N), 2), dtype=np.float64)
    st = lib.oracle_correlate_cd(_ptr(xv), N, C, T, _ptr(out))
    if st != 0:
        raise RuntimeError("oracle_correlate_cd failed: %d" % st)
    return out[..., 0] + 1j * out[..., 1]


def normalise(vis: np.ndarray, n_inputs: int):
    """FP64 correlation coefficients [C][B][2] and zero-denominator flags [C][B]."""
    lib = _load()
    vis = np.ascontiguousarray(vis, dtype=np.int64)
    C = vis.shape[0]
    rho = np.zeros(vis.shape, dtype=np.float64)
    flags = np.zeros(vis.shape[:2], dtype=np.uint8)
    st = lib.oracle_normalise(_ptr(vis), n_inputs, C, _ptr(rho), _ptr(flags))
    if st != 0:
        raise RuntimeError("oracle_normalise failed: %d" % st)
    return rho, flags


def projected_power(block, n_inputs, n_chans, n_time, w, bits=4, layout=L_TCI, hi_is_real=True,
                    chans=None, threads=None):
    """sum_t |sum_i conj(w_v,i) x_i(c,t)|^2 for integer complex weights w[nvec][N],
    int64 [n_chans or len(chans)][nvec]; channels spread over ``threads``
    threads (default: every core)."""
    lib = _load()
    blk = np.ascontiguousarray(np.asarray(block, dtype=np.uint8).reshape(-1))
    w = np.asarray(w)
    nvec = w.shape[0]
    wi = np.ascontiguousarray(np.stack([w.real, w.imag], axis=-1).astype(np.int32))
    ch = None
    nch = n_chans
    if chans is not None:
        ch = np.ascontiguousarray(np.asarray(chans, dtype=np.int32))
        nch = ch.size
    out = np.zeros((nch, nvec), dtype=np.int64)
    need = n_inputs * n_chans * n_time * (bits // 4)
    if blk.size != need:
        raise ValueError("block has %d bytes, expected %d" % (blk.size, need))
    if wi.shape != (nvec, n_inputs, 2):
        raise ValueError("w must be [nvec][n_inputs] complex integers")
    if threads is None:
        threads = os.cpu_count() or 1
    st = lib.oracle_projected_power(_ptr(blk), layout, bits, 1 if hi_is_real else 0, n_inputs,
                                    n_chans, n_time, _ptr(ch) if ch is not None else None, nch,
                                    _ptr(wi), nvec, _ptr(out), int(threads))
    if st not in (0, ERANGE):
        raise RuntimeError("oracle_projected_power failed: %d" % st)
    return out
