"""Python binding of the F-engine C ABI (include/fengine.h).

Argument marshalling only: the filter bank, FFT, separation, rounding and
equaliser all run in the CUDA kernel of ``libxengine.so`` (no CPU fallback).
"""
from __future__ import annotations

import ctypes

import numpy as np

from .xengine import (_CUDA_STREAM_LEGACY, CORR_L_CIT, CORR_L_TCI, CORR_OK, CorrError,  # noqa: F401
                      _lib, _ptr_and_size)

FE_F_LO_IS_REAL = 1
EXPORTS = ["fe_create", "fe_set_gains", "fe_channelise", "fe_gains_from_power", "fe_sync",
           "fe_destroy"]

_P, _I, _U, _LL, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_longlong, ctypes.c_double
_lib.fe_create.argtypes = [_I, _I, _I, _I, _U, _P, ctypes.POINTER(_P)]
_lib.fe_set_gains.argtypes = [_P, _P]
_lib.fe_channelise.argtypes = [_P, _P, _LL, _I, _P, _I, _LL, _P, _P, _P]
_lib.fe_gains_from_power.argtypes = [_P, _I, _I, _LL, _D, _P]
_lib.fe_sync.argtypes = [_P]
_lib.fe_destroy.argtypes = [_P]
_lib.fe_destroy.restype = None
for _f in ("fe_create", "fe_set_gains", "fe_channelise", "fe_gains_from_power", "fe_sync"):
    getattr(_lib, _f).restype = _I


def _ptr(buf):
    return None if buf is None else _P(_ptr_and_size(buf)[0])


def fe_gains_from_power(power, n_spectra: int, target_rms: float = 2.5) -> np.ndarray:
    """Eq. 3 gain rule on the host: power int64 [C][N] -> uint32 gains [C][N]."""
    p = np.ascontiguousarray(power, dtype=np.int64)
    g = np.empty(p.shape, dtype=np.uint32)
    st = _lib.fe_gains_from_power(_P(p.ctypes.data), p.shape[0], p.shape[1], n_spectra,
                                  target_rms, _P(g.ctypes.data))
    if st != CORR_OK:
        raise CorrError(st, "fe_gains_from_power")
    return g


class FEngine:
    """One channeliser: PFB + FFT + Eq. 2 + 18-bit rounding + equaliser."""

    def __init__(self, n_inputs, n_chans, taps=4, shift=0, lo_is_real=False, stream=None):
        if stream is None:  # torch's current stream (its default stream is the legacy one)
            import torch
            stream = torch.cuda.current_stream().cuda_stream or _CUDA_STREAM_LEGACY
        out = _P()
        flags = FE_F_LO_IS_REAL if lo_is_real else 0
        st = _lib.fe_create(n_inputs, n_chans, taps, shift, flags, _P(stream), ctypes.byref(out))
        if st != CORR_OK:
            raise CorrError(st, "fe_create")
        self._f = out
        self.n_inputs, self.n_chans, self.taps, self.shift = n_inputs, n_chans, taps, shift

    def set_gains(self, gain):
        if isinstance(gain, np.ndarray):
            gain = np.ascontiguousarray(gain, dtype=np.uint32)
        p, n = _ptr_and_size(gain)
        if n != self.n_chans * self.n_inputs * 4:
            raise ValueError("gain must hold n_chans * n_inputs uint32")
        st = _lib.fe_set_gains(self._f, _P(p))
        if st != CORR_OK:
            raise CorrError(st, "fe_set_gains")

    def channelise(self, adc, n_spectra, out=None, layout=CORR_L_CIT, out_stride=None,
                   v18=None, spec=None, power=None, adc_stride=None):
        """adc: device int8 [n_inputs][samples]; outputs are device tensors or None."""
        if adc_stride is None:
            adc_stride = adc.shape[-1]
        if out_stride is None:
            out_stride = n_spectra
        st = _lib.fe_channelise(self._f, _ptr(adc), adc_stride, n_spectra, _ptr(out), layout,
                                out_stride, _ptr(v18), _ptr(spec), _ptr(power))
        if st != CORR_OK:
            raise CorrError(st, "fe_channelise")

    def sync(self):
        st = _lib.fe_sync(self._f)
        if st != CORR_OK:
            raise CorrError(st, "fe_sync")

    def close(self):
        if getattr(self, "_f", None):
            _lib.fe_destroy(self._f)
            self._f = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()
