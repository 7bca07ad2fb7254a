"""Python binding of the X-engine C ABI (include/xengine.h).

Argument marshalling only: every step of the data path runs in the CUDA
kernels of ``libxengine.so``.  There is no CPU fallback -- importing this
module raises if the library has not been built.

Functions carry the C names (``corr_create``, ``corr_push``, ...) and take
plain integers/pointers; ``Correlator`` wraps them for numpy arrays and torch
tensors (host or device).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxengine.so")

CORR_OK, CORR_EINVAL, CORR_ENOMEM, CORR_EBUSY = 0, -1, -2, -3
CORR_ERANGE, CORR_ESEQ, CORR_ETIMEDOUT, CORR_ECUDA, CORR_ESTATE = -4, -5, -6, -7, -8
CORR_ECORRUPT = -9
CORR_L_TCI, CORR_L_TIC, CORR_L_CIT = 0, 1, 2
CORR_F_LO_IS_REAL = 1
CORR_SEQ_ANY = (1 << 64) - 1
_CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy

EXPORTS = ["corr_create", "corr_push", "corr_dump", "corr_normalise", "corr_sync",
           "corr_destroy", "corr_strerror", "corr_n_baselines", "corr_set_timing",
           "corr_get_stats", "corr_correlate_noalloc"]

if not os.path.exists(LIB_PATH):
    raise ImportError("libxengine.so is not built (run paper_1904_07778_gb300.build.build()); "
                      "the X-engine has no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)
_P, _I, _U, _SZ, _U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_size_t, ctypes.c_uint64
_lib.corr_create.argtypes = [_I, _I, _I, _I, _I, _U, _P, ctypes.POINTER(_P)]
_lib.corr_push.argtypes = [_P, _P, _SZ, _U64]
_lib.corr_dump.argtypes = [_P, _P, _I]
_lib.corr_normalise.argtypes = [_P, _P]
_lib.corr_sync.argtypes = [_P]
_lib.corr_destroy.argtypes = [_P]
_lib.corr_strerror.argtypes = [_I]
_lib.corr_strerror.restype = ctypes.c_char_p
_lib.corr_n_baselines.argtypes = [_I]
_lib.corr_n_baselines.restype = ctypes.c_int64


class CorrStats(ctypes.Structure):
    """Mirror of struct corr_stats."""
    _fields_ = [(n, ctypes.c_uint64) for n in ("blocks", "seq_rejects", "dumps", "turn_launches",
                                                "herk_launches", "norm_launches")] + \
               [(n, ctypes.c_double) for n in ("turn_ms", "herk_ms", "copy_in_ms", "dump_ms",
                                                "norm_ms")] + \
               [(n, ctypes.c_uint64) for n in ("timed_turn", "timed_herk")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib.corr_set_timing.argtypes = [_P, _I]
_lib.corr_set_fault_injection.argtypes = [_P, _I, _I]
_lib.corr_set_fault_injection.restype = _I
EXPORTS.append("corr_set_fault_injection")
_lib.corr_normalise_flags.argtypes = [_P, _P, _P]
_lib.corr_normalise_flags.restype = _I
EXPORTS.append("corr_normalise_flags")
_lib.corr_restore.argtypes = [_P, _P]
_lib.corr_restore.restype = _I
EXPORTS.append("corr_restore")
_lib.corr_set_pipeline.argtypes = [_P, _I]
_lib.corr_set_pipeline.restype = _I
EXPORTS.append("corr_set_pipeline")
_lib.corr_dump_async.argtypes = [_P, _P, _I]
_lib.corr_dump_async.restype = _I
_lib.corr_dump_wait.argtypes = [_P]
_lib.corr_dump_wait.restype = _I
_lib.corr_bind.argtypes = [_P, _P]
_lib.corr_bind.restype = _I
EXPORTS += ["corr_dump_async", "corr_dump_wait", "corr_bind"]
CORR_MAX_ASYNC_DUMPS = 4
_lib.corr_correlate_noalloc.argtypes = [_P, _I, _I, _I, _I, _U, _P, _P, _P]
_lib.corr_correlate_noalloc.restype = _I
_lib.corr_correlate_noalloc_bits.argtypes = [_P, _I, _I, _I, _I, _I, _U, _P, _P, _P]
_lib.corr_correlate_noalloc_bits.restype = _I
EXPORTS.append("corr_correlate_noalloc_bits")
CORR_NOALLOC_SCRATCH_BYTES = 16 << 20
_lib.corr_get_stats.argtypes = [_P, ctypes.POINTER(CorrStats)]
_lib.corr_push_many.argtypes = [_P, ctypes.POINTER(_P), _I, _SZ, _U64]
_lib.corr_push_many.restype = _I
EXPORTS.append("corr_push_many")
CORR_MAX_PUSH_MANY = 4096
for _f in ("corr_create", "corr_push", "corr_dump", "corr_normalise", "corr_sync", "corr_destroy",
           "corr_set_timing", "corr_get_stats"):
    getattr(_lib, _f).restype = _I


class CorrError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__("%s: %s (%d)" % (where, corr_strerror(status), status))
        self.status = status


def corr_strerror(status: int) -> str:
    return _lib.corr_strerror(status).decode()


def corr_n_baselines(n_inputs: int) -> int:
    return int(_lib.corr_n_baselines(n_inputs))


def corr_create(n_inputs, n_chans, n_time, bits=4, layout=CORR_L_TCI, flags=0, stream=0):
    ctx = _P()
    st = _lib.corr_create(n_inputs, n_chans, n_time, bits, layout, flags,
                          _P(stream) if stream else None, ctypes.byref(ctx))
    if st != CORR_OK:
        raise CorrError(st, "corr_create")
    return ctx


def corr_push(ctx, block_ptr: int, nbytes: int, seq: int = CORR_SEQ_ANY) -> int:
    return _lib.corr_push(ctx, _P(block_ptr), nbytes, seq)


def corr_dump(ctx, vis_ptr: int, reset: int = 1) -> int:
    return _lib.corr_dump(ctx, _P(vis_ptr) if vis_ptr else None, reset)


def corr_normalise(ctx, rho_ptr: int) -> int:
    return _lib.corr_normalise(ctx, _P(rho_ptr))


def corr_normalise_flags(ctx, rho_ptr: int, flag_ptr: int) -> int:
    return _lib.corr_normalise_flags(ctx, _P(rho_ptr), _P(flag_ptr) if flag_ptr else None)


def corr_sync(ctx) -> int:
    return _lib.corr_sync(ctx)


def corr_destroy(ctx) -> int:
    return _lib.corr_destroy(ctx)


def corr_correlate_noalloc(block_ptr: int, n_inputs: int, n_chans: int, n_time: int, layout: int,
                           flags: int, vis_ptr: int, status_ptr: int = 0, stream: int = 0) -> int:
    """One block's visibilities into device memory; the library allocates nothing."""
    return _lib.corr_correlate_noalloc(_P(block_ptr), n_inputs, n_chans, n_time, layout, flags,
                                       _P(vis_ptr), _P(status_ptr) if status_ptr else None,
                                       _P(stream) if stream else None)


def corr_correlate_noalloc_bits(block_ptr: int, n_inputs: int, n_chans: int, n_time: int, bits: int,
                                layout: int, flags: int, vis_ptr: int, status_ptr: int = 0,
                                stream: int = 0) -> int:
    """corr_correlate_noalloc for 4- or 8-bit samples."""
    return _lib.corr_correlate_noalloc_bits(_P(block_ptr), n_inputs, n_chans, n_time, bits, layout,
                                            flags, _P(vis_ptr), _P(status_ptr) if status_ptr else None,
                                            _P(stream) if stream else None)


def corr_set_timing(ctx, on: int) -> int:
    return _lib.corr_set_timing(ctx, on)


def corr_get_stats(ctx, out: CorrStats) -> int:
    return _lib.corr_get_stats(ctx, ctypes.byref(out))


def _ptr_and_size(buf):
    """(address, nbytes) of a numpy array or torch tensor (host or device)."""
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("buffer must be contiguous")
        return buf.ctypes.data, buf.nbytes
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr(), buf.numel() * buf.element_size()
    raise TypeError("expected a numpy array or a torch tensor")


class Correlator:
    """One X-engine context: push blocks, dump integrated visibilities."""

    def __init__(self, n_inputs, n_chans, n_time, bits=4, layout=CORR_L_TCI, lo_is_real=False,
                 stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
            if stream == 0:
                stream = _CUDA_STREAM_LEGACY  # torch's default stream is the legacy stream
        self.n_inputs, self.n_chans, self.n_time, self.bits = n_inputs, n_chans, n_time, bits
        self.layout = layout
        self.n_baselines = corr_n_baselines(n_inputs)
        self.block_bytes = n_inputs * n_chans * n_time * bits // 4
        self._ctx = corr_create(n_inputs, n_chans, n_time, bits, layout,
                                CORR_F_LO_IS_REAL if lo_is_real else 0, stream)

    def push(self, block, seq=CORR_SEQ_ANY, check=True):
        p, n = _ptr_and_size(block)
        st = corr_push(self._ctx, p, n, seq)
        if check and st != CORR_OK:
            raise CorrError(st, "corr_push")
        return st

    def push_many(self, blocks, seq=CORR_SEQ_ANY, check=True):
        """Integrate several blocks of one shape (corr_push_many): one
        cross-multiply launch over all of them where they are device blocks
        read in place."""
        ptrs, size = [], None
        for blk in blocks:
            p, n = _ptr_and_size(blk)
            if size is not None and n != size:
                raise ValueError("every block must have the same size")
            ptrs.append(p)
            size = n
        if not ptrs:
            raise ValueError("no blocks")
        arr = (_P * len(ptrs))(*ptrs)
        st = _lib.corr_push_many(self._ctx, arr, len(ptrs), size, seq)
        if check and st != CORR_OK:
            raise CorrError(st, "corr_push_many")
        return st

    def dump_into(self, vis, reset=True, check=True):
        """Copy the integration into ``vis``.  With check=False a non-OK
        status (CORR_ERANGE after an 8-bit -128, for instance) does not
        raise; it is left in ``last_status`` and ``vis`` still holds the sums."""
        p, n = _ptr_and_size(vis)
        if n != self.n_chans * self.n_baselines * 16:
            raise ValueError("vis must hold n_chans * n_baselines * 2 int64")
        st = corr_dump(self._ctx, p, 1 if reset else 0)
        self.last_status = st
        if check and st != CORR_OK:
            raise CorrError(st, "corr_dump")
        return vis

    def set_pipeline(self, turn_sms: int):
        """Overlap each block's corner turn (on turn_sms SMs) with the previous
        block's cross-multiply (corr_set_pipeline); 0 turns it off."""
        st = _lib.corr_set_pipeline(self._ctx, turn_sms)
        if st != CORR_OK:
            raise CorrError(st, "corr_set_pipeline")

    def dump_async(self, vis, reset=True):
        """Queue the copy of the integration into ``vis`` (corr_dump_async);
        ``vis`` holds it once the matching :meth:`dump_wait` returns."""
        p, n = _ptr_and_size(vis)
        if n != self.n_chans * self.n_baselines * 16:
            raise ValueError("vis must hold n_chans * n_baselines * 2 int64")
        st = _lib.corr_dump_async(self._ctx, _P(p), 1 if reset else 0)
        if st != CORR_OK:
            raise CorrError(st, "corr_dump_async")
        return vis

    def bind(self, vis):
        """Accumulate the next integration in place in the device tensor
        ``vis`` (corr_bind); a dump into ``vis`` then copies nothing.  The
        binding ends with the next dump with reset."""
        p, n = _ptr_and_size(vis)
        if n != self.n_chans * self.n_baselines * 16:
            raise ValueError("vis must hold n_chans * n_baselines * 2 int64")
        st = _lib.corr_bind(self._ctx, _P(p))
        if st != CORR_OK:
            raise CorrError(st, "corr_bind")
        self._bound = vis   # kept alive while the library may still write it
        return vis

    def dump_wait(self, check=True):
        """Wait for the oldest queued dump; returns (and with check, raises
        on) its deferred device status."""
        st = _lib.corr_dump_wait(self._ctx)
        self.last_status = st
        if check and st != CORR_OK:
            raise CorrError(st, "corr_dump_wait")
        return st

    def dump(self, reset=True, check=True):
        vis = np.empty((self.n_chans, self.n_baselines, 2), dtype=np.int64)
        return self.dump_into(vis, reset, check)

    def restore(self, vis):
        """Resume from a saved integration (a dump taken with reset=False)."""
        p, n = _ptr_and_size(vis)
        if n != self.n_chans * self.n_baselines * 16:
            raise ValueError("vis must hold n_chans * n_baselines * 2 int64")
        st = _lib.corr_restore(self._ctx, _P(p))
        if st != CORR_OK:
            raise CorrError(st, "corr_restore")

    def normalise_into(self, rho):
        p, n = _ptr_and_size(rho)
        if n != self.n_chans * self.n_baselines * 16:
            raise ValueError("rho must hold n_chans * n_baselines * 2 float64")
        st = corr_normalise(self._ctx, p)
        if st != CORR_OK:
            raise CorrError(st, "corr_normalise")
        return rho

    def normalise(self, flags=False):
        """FP64 correlation coefficients [C][B][2]; with flags=True also the
        zero-denominator flags [C][B] (1 where V_ii V_jj = 0)."""
        rho = np.empty((self.n_chans, self.n_baselines, 2), dtype=np.float64)
        if not flags:
            return self.normalise_into(rho)
        zf = np.empty((self.n_chans, self.n_baselines), dtype=np.uint8)
        st = corr_normalise_flags(self._ctx, rho.ctypes.data, zf.ctypes.data)
        if st != CORR_OK:
            raise CorrError(st, "corr_normalise_flags")
        return rho, zf

    def set_fault_injection(self, stage, wait_log2=0):
        """Test hook (corr_set_fault_injection): the first CTA of later
        cross-multiplies never loads its stage ``stage`` (-1: off), and every
        device wait gives up after 2^wait_log2 cycles (0: default budget)."""
        st = _lib.corr_set_fault_injection(self._ctx, stage, wait_log2)
        if st != CORR_OK:
            raise CorrError(st, "corr_set_fault_injection")

    def set_timing(self, on=True):
        corr_set_timing(self._ctx, 1 if on else 0)

    def stats(self):
        out = CorrStats()
        st = corr_get_stats(self._ctx, out)
        if st != CORR_OK:
            raise CorrError(st, "corr_get_stats")
        return out.as_dict()

    def sync(self):
        st = corr_sync(self._ctx)
        if st != CORR_OK:
            raise CorrError(st, "corr_sync")

    def close(self):
        if self._ctx:
            corr_destroy(self._ctx)   # waits for the context's work
            self._ctx = None
        self._bound = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------- batches
EXPORTS += ["corr_batch_create", "corr_batch_input", "corr_batch_output", "corr_batch_set_input",
            "corr_batch_get_output", "corr_batch_run", "corr_batch_run_plain", "corr_batch_sync",
            "corr_batch_info_get", "corr_batch_destroy", "corr_plan_schedule", "corr_batch_set_pipeline"]
CORR_SCHED_PAIRS_LPT, CORR_SCHED_SINGLES_LPT, CORR_SCHED_PAIRS_RR = 0, 1, 2


class CorrShape(ctypes.Structure):
    """Mirror of struct corr_shape."""
    _fields_ = [("n_inputs", _I), ("n_chans", _I), ("n_time", _I), ("bits", _I), ("layout", _I),
                ("flags", _U)]


class CorrBatchInfo(ctypes.Structure):
    """Mirror of struct corr_batch_info."""
    _fields_ = [("schedule", _I), ("n_tasks", _I), ("n_ctas", _I), ("launches_per_run", _I),
                ("tuned_ms", ctypes.c_double * 3), ("tune_source", _I)]


_lib.corr_batch_create.argtypes = [ctypes.POINTER(CorrShape), _I, _P, _I, ctypes.POINTER(_P)]
_lib.corr_batch_input.argtypes = [_P, _I]
_lib.corr_batch_input.restype = _P
_lib.corr_batch_output.argtypes = [_P, _I]
_lib.corr_batch_output.restype = _P
_lib.corr_batch_set_input.argtypes = [_P, _I, _P, _SZ]
_lib.corr_batch_get_output.argtypes = [_P, _I, _P]
_lib.corr_batch_run.argtypes = [_P]
_lib.corr_batch_run_plain.argtypes = [_P]
_lib.corr_batch_set_pipeline.argtypes = [_P, _I, _I]
_lib.corr_batch_sync.argtypes = [_P]
_lib.corr_batch_info_get.argtypes = [_P, ctypes.POINTER(CorrBatchInfo)]
_lib.corr_batch_destroy.argtypes = [_P]
_lib.corr_batch_destroy.restype = None
_lib.corr_plan_schedule.argtypes = [_P, _I, _I, _P, _P]
for _f in ("corr_batch_create", "corr_batch_set_input", "corr_batch_get_output", "corr_batch_run",
           "corr_batch_run_plain", "corr_batch_sync", "corr_batch_info_get", "corr_plan_schedule"):
    getattr(_lib, _f).restype = _I


def corr_plan_schedule(cost, n_ctas):
    """Longest-first assignment of tasks to CTAs (host only): (order, cta_first)."""
    c = np.ascontiguousarray(np.asarray(cost, dtype=np.float64))
    order = np.empty(c.size, dtype=np.int32)
    first = np.empty(n_ctas + 1, dtype=np.int32)
    st = _lib.corr_plan_schedule(c.ctypes.data, c.size, n_ctas, order.ctypes.data,
                                 first.ctypes.data)
    if st != CORR_OK:
        raise CorrError(st, "corr_plan_schedule")
    return order, first


class Batch:
    """Several arrays correlated by one persistent launch per run (corr_batch_*).

    ``shapes`` is a list of (n_inputs, n_chans, n_time, bits, layout[, flags])."""

    def __init__(self, shapes, tune=False, stream=None):
        arr = (CorrShape * len(shapes))()
        for k, sh in enumerate(shapes):
            n, c, t, bits, layout = sh[:5]
            flags = sh[5] if len(sh) > 5 else 0
            arr[k] = CorrShape(n, c, t, bits, layout, flags)
        self.shapes = [tuple(s[:5]) for s in shapes]
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream or _CUDA_STREAM_LEGACY
        out = _P()
        st = _lib.corr_batch_create(arr, len(shapes), _P(stream), 1 if tune else 0,
                                    ctypes.byref(out))
        if st != CORR_OK:
            raise CorrError(st, "corr_batch_create")
        self._b = out

    def set_input(self, k, block):
        p, n = _ptr_and_size(block)
        st = _lib.corr_batch_set_input(self._b, k, _P(p), n)
        if st != CORR_OK:
            raise CorrError(st, "corr_batch_set_input")

    def output(self, k):
        n, c = self.shapes[k][0], self.shapes[k][1]
        vis = np.empty((c, n * (n + 1) // 2, 2), dtype=np.int64)
        st = _lib.corr_batch_get_output(self._b, k, _P(vis.ctypes.data))
        if st != CORR_OK:
            raise CorrError(st, "corr_batch_get_output")
        return vis

    def run(self):
        st = _lib.corr_batch_run(self._b)
        if st != CORR_OK:
            raise CorrError(st, "corr_batch_run")

    def run_plain(self):
        st = _lib.corr_batch_run_plain(self._b)
        if st != CORR_OK:
            raise CorrError(st, "corr_batch_run_plain")

    def set_pipeline(self, turn_sms, n_chunks=8):
        """Turn the largest array in channel ranges on turn_sms SMs beside the
        cross-multiply of the ranges already turned (corr_batch_set_pipeline);
        0 restores the single-launch graph."""
        st = _lib.corr_batch_set_pipeline(self._b, turn_sms, n_chunks)
        if st != CORR_OK:
            raise CorrError(st, "corr_batch_set_pipeline")

    def sync(self):
        return _lib.corr_batch_sync(self._b)

    def info(self):
        out = CorrBatchInfo()
        st = _lib.corr_batch_info_get(self._b, ctypes.byref(out))
        if st != CORR_OK:
            raise CorrError(st, "corr_batch_info_get")
        return {"schedule": out.schedule, "n_tasks": out.n_tasks, "n_ctas": out.n_ctas,
                "launches_per_run": out.launches_per_run, "tuned_ms": list(out.tuned_ms),
                "tune_source": out.tune_source}

    def close(self):
        if getattr(self, "_b", None):
            _lib.corr_batch_destroy(self._b)
            self._b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()


# ------------------------------------------------------------------- service
EXPORTS += ["corr_svc_create", "corr_svc_submit", "corr_svc_state", "corr_svc_push", "corr_svc_tick",
            "corr_svc_fetch", "corr_svc_wait", "corr_svc_stats_get", "corr_svc_destroy"]
CORR_SVC_DRY_RUN = 1
CORR_REQ_QUEUED, CORR_REQ_ACTIVE, CORR_REQ_DONE, CORR_REQ_FETCHED = 0, 1, 2, 3


class CorrReq(ctypes.Structure):
    """Mirror of struct corr_req."""
    _fields_ = [("n_inputs", _I), ("n_chans", _I), ("bits", _I), ("layout", _I), ("flags", _U),
                ("block_spectra", _I), ("n_blocks", ctypes.c_int64)]


class CorrSvcStats(ctypes.Structure):
    """Mirror of struct corr_svc_stats."""
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "completed", "fetched",
                                                "ticks", "launches", "blocks")] + \
               [(n, ctypes.c_double) for n in ("chan_spectra", "ops", "p50_ms", "p99_ms", "max_ms")] + \
               [(n, ctypes.c_uint64) for n in ("budget", "in_use", "peak_in_use")] + \
               [("active", _I), ("queued", _I)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib.corr_svc_create.argtypes = [_SZ, _U, _P, ctypes.POINTER(_P)]
_lib.corr_svc_submit.argtypes = [_P, ctypes.POINTER(CorrReq), ctypes.POINTER(ctypes.c_int64)]
_lib.corr_svc_state.argtypes = [_P, ctypes.c_int64, ctypes.POINTER(_I)]
_lib.corr_svc_push.argtypes = [_P, ctypes.c_int64, _P, _SZ]
_lib.corr_svc_tick.argtypes = [_P, ctypes.POINTER(_I)]
_lib.corr_svc_fetch.argtypes = [_P, ctypes.c_int64, _P]
_lib.corr_svc_wait.argtypes = [_P]
_lib.corr_svc_stats_get.argtypes = [_P, ctypes.POINTER(CorrSvcStats)]
_lib.corr_svc_destroy.argtypes = [_P]
_lib.corr_svc_destroy.restype = None
for _f in ("corr_svc_create", "corr_svc_submit", "corr_svc_state", "corr_svc_push", "corr_svc_tick",
           "corr_svc_fetch", "corr_svc_wait", "corr_svc_stats_get"):
    getattr(_lib, _f).restype = _I


class Service:
    """Continuous batching of integration requests (corr_svc_*)."""

    def __init__(self, hbm_budget, dry_run=False, stream=None):
        if stream is None and not dry_run:
            import torch
            stream = torch.cuda.current_stream().cuda_stream or _CUDA_STREAM_LEGACY
        out = _P()
        st = _lib.corr_svc_create(int(hbm_budget), CORR_SVC_DRY_RUN if dry_run else 0,
                                  _P(stream or 0), ctypes.byref(out))
        if st != CORR_OK:
            raise CorrError(st, "corr_svc_create")
        self._s = out
        self._shape = {}

    def submit(self, n_inputs, n_chans, bits, layout, block_spectra, n_blocks, flags=0, check=True):
        rid = ctypes.c_int64()
        r = CorrReq(n_inputs, n_chans, bits, layout, flags, block_spectra, n_blocks)
        st = _lib.corr_svc_submit(self._s, ctypes.byref(r), ctypes.byref(rid))
        if st != CORR_OK:
            if check:
                raise CorrError(st, "corr_svc_submit")
            return st
        self._shape[rid.value] = (n_inputs, n_chans)
        return rid.value

    def state(self, rid):
        out = _I()
        st = _lib.corr_svc_state(self._s, rid, ctypes.byref(out))
        if st != CORR_OK:
            raise CorrError(st, "corr_svc_state")
        return out.value

    def push(self, rid, block, check=True):
        p, n = _ptr_and_size(block)
        st = _lib.corr_svc_push(self._s, rid, _P(p), n)
        if check and st != CORR_OK:
            raise CorrError(st, "corr_svc_push")
        return st

    def tick(self):
        n = _I()
        st = _lib.corr_svc_tick(self._s, ctypes.byref(n))
        if st != CORR_OK:
            raise CorrError(st, "corr_svc_tick")
        return n.value

    def fetch(self, rid, vis=None, check=True):
        """Copy a done request's visibilities into ``vis`` (or a new array)."""
        if vis is None and rid in self._shape:
            n, c = self._shape[rid]
            vis = np.empty((c, n * (n + 1) // 2, 2), dtype=np.int64)
        p = _ptr_and_size(vis)[0] if vis is not None else 0
        st = _lib.corr_svc_fetch(self._s, rid, _P(p))
        if st != CORR_OK:
            if check:
                raise CorrError(st, "corr_svc_fetch")
            return st
        return vis

    def wait(self):
        return _lib.corr_svc_wait(self._s)

    def stats(self):
        out = CorrSvcStats()
        st = _lib.corr_svc_stats_get(self._s, ctypes.byref(out))
        if st != CORR_OK:
            raise CorrError(st, "corr_svc_stats_get")
        return out.as_dict()

    def close(self):
        if getattr(self, "_s", None):
            _lib.corr_svc_destroy(self._s)
            self._s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()
