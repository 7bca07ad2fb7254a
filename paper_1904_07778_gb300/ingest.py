"""Python binding of the packet assembler C ABI (include/ingest.h).

Argument marshalling only: parsing, CRC checks and block assembly run in the
native code of ``libxengine.so``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .xengine import CORR_EBUSY, CORR_OK, CORR_ETIMEDOUT, CorrError, _lib  # noqa: F401

PK_F_NO_CRC = 1
PK_F_PACKET_ORDER = 2
EXPORTS = ["pk_create", "pk_push", "pk_push_many", "pk_turn", "pk_next", "pk_release", "pk_flush", "pk_get_stats",
           "pk_crc32", "pk_destroy"]


class PkLayout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("n_fids", "n_inputs_pkt", "n_xids", "n_chans_pkt",
                                            "n_time")]


class PkBlock(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("index", ctypes.c_uint64), ("mcnt0", ctypes.c_uint64),
                ("n_packets", ctypes.c_int), ("n_missing", ctypes.c_int),
                ("received", ctypes.c_void_p)]


class PkStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "packets", "bad_length", "bad_crc", "bad_id", "late", "duplicate", "missing", "mcnt_gaps",
        "mcnt_skipped", "blocks", "blocks_with_loss", "busy")]


_P, _I, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
_lib.pk_create.argtypes = [ctypes.POINTER(PkLayout), _I, ctypes.c_uint, ctypes.POINTER(_P)]
_lib.pk_push.argtypes = [_P, ctypes.c_char_p, _SZ]
_lib.pk_next.argtypes = [_P, _I, ctypes.POINTER(PkBlock)]
_lib.pk_release.argtypes = [_P]
_lib.pk_flush.argtypes = [_P]
_lib.pk_get_stats.argtypes = [_P, ctypes.POINTER(PkStats)]
_lib.pk_crc32.argtypes = [ctypes.c_char_p, _SZ]
_lib.pk_crc32.restype = ctypes.c_uint32
_lib.pk_push_many.argtypes = [_P, _P, _SZ, _SZ, _SZ, _P]
_lib.pk_push_many.restype = _SZ
_lib.pk_turn.argtypes = [ctypes.POINTER(PkLayout), _P, _P, ctypes.c_longlong, _P]
_lib.pk_turn.restype = _I
_lib.pk_destroy.argtypes = [_P]
_lib.pk_destroy.restype = None
for _f in ("pk_create", "pk_push", "pk_next", "pk_release", "pk_flush", "pk_get_stats"):
    getattr(_lib, _f).restype = _I


def pk_crc32(data: bytes) -> int:
    return _lib.pk_crc32(data, len(data))


class PacketRing:
    """F-engine packets in, [t][c][i] blocks out (in block order)."""

    def __init__(self, n_fids, n_inputs_pkt, n_xids, n_chans_pkt, n_time, n_segments=3,
                 check_crc=True, packet_order=False):
        self.layout = PkLayout(n_fids, n_inputs_pkt, n_xids, n_chans_pkt, n_time)
        self.packet_order = packet_order
        if packet_order:
            self.shape = (n_time // 8, n_fids, n_xids, 8, n_chans_pkt, n_inputs_pkt)
        else:
            self.shape = (n_time, n_xids * n_chans_pkt, n_fids * n_inputs_pkt)
        flags = (0 if check_crc else PK_F_NO_CRC) | (PK_F_PACKET_ORDER if packet_order else 0)
        out = _P()
        st = _lib.pk_create(ctypes.byref(self.layout), n_segments, flags, ctypes.byref(out))
        if st != CORR_OK:
            raise CorrError(st, "pk_create")
        self._r = out

    def push(self, packet: bytes) -> int:
        """Status of one packet (CORR_OK, or why it was dropped / refused)."""
        return _lib.pk_push(self._r, packet, len(packet))

    def push_many(self, packets: np.ndarray, codes: np.ndarray | None = None) -> int:
        """Push the rows of a [n][len] uint8 array in order; returns how many
        were consumed (it stops at the first CORR_EBUSY)."""
        packets = np.ascontiguousarray(packets, dtype=np.uint8)
        n, ln = packets.shape
        cp = None if codes is None else _P(codes.ctypes.data)
        return _lib.pk_push_many(self._r, _P(packets.ctypes.data), n, ln, ln, cp)

    def next(self, timeout_ms=0):
        """(data view [T][C][N] uint8, info dict) of the next block, or None."""
        b = PkBlock()
        st = _lib.pk_next(self._r, timeout_ms, ctypes.byref(b))
        if st == CORR_ETIMEDOUT:
            return None
        if st != CORR_OK:
            raise CorrError(st, "pk_next")
        L = self.layout
        nbytes = L.n_time * L.n_xids * L.n_chans_pkt * L.n_fids * L.n_inputs_pkt
        buf = (ctypes.c_uint8 * nbytes).from_address(b.data)
        data = np.frombuffer(buf, dtype=np.uint8).reshape(self.shape)
        rbuf = (ctypes.c_uint8 * b.n_packets).from_address(b.received)
        received = np.frombuffer(rbuf, dtype=np.uint8).reshape(L.n_time // 8, L.n_fids, L.n_xids)
        return data, {"index": b.index, "mcnt0": b.mcnt0, "n_packets": b.n_packets,
                      "n_missing": b.n_missing, "received": received.astype(bool)}

    def turn(self, packets_dev, out_dev, out_stride=None, stream=None):
        """pk_turn: a packet-order block on the device -> [c][i][t] rows."""
        from .xengine import _ptr_and_size
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        st = _lib.pk_turn(ctypes.byref(self.layout), _P(_ptr_and_size(packets_dev)[0]),
                          _P(_ptr_and_size(out_dev)[0]),
                          out_stride if out_stride is not None else self.layout.n_time,
                          _P(stream) if stream else None)
        if st != CORR_OK:
            raise CorrError(st, "pk_turn")

    def release(self):
        st = _lib.pk_release(self._r)
        if st != CORR_OK:
            raise CorrError(st, "pk_release")

    def flush(self):
        _lib.pk_flush(self._r)

    def stats(self):
        s = PkStats()
        _lib.pk_get_stats(self._r, ctypes.byref(s))
        return {n: getattr(s, n) for n, _ in s._fields_}

    def close(self):
        if getattr(self, "_r", None):
            _lib.pk_destroy(self._r)
            self._r = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()
