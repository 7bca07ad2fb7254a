"""Packet-ingest oracle -- TEST INFRASTRUCTURE ONLY.

A plain restatement of the F-engine -> X-engine packet stream of
arXiv:1904.07778 (Sec. 2.3, "Network and Data Packet"; Sec. 2.2 on the
Hashpipe ring buffers): every UDP payload carries an 8-byte application
header -- a 6-byte packet counter MCNT, the F-engine id Fid and the X-engine
id Xid -- then 8 stacked spectra of n_chans_pkt channels x n_inputs_pkt inputs
of 4+4-bit complex samples in [time][channel][input] order, then a CRC.  Lost
packets show as jumps in the MCNT sequence.

Readings (the paper gives the sizes, 8208 bytes = 32 x 32 x 8 + header +
CRC, but not the byte layout):
  * MCNT is big-endian (network order), Fid then Xid follow it;
  * the trailer is 8 bytes: 4 zero bytes, then the IEEE 802.3 CRC-32 of
    header and payload, big-endian (zlib.crc32 is the library step here);
  * Fid f carries inputs f n_inputs_pkt .. (f + 1) n_inputs_pkt - 1, Xid x
    carries channels x n_chans_pkt .. (x + 1) n_chans_pkt - 1, and MCNT m
    carries spectra 8 m .. 8 m + 7 (one packet per 8 spectra per stream);
  * block b of T spectra holds MCNT b T/8 .. (b + 1) T/8 - 1 (blocks are
    aligned to multiples of T/8 in MCNT); a packet that never arrived leaves
    zeros, which the correlator integrates as nothing.
Only ``tests/`` may use this module.
"""
from __future__ import annotations

import zlib

import numpy as np

HEADER, TRAILER, STACK = 8, 8, 8


def payload_bytes(n_chans_pkt: int, n_inputs_pkt: int) -> int:
    return STACK * n_chans_pkt * n_inputs_pkt


def crc32(data: bytes) -> int:
    return zlib.crc32(data) & 0xFFFFFFFF


def parse(pkt: bytes, n_chans_pkt: int, n_inputs_pkt: int):
    """(mcnt, fid, xid, payload [8][chans][inputs] uint8) or None if the
    length or the CRC is wrong."""
    P = payload_bytes(n_chans_pkt, n_inputs_pkt)
    if len(pkt) != HEADER + P + TRAILER:
        return None
    body, trailer = pkt[:HEADER + P], pkt[HEADER + P:]
    if trailer[:4] != b"\0\0\0\0" or int.from_bytes(trailer[4:], "big") != crc32(body):
        return None
    mcnt = int.from_bytes(pkt[0:6], "big")
    fid, xid = pkt[6], pkt[7]
    pay = np.frombuffer(pkt, dtype=np.uint8, count=P, offset=HEADER)
    return mcnt, fid, xid, pay.reshape(STACK, n_chans_pkt, n_inputs_pkt)


def assemble(packets, n_fids, n_inputs_pkt, n_xids, n_chans_pkt, n_time):
    """Blocks built from every valid packet, in any arrival order (the
    definition the ring implements when no packet is late).

    Returns {block: (data uint8 [T][C][N], received bool [T/8][n_fids][n_xids])}
    and the list of rejected packet indices."""
    C, N = n_xids * n_chans_pkt, n_fids * n_inputs_pkt
    per = n_time // STACK
    blocks, rejected = {}, []
    for k, pkt in enumerate(packets):
        r = parse(pkt, n_chans_pkt, n_inputs_pkt)
        if r is None or r[1] >= n_fids or r[2] >= n_xids:
            rejected.append(k)
            continue
        mcnt, fid, xid, pay = r
        b, slot = divmod(mcnt, per)
        if b not in blocks:
            blocks[b] = (np.zeros((n_time, C, N), dtype=np.uint8),
                         np.zeros((per, n_fids, n_xids), dtype=bool))
        data, got = blocks[b]
        if got[slot, fid, xid]:
            rejected.append(k)           # duplicate: the first copy stands
            continue
        got[slot, fid, xid] = True
        t0 = slot * STACK
        for tt in range(STACK):
            for cc in range(n_chans_pkt):
                c = xid * n_chans_pkt + cc
                data[t0 + tt, c, fid * n_inputs_pkt:(fid + 1) * n_inputs_pkt] = pay[tt, cc]
    return blocks, rejected


def mcnt_gaps(packets, n_chans_pkt, n_inputs_pkt, n_fids=256, n_xids=256):
    """Loss as the paper detects it: per (Fid, Xid) stream, in arrival
    order, every forward jump of MCNT by more than one counts the skipped
    packets (packets with a bad length, CRC or id are not part of any
    stream).  Returns (gap events, skipped packets)."""
    last, events, skipped = {}, 0, 0
    for pkt in packets:
        r = parse(pkt, n_chans_pkt, n_inputs_pkt)
        if r is None or r[1] >= n_fids or r[2] >= n_xids:
            continue
        mcnt, fid, xid, _ = r
        key = (fid, xid)
        if key in last and mcnt > last[key] + 1:
            events += 1
            skipped += mcnt - last[key] - 1
        if key not in last or mcnt > last[key]:
            last[key] = mcnt
    return events, skipped


def packet_order(data_tci, n_fids, n_inputs_pkt, n_xids, n_chans_pkt):
    """A [T][C][N] block rearranged as the packets carry it, slot by slot:
    [T/8][fid][xid][8][n_chans_pkt][n_inputs_pkt] -- each payload whole, the
    layout of a packet-order ring (written out packet by packet)."""
    T = data_tci.shape[0]
    out = np.zeros((T // STACK, n_fids, n_xids, STACK, n_chans_pkt, n_inputs_pkt), dtype=np.uint8)
    for slot in range(T // STACK):
        for fid in range(n_fids):
            for xid in range(n_xids):
                out[slot, fid, xid] = data_tci[STACK * slot:STACK * slot + STACK,
                                               xid * n_chans_pkt:(xid + 1) * n_chans_pkt,
                                               fid * n_inputs_pkt:(fid + 1) * n_inputs_pkt]
    return out
