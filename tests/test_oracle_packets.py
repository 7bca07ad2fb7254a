"""Pins of the packet-ingest oracle (oracle/packets.py): the published
CRC-32 check value, hand-built headers, the paper's 8208-byte packet size,
hand-placed payload bytes, and MCNT gap counting on hand sequences."""
import zlib

import numpy as np

from oracle import packets as op
from paper_1904_07778_gb300 import synth


def _pkt(mcnt, fid, xid, payload: bytes, crc=None):
    body = mcnt.to_bytes(6, "big") + bytes([fid, xid]) + payload
    c = (zlib.crc32(body) & 0xFFFFFFFF) if crc is None else crc
    return body + b"\0\0\0\0" + c.to_bytes(4, "big")


def test_crc32_check_value():
    assert op.crc32(b"123456789") == 0xCBF43926     # the standard CRC-32 check value


def test_paper_packet_size():
    # Sec. 2.3: N_chan x N_input x 8 + header + CRC = 8208 bytes (32 x 32)
    assert op.payload_bytes(32, 32) + op.HEADER + op.TRAILER == 8208


def test_header_fields_by_hand():
    pay = bytes(range(8 * 2 * 2))
    pkt = bytes([0x01, 0x02, 0x03, 0x04, 0x05, 0x06, 3, 7]) + pay
    pkt += b"\0\0\0\0" + (zlib.crc32(pkt) & 0xFFFFFFFF).to_bytes(4, "big")
    mcnt, fid, xid, p = op.parse(pkt, 2, 2)
    assert mcnt == 0x010203040506 and fid == 3 and xid == 7
    assert p.shape == (8, 2, 2) and p[1, 0, 1] == 5 and p[7, 1, 1] == 31


def test_bad_length_and_crc_rejected():
    good = _pkt(0, 0, 0, bytes(16 * 8))
    assert op.parse(good, 4, 4) is not None
    assert op.parse(good[:-1], 4, 4) is None
    assert op.parse(_pkt(0, 0, 0, bytes(16 * 8), crc=1), 4, 4) is None
    flipped = bytearray(good)
    flipped[20] ^= 0x10
    assert op.parse(bytes(flipped), 4, 4) is None


def test_assemble_places_bytes_by_hand():
    # 2 Fids x 1 input, 2 Xids x 1 channel, T = 16 (two MCNTs per block)
    pk = []
    for mcnt in (2, 3):                      # block 1 (MCNT 2, 3 -> spectra 0..7, 8..15)
        for fid in (0, 1):
            for xid in (0, 1):
                pay = bytes([(mcnt << 5) | (fid << 4) | (xid << 3) | t for t in range(8)])
                pk.append(_pkt(mcnt, fid, xid, pay))
    blocks, rej = op.assemble(pk[::-1], 2, 1, 2, 1, 16)   # arrival order does not matter
    assert rej == [] and list(blocks) == [1]
    data, got = blocks[1]
    assert got.all()
    # spectrum t = 8 (mcnt - 2) + tt, channel = xid, input = fid
    assert data[0, 0, 0] == (2 << 5) and data[9, 1, 0] == (3 << 5) | (1 << 3) | 1
    assert data[15, 1, 1] == (3 << 5) | (1 << 4) | (1 << 3) | 7


def test_assemble_round_trips_the_generator_and_marks_losses():
    rng = np.random.default_rng(1)
    blk = rng.integers(0, 256, (32, 8, 6), dtype=np.uint8)      # T=32, C=8, N=6
    pk = synth.packets(blk, 3, 2, 2, 4, block_index=5)
    assert len(pk) == 4 * 3 * 2
    blocks, rej = op.assemble(pk, 3, 2, 2, 4, 32)
    assert rej == [] and np.array_equal(blocks[5][0], blk)
    lost = pk[:3] + pk[4:]                                       # drop MCNT 20, Fid 1, Xid 1
    data, got = op.assemble(lost + [pk[0]], 3, 2, 2, 4, 32)[0][5]  # and repeat one
    assert not got[0, 1, 1] and got.sum() == 23
    want = blk.copy()
    want[0:8, 4:8, 2:4] = 0
    assert np.array_equal(data, want)


def test_mcnt_gap_counting_by_hand():
    pk = [_pkt(m, 0, 0, bytes(8)) for m in (0, 1, 2, 5, 6, 10)]
    assert op.mcnt_gaps(pk, 1, 1) == (2, 5)        # 3, 4 and 7, 8, 9 skipped
    # streams are separate; a late packet does not count as a gap
    pk = [_pkt(0, 0, 0, bytes(8)), _pkt(0, 1, 0, bytes(8)), _pkt(2, 0, 0, bytes(8)),
          _pkt(1, 0, 0, bytes(8)), _pkt(1, 1, 0, bytes(8))]
    assert op.mcnt_gaps(pk, 1, 1) == (1, 1)


def test_packet_order_by_hand():
    # 2 Fids x 1 input, 2 Xids x 1 channel, T = 16: payload (slot, fid, xid) holds
    # spectra 8 slot .. 8 slot + 7 of channel xid, input fid
    data = np.arange(16 * 2 * 2, dtype=np.uint8).reshape(16, 2, 2)
    po = op.packet_order(data, 2, 1, 2, 1)
    assert po.shape == (2, 2, 2, 8, 1, 1)
    assert po[1, 0, 1, 3, 0, 0] == data[11, 1, 0]
    assert po[0, 1, 0, 7, 0, 0] == data[7, 0, 1]
