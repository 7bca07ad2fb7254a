"""The packet assembler (include/ingest.h) against the packet oracle: block
bytes and loss marks bit-exact, drop reasons counted, MCNT gaps as the oracle
counts them, the ring's closing and hand-out order, and a producer thread
feeding a consumer thread.  Fault injection happens on the host: packets are
dropped, duplicated, reordered, truncated, corrupted or given bad ids before
they reach pk_push.  The last test correlates assembled blocks on the GPU."""
import threading

import numpy as np
import pytest

from oracle import packets as op
from paper_1904_07778_gb300 import synth
from paper_1904_07778_gb300.ingest import PacketRing, pk_crc32
from paper_1904_07778_gb300.xengine import CORR_EBUSY, CORR_ECORRUPT, CORR_EINVAL, CORR_OK, CORR_ESEQ

# 3 F-engines x 4 inputs, 2 bands x 8 channels, 32 spectra per block
LAY = dict(n_fids=3, n_inputs_pkt=4, n_xids=2, n_chans_pkt=8, n_time=32)
N, C, T = 12, 16, 32


def _blocks(n, seed=0):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 256, (T, C, N), dtype=np.uint8) for _ in range(n)]


def _stream(blocks, first=0):
    out = []
    for k, b in enumerate(blocks):
        out += synth.packets(b, 3, 4, 2, 8, block_index=first + k)
    return out


def _ring(**kw):
    return PacketRing(LAY["n_fids"], LAY["n_inputs_pkt"], LAY["n_xids"], LAY["n_chans_pkt"],
                      LAY["n_time"], **kw)


def _drain(ring):
    got = []
    while True:
        r = ring.next(0)
        if r is None:
            return got
        data, info = r
        got.append((info["index"], data.copy(), info))
        ring.release()


def _feed(ring, packets):
    """Push every packet; when the ring is full, take the next block out
    first (what a consumer thread would do).  Returns (push codes, taken)."""
    codes, taken = [], []
    for p in packets:
        st = ring.push(p)
        while st == CORR_EBUSY:
            taken += _drain(ring)
            st = ring.push(p)
        codes.append(st)
    return codes, taken


def test_crc_is_the_ieee_crc32():
    """Short messages take one table chain, from 256 bytes four segments
    joined by the GF(2) shift: lengths around the switch and every
    remainder of the segment split."""
    import zlib
    rng = np.random.default_rng(1)
    for n in (0, 1, 7, 8, 9, 63, 255, 256, 257, 263, 264, 287, 288, 289, 1000, 4101, 8191,
              8200, 8208, 65536 + 37, (1 << 20) + 3):
        d = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert pk_crc32(d) == zlib.crc32(d) & 0xFFFFFFFF


def test_crc_random_lengths_and_offsets():
    """Any length and any start address (the four segments and the tail
    step through unaligned bytes)."""
    import zlib
    rng = np.random.default_rng(2)
    buf = rng.integers(0, 256, 40000, dtype=np.uint8).tobytes()
    for _ in range(60):
        off = int(rng.integers(0, 16))
        n = int(rng.integers(0, 30000))
        d = buf[off:off + n]
        assert pk_crc32(d) == zlib.crc32(d) & 0xFFFFFFFF, (off, n)


@pytest.mark.gpu
def test_crc_on_the_gpu_hosts_cpu():
    """The CRC-32 on the host of a GPU machine, where the ARMv8 CRC
    instructions replace the tables when the CPU has them: the lengths of
    the two tests above, and every start address of a packet-sized message."""
    import zlib
    rng = np.random.default_rng(3)
    for n in (0, 1, 7, 8, 9, 63, 255, 256, 257, 263, 264, 287, 288, 289, 1000, 4101, 8191,
              8200, 8208, 65536 + 37, (1 << 20) + 3):
        d = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert pk_crc32(d) == zlib.crc32(d) & 0xFFFFFFFF, n
    buf = rng.integers(0, 256, 40000, dtype=np.uint8).tobytes()
    for off in range(16):
        for n in (8204, 8208, 30000):
            d = buf[off:off + n]
            assert pk_crc32(d) == zlib.crc32(d) & 0xFFFFFFFF, (off, n)


def test_clean_stream_round_trips():
    blocks = _blocks(4)
    with _ring() as ring:
        codes, got = _feed(ring, _stream(blocks, first=7))
        assert set(codes) == {CORR_OK}
        got += _drain(ring)
        st = ring.stats()
    assert [g[0] for g in got] == [7, 8, 9, 10]
    for (idx, data, info), b in zip(got, blocks):
        assert np.array_equal(data, b) and info["n_missing"] == 0 and info["received"].all()
        assert info["mcnt0"] == idx * (T // 8)
    assert st["packets"] == 4 * 4 * 6 and st["blocks"] == 4 and st["missing"] == 0
    assert st["mcnt_gaps"] == 0


def test_faults_match_the_oracle():
    """Drops, duplicates, in-block reordering, bad CRCs, truncation and bad
    ids: every delivered block equals the oracle's assembly of the packets
    that survive, with the same loss marks; counters match the injections."""
    rng = np.random.default_rng(2)
    blocks = _blocks(3, seed=3)
    clean = _stream(blocks)
    per = len(clean) // 3
    stream, n_dup, n_crc, n_len, n_id = [], 0, 0, 0, 0
    for b in range(3):
        chunk = clean[b * per:(b + 1) * per]
        order = rng.permutation(per)                         # reorder inside the block
        for k in order:
            p = chunk[k]
            u = rng.random()
            if u < 0.08:
                continue                                     # lost
            if u < 0.12:
                bad = bytearray(p)
                bad[40] ^= 0x01
                stream.append(bytes(bad))
                n_crc += 1
                continue
            stream.append(p)
            if u > 0.95:
                stream.append(p)                             # duplicate
                n_dup += 1
    stream.insert(5, stream[3][:-3])                          # truncated
    n_len += 1
    bad_id = bytearray(clean[0][:8]) + clean[0][8:-8]
    bad_id[6] = 9                                             # Fid 9 of 3
    import zlib
    body = bytes(bad_id)
    stream.insert(9, body + b"\0\0\0\0" + (zlib.crc32(body) & 0xFFFFFFFF).to_bytes(4, "big"))
    n_id += 1
    with _ring() as ring:
        codes = [ring.push(p) for p in stream]
        ring.flush()
        got = _drain(ring)
        st = ring.stats()
    want, _ = op.assemble(stream, 3, 4, 2, 8, T)
    assert [g[0] for g in got] == sorted(want)
    for idx, data, info in got:
        wd, wr = want[idx]
        assert np.array_equal(data, wd)
        assert np.array_equal(info["received"], wr)
        assert info["n_missing"] == wr.size - wr.sum()
    assert codes.count(CORR_ECORRUPT) == n_crc == st["bad_crc"]
    assert st["duplicate"] == n_dup and st["bad_length"] == n_len and st["bad_id"] == n_id
    assert codes.count(CORR_EINVAL) == n_len + n_id and codes.count(CORR_ESEQ) == n_dup
    assert st["missing"] == sum(w[1].size - w[1].sum() for w in want.values())
    assert (st["mcnt_gaps"], st["mcnt_skipped"]) == op.mcnt_gaps(stream, 8, 4, 3, 2)


def test_late_packets_after_hand_out_are_dropped():
    blocks = _blocks(2, seed=4)
    pk = _stream(blocks)
    per = len(pk) // 2
    with _ring() as ring:
        for p in pk[:per - 1]:
            ring.push(p)
        for p in pk[per:]:
            ring.push(p)                 # block 1 completes while block 0 misses one
        assert ring.next(0) is None      # block 0 is still open: nothing is handed out
        ring.flush()
        got = _drain(ring)
        assert [g[0] for g in got] == [0, 1] and got[0][2]["n_missing"] == 1
        assert ring.push(pk[per - 1]) == CORR_ESEQ       # block 0 is gone: late
        assert ring.stats()["late"] == 1


def test_window_closes_old_blocks_and_busy_forces_progress():
    blocks = _blocks(6, seed=5)
    pk = _stream(blocks)
    per = len(pk) // 6
    with _ring(n_segments=3) as ring:
        ring.push(pk[0])                             # block 0 open with one packet
        ring.push(pk[3 * per])                       # block 3 >= 0 + 3: block 0 closes
        data, info = ring.next(0)
        assert info["index"] == 0 and info["n_missing"] == per - 1
        # hold block 0; open blocks 3, 4: the third segment is block 0's
        assert ring.push(pk[4 * per]) == CORR_OK
        assert ring.push(pk[5 * per]) == CORR_EBUSY  # no free segment: block 3 is closed
        assert ring.stats()["busy"] == 1
        ring.release()
        assert ring.push(pk[5 * per]) == CORR_OK
        nxt = ring.next(0)
        assert nxt is not None and nxt[1]["index"] == 3 and nxt[1]["n_missing"] == per - 1
        ring.release()


def test_push_many_equals_single_pushes():
    blocks = _blocks(5, seed=10)
    pk = _stream(blocks)
    arr = np.frombuffer(b"".join(pk), dtype=np.uint8).reshape(len(pk), -1).copy()
    arr[7, 30] ^= 1                                   # one bad CRC
    codes = np.full(len(pk), 99, dtype=np.int32)
    got = []
    with _ring() as ring:
        k = 0
        while k < len(pk):
            k += ring.push_many(arr[k:], codes[k:])
            got += _drain(ring)
        ring.flush()
        got += _drain(ring)
    assert codes[7] == CORR_ECORRUPT and np.all(np.delete(codes, 7) == CORR_OK)
    assert [g[0] for g in got] == list(range(5))
    slot, rest = divmod(7, 6)
    fid, xid = divmod(rest, 2)
    want = blocks[0].copy()
    want[8 * slot:8 * slot + 8, xid * 8:xid * 8 + 8, fid * 4:fid * 4 + 4] = 0
    assert np.array_equal(got[0][1], want)
    assert all(np.array_equal(g[1], b) for g, b in zip(got[1:], blocks[1:]))


def test_packet_order_ring_matches_the_oracle():
    """The same faulty stream into a packet-order ring: every block equals the
    oracle's assembly rearranged into packet order, losses zero."""
    rng = np.random.default_rng(21)
    blocks = _blocks(3, seed=22)
    clean = _stream(blocks)
    stream = [p for p in clean if rng.random() > 0.1]
    stream += stream[:5]                                   # duplicates
    with _ring(packet_order=True) as ring:
        _feed(ring, stream)
        ring.flush()
        got = _drain(ring)
    want, _ = op.assemble(stream, 3, 4, 2, 8, T)
    assert [g[0] for g in got] == sorted(want)
    for idx, data, info in got:
        assert np.array_equal(data, op.packet_order(want[idx][0], 3, 4, 2, 8))
        assert np.array_equal(info["received"], want[idx][1])


def test_no_crc_mode_accepts_corrupt_packets():
    pk = _stream(_blocks(1, seed=6))
    bad = bytearray(pk[0])
    bad[-1] ^= 0xFF
    with _ring(check_crc=False) as ring:
        assert ring.push(bytes(bad)) == CORR_OK


def test_producer_and_consumer_threads():
    blocks = _blocks(12, seed=7)
    pk = _stream(blocks)
    out, err = [], []
    with _ring(n_segments=3) as ring:
        def produce():
            for p in pk:
                while True:
                    st = ring.push(p)
                    if st != CORR_EBUSY:
                        break
                    threading.Event().wait(0.0005)
                if st != CORR_OK:
                    err.append(st)
            ring.flush()

        def consume():
            while len(out) < len(blocks):
                r = ring.next(2000)
                if r is None:
                    err.append("timeout")
                    return
                out.append((r[1]["index"], r[0].copy()))
                ring.release()

        th = [threading.Thread(target=produce), threading.Thread(target=consume)]
        for t in th:
            t.start()
        for t in th:
            t.join(30)
    assert not err
    assert [o[0] for o in out] == list(range(12))
    assert all(np.array_equal(d, b) for (_, d), b in zip(out, blocks))


def test_bad_layouts_rejected():
    from paper_1904_07778_gb300.xengine import CorrError
    for kw in (dict(n_time=12), dict(n_fids=0), dict(n_xids=300)):
        lay = dict(LAY, **kw)
        with pytest.raises(CorrError):
            PacketRing(lay["n_fids"], lay["n_inputs_pkt"], lay["n_xids"], lay["n_chans_pkt"],
                       lay["n_time"])
    with pytest.raises(CorrError):
        _ring(n_segments=1)


@pytest.mark.gpu
@pytest.mark.parametrize("geom,T,pad", [
    ((6, 32, 32, 32), 1024, 0),      # the cylinder's packets
    ((6, 32, 32, 32), 264, 0),       # a ragged last tile of spectra
    ((3, 12, 5, 10), 72, 8),         # rows of 120 bytes: the byte path; padded output rows
    ((1, 16, 3, 8), 512, 32)])
def test_pk_turn_reorders_exactly(geom, T, pad):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F, I, X, K = geom
    N, C = F * I, X * K
    rng = np.random.default_rng(T + F)
    data = rng.integers(0, 256, (T, C, N), dtype=np.uint8)           # [t][c][i]
    po = op.packet_order(data, F, I, X, K)
    ring = PacketRing(F, I, X, K, T)
    dev_in = torch.from_numpy(np.ascontiguousarray(po).reshape(-1)).cuda()
    os_ = T + pad
    out = torch.full((C * N * os_,), 0x5A, dtype=torch.uint8, device="cuda")
    ring.turn(dev_in, out, out_stride=os_)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(C, N, os_)
    assert np.array_equal(got[:, :, :T], data.transpose(1, 2, 0))
    assert np.all(got[:, :, T:] == 0x5A)
    ring.close()


@pytest.mark.gpu
def test_packet_order_to_visibilities():
    """Packets -> packet-order ring -> device -> pk_turn -> corr_push ([c][i][t])."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1904_07778_gb300.xengine import CORR_L_CIT, Correlator
    rng = np.random.default_rng(23)
    blocks = _blocks(2, seed=24)
    pk = _stream(blocks, first=3)
    keep = [p for p in pk if rng.random() > 0.1]
    assembled, _ = op.assemble(keep, 3, 4, 2, 8, T)
    with _ring(packet_order=True) as ring, Correlator(N, C, T, bits=4, layout=CORR_L_CIT) as cor:
        for p in keep:
            assert ring.push(p) == CORR_OK
        ring.flush()
        dev = torch.empty(T * C * N, dtype=torch.uint8, device="cuda")
        cit = torch.empty(T * C * N, dtype=torch.uint8, device="cuda")
        want = None
        for _ in range(2):
            data, info = ring.next(0)
            dev.copy_(torch.from_numpy(data.reshape(-1)))
            ring.turn(dev, cit)
            cor.push(cit, seq=info["index"])
            cor.sync()
            ring.release()
            want = oracle.correlate(assembled[info["index"]][0].reshape(-1), N, C, T,
                                    layout=oracle.L_TCI, out=want)
        vis = cor.dump()
    assert np.array_equal(vis, want)


@pytest.mark.gpu
def test_packets_to_visibilities():
    """Packets of two blocks (one with losses) -> ring -> corr_push with the
    block number as sequence number -> the X-engine oracle's visibilities of
    the zero-filled blocks."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1904_07778_gb300 import build
    build.build()
    from paper_1904_07778_gb300.xengine import CORR_L_TCI, Correlator
    rng = np.random.default_rng(8)
    blocks = _blocks(2, seed=9)
    pk = _stream(blocks, first=40)
    keep = [p for p in pk if rng.random() > 0.1]
    with _ring() as ring, Correlator(N, C, T, bits=4, layout=CORR_L_TCI) as cor:
        for p in keep:
            assert ring.push(p) == CORR_OK
        ring.flush()
        want = None
        assembled, _ = op.assemble(keep, 3, 4, 2, 8, T)
        for _ in range(2):
            data, info = ring.next(0)
            cor.push(data, seq=info["index"])
            cor.sync()
            ring.release()
            want = oracle.correlate(assembled[info["index"]][0].reshape(-1), N, C, T,
                                    layout=oracle.L_TCI, out=want)
        vis = cor.dump()
    assert np.array_equal(vis, want)
