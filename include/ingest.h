/*
 * ingest.h -- C ABI of the packet assembler between the F-engines and the
 * X-engine (arXiv:1904.07778, Sec. 2.3 "Network and Data Packet", and the
 * Hashpipe ring buffers of Sec. 2.2).
 *
 * Packet (UDP payload) format, one reading of Sec. 2.3:
 *   bytes 0..5   MCNT, the packet counter, big-endian; MCNT m carries
 *                spectra 8m .. 8m+7
 *   byte  6      Fid, the F-engine: inputs Fid * n_inputs_pkt + (0 .. n_inputs_pkt-1)
 *   byte  7      Xid, the band: channels Xid * n_chans_pkt + (0 .. n_chans_pkt-1)
 *   bytes 8..    payload, 8 x n_chans_pkt x n_inputs_pkt bytes in
 *                [spectrum][channel][input] order, one packed 4+4-bit complex
 *                sample per byte (the X-engine's 4-bit encoding)
 *   last 8       4 zero bytes, then the IEEE 802.3 CRC-32 of header and
 *                payload, big-endian (pk_crc32)
 * 32 channels x 32 inputs gives the paper's 8208-byte packet.
 *
 * Blocks: block b holds MCNT b T/8 .. (b+1) T/8 - 1 of every (Fid, Xid)
 * stream as one [t][c][i] byte array (CORR_L_TCI of xengine.h) of T spectra,
 * C = n_xids n_chans_pkt channels and N = n_fids n_inputs_pkt inputs -- the
 * block corr_push takes.  A packet that never arrives leaves zeros (integrated
 * as nothing) and is reported.  With PK_F_PACKET_ORDER each payload is instead
 * copied whole, in arrival-slot order, and pk_turn reorders the block on the
 * GPU: one 8 KB copy per packet on the host instead of 8 n_chans_pkt rows.
 *
 * Ring: n_segments block buffers (3 in the paper's Hashpipe setup), each
 * free, open (filling), closed (complete or given up) or handed out.  A block
 * closes when all its packets are in, when a packet n_segments or more blocks
 * newer arrives, when a newer block needs a segment and none is free (the
 * oldest open block is closed to make progress), or at pk_flush.  Closed
 * blocks are handed out in block order.  Per (Fid, Xid) stream, every forward
 * jump of MCNT by more than one is counted as a gap (the paper's loss check).
 *
 * Thread safety: every call may come from any thread; one producer thread
 * calling pk_push and one consumer thread calling pk_next / pk_release is the
 * intended use.  Status codes are xengine.h's CORR_* values.
 */
#pragma once
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pk_ring pk_ring;

typedef struct pk_layout {
  int n_fids;        /* F-engines (groups of inputs), 1 .. 256            */
  int n_inputs_pkt;  /* inputs per packet                                 */
  int n_xids;        /* bands, 1 .. 256                                   */
  int n_chans_pkt;   /* channels per packet                               */
  int n_time;        /* spectra per block, a positive multiple of 8       */
} pk_layout;

#define PK_F_NO_CRC 0x1u        /* accept packets without checking the CRC     */
#define PK_F_PACKET_ORDER 0x2u  /* blocks in packet order (see pk_turn)         */

typedef struct pk_block {
  const uint8_t* data;      /* [T][C][N] bytes -- or, with PK_F_PACKET_ORDER,
                               [T/8][n_fids][n_xids][8][n_chans_pkt][n_inputs_pkt]:
                               each payload as it arrived, one contiguous copy --
                               owned by the ring (page-locked
                               when a CUDA device is present); valid until
                               pk_release                                    */
  uint64_t index;           /* block number b                                */
  uint64_t mcnt0;           /* b T / 8, its first MCNT                       */
  int n_packets;            /* packets of a complete block: T/8 n_fids n_xids */
  int n_missing;            /* of those never received (zeros in data)      */
  const uint8_t* received;  /* [T/8][n_fids][n_xids], 1 = received          */
} pk_block;

typedef struct pk_stats {
  uint64_t packets;          /* placed into a block                          */
  uint64_t bad_length;       /* wrong size                                   */
  uint64_t bad_crc;          /* CRC mismatch                                 */
  uint64_t bad_id;           /* Fid or Xid out of range                      */
  uint64_t late;             /* for a block already closed or handed out     */
  uint64_t duplicate;        /* a second copy of a placed packet             */
  uint64_t missing;          /* never received, over all closed blocks       */
  uint64_t mcnt_gaps;        /* forward MCNT jumps > 1, per (Fid, Xid) stream */
  uint64_t mcnt_skipped;     /* packets those jumps skipped                  */
  uint64_t blocks;           /* blocks closed                                */
  uint64_t blocks_with_loss; /* closed with n_missing > 0                    */
  uint64_t busy;             /* pushes refused with CORR_EBUSY               */
} pk_stats;

/*
 * pk_create -- a ring of n_segments (>= 2) block buffers for the layout.
 * CORR_EINVAL for a bad layout or flags, CORR_ENOMEM.
 */
int pk_create(const pk_layout* layout, int n_segments, unsigned flags, pk_ring** out);

/*
 * pk_push -- one packet.  CORR_OK: placed.  Dropped, with the reason
 * counted: CORR_EINVAL (length, Fid or Xid), CORR_ECORRUPT (CRC),
 * CORR_ESEQ (late or duplicate).  CORR_EBUSY: its block needs a segment and
 * none is free -- nothing was placed; retry after the consumer releases a
 * block (the oldest open block may have been closed meanwhile).
 */
int pk_push(pk_ring* ring, const void* packet, size_t len);

/*
 * pk_push_many -- n packets laid out stride bytes apart (a receive batch),
 * each of len bytes, pushed in order; codes (may be NULL) receives each
 * packet's pk_push status.  Stops at the first CORR_EBUSY and returns the
 * number of packets consumed (the refused one not included).
 */
size_t pk_push_many(pk_ring* ring, const void* packets, size_t n, size_t stride, size_t len,
                    int* codes);

/*
 * pk_next -- the oldest closed block, waiting up to timeout_ms (0 polls,
 * negative waits without limit).  CORR_ETIMEDOUT if none; CORR_ESTATE if a
 * block is already handed out and not released.
 */
int pk_next(pk_ring* ring, int timeout_ms, pk_block* out);

/* pk_release -- give back the block pk_next handed out.  CORR_ESTATE if none. */
int pk_release(pk_ring* ring);

/* pk_flush -- close every open block (end of the stream). */
int pk_flush(pk_ring* ring);

int pk_get_stats(pk_ring* ring, pk_stats* out);

/*
 * pk_turn -- GPU: a block in packet order (device memory, as a
 * PK_F_PACKET_ORDER ring hands it out, copied to the device) into the
 * X-engine's [c][i][t] order (CORR_L_CIT): out[(c N + i) out_stride + t]
 * with c = Xid n_chans_pkt + cc, i = Fid n_inputs_pkt + ii, t = 8 slot + tt.
 * out_stride >= n_time.  Queued on `stream` (a cudaStream_t, or NULL for the
 * legacy stream).  CORR_EINVAL for a bad layout, a host pointer, or
 * n_fids * n_xids > 65535.
 */
int pk_turn(const pk_layout* layout, const void* packets, void* out, long long out_stride,
            void* stream);

/* pk_crc32 -- IEEE 802.3 CRC-32 (reflected polynomial 0xEDB88320, initial and
 * final XOR 0xFFFFFFFF): the value a packet's trailer carries. */
uint32_t pk_crc32(const void* data, size_t n);

/* pk_destroy -- free the ring and its buffers.  NULL is ok. */
void pk_destroy(pk_ring* ring);

#ifdef __cplusplus
}
#endif
