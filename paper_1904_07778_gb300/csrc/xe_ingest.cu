// Packet assembler between the F-engines and the X-engine (Sec. 2.3; the
// Hashpipe net thread and its ring of segments, Sec. 2.2): F-engine UDP
// payloads are checked (length, CRC-32, ids), placed into [t][c][i] blocks,
// and handed out in block order; lost packets leave zeros and are counted,
// and MCNT jumps are counted per (Fid, Xid) stream.  Host code.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "ingest.h"
#include "xe_crc.h"
#include "xe_internal.h"
#include "xengine.h"

namespace {

// ---------------------------------------------------------------- CRC-32
// Table-driven IEEE 802.3 CRC-32 (reflected polynomial 0xEDB88320),
// eight bytes per step with eight tables ("slicing by 8"): table t maps a
// byte to the CRC contribution of that byte followed by t zero bytes.
//
// One slicing chain is a serial dependency (each step needs the previous
// register), so a long message is cut into four equal segments whose
// registers advance in lockstep, and the four are joined afterwards.  The
// raw register (no initial or final inversion) is linear over GF(2):
// running segment B from register x gives R(B, 0) ^ x * x^(8|B|) mod P, so
//   R(S0 S1 S2 S3, init) = ((R(S0, init) X ^ R(S1, 0)) X ^ R(S2, 0)) X ^ R(S3, 0)
// with X = x^(8L) mod P for segments of L bytes; the remaining tail bytes
// continue from that register.
uint32_t g_crc[8][256];
std::once_flag g_crc_once;

void crc_tables() {
  for (uint32_t n = 0; n < 256; ++n) {
    uint32_t c = n;
    for (int k = 0; k < 8; ++k) c = (c & 1u) ? (c >> 1) ^ 0xEDB88320u : c >> 1;
    g_crc[0][n] = c;
  }
  for (int t = 1; t < 8; ++t)
    for (uint32_t n = 0; n < 256; ++n)
      g_crc[t][n] = (g_crc[t - 1][n] >> 8) ^ g_crc[0][g_crc[t - 1][n] & 0xFFu];
}

inline uint32_t load_le32(const uint8_t* p) {
  return (uint32_t)p[0] | (uint32_t)p[1] << 8 | (uint32_t)p[2] << 16 | (uint32_t)p[3] << 24;
}

// One slicing-by-8 step: register c after the 8 bytes at p.
inline uint32_t crc_step8(uint32_t c, const uint8_t* p) {
  const uint32_t a = c ^ load_le32(p);
  return g_crc[7][a & 0xFFu] ^ g_crc[6][(a >> 8) & 0xFFu] ^ g_crc[5][(a >> 16) & 0xFFu] ^
         g_crc[4][a >> 24] ^ g_crc[3][p[4]] ^ g_crc[2][p[5]] ^ g_crc[1][p[6]] ^ g_crc[0][p[7]];
}

// a * b mod P for polynomials in the reflected representation (bit 31 is
// the coefficient of x^0): the schoolbook product, reduced as it goes.
uint32_t gf2_mulmod(uint32_t a, uint32_t b) {
  uint32_t p = 0;
  for (int i = 0; i < 32; ++i, a <<= 1) {
    if (a & 0x80000000u) p ^= b;
    b = (b & 1u) ? (b >> 1) ^ 0xEDB88320u : b >> 1;  // b *= x
  }
  return p;
}

// x^(8 n) mod P by square and multiply.
uint32_t x8n_mod(uint64_t n) {
  uint32_t r = 0x80000000u, base = 0x00800000u;  // 1 and x^8
  for (; n; n >>= 1, base = gf2_mulmod(base, base))
    if (n & 1u) r = gf2_mulmod(r, base);
  return r;
}

uint32_t crc32(const uint8_t* p, size_t n) {
  // on CPUs with CRC instructions (xe_crc.cpp) those advance the registers;
  // the segments and their join are the same
  static const bool hw = xe::crc32_hw_available();
  if (!hw) std::call_once(g_crc_once, crc_tables);
  uint32_t c = 0xFFFFFFFFu;
  if (n >= 256) {
    const size_t L = (n / 4) & ~(size_t)7;  // bytes per segment, whole steps
    // every packet of a ring has the same length: keep the last constant
    thread_local size_t cached_L = 0;
    thread_local uint32_t cached_X = 0;
    if (cached_L != L) {
      cached_X = x8n_mod(L);
      cached_L = L;
    }
    const uint8_t *p1 = p + L, *p2 = p1 + L, *p3 = p2 + L;
    uint32_t c1 = 0, c2 = 0, c3 = 0;
    if (hw) {
      uint32_t r[4] = {c, 0u, 0u, 0u};
      xe::crc32_raw4_hw(p, L, r);
      c = r[0], c1 = r[1], c2 = r[2], c3 = r[3];
    } else {
      for (size_t k = 0; k < L; k += 8) {
        c = crc_step8(c, p + k);
        c1 = crc_step8(c1, p1 + k);
        c2 = crc_step8(c2, p2 + k);
        c3 = crc_step8(c3, p3 + k);
      }
    }
    const uint32_t X = cached_X;
    c = gf2_mulmod(gf2_mulmod(gf2_mulmod(c, X) ^ c1, X) ^ c2, X) ^ c3;
    p += 4 * L;
    n -= 4 * L;
  }
  if (hw) return xe::crc32_raw_hw(c, p, n) ^ 0xFFFFFFFFu;
  for (; n >= 8; p += 8, n -= 8) c = crc_step8(c, p);
  for (; n; --n, ++p) c = (c >> 8) ^ g_crc[0][(c ^ *p) & 0xFFu];
  return c ^ 0xFFFFFFFFu;
}

enum SegState { kFree, kOpen, kClosing, kClosed, kHanded };

struct Segment {
  uint8_t* data = nullptr;
  bool pinned = false;
  std::vector<uint8_t> received;  // [T/8][n_fids][n_xids]
  SegState state = kFree;
  uint64_t index = 0;
  int count = 0;     // packets claimed
  int inflight = 0;  // claimed packets whose payload copy has not landed
  int missing = 0;
};

}  // namespace

struct pk_ring {
  pk_layout L{};
  int n_seg = 0;
  unsigned flags = 0;
  int C = 0, N = 0, slots = 0, per_block = 0;
  size_t payload = 0, pkt_len = 0, block_bytes = 0;
  std::vector<Segment> seg;
  std::mutex mu;
  std::condition_variable cv;
  int handed = -1;
  uint64_t next_deliver = 0;        // blocks below it were handed out: late
  std::vector<int64_t> last_mcnt;   // per (Fid, Xid) stream, -1 before the first
  pk_stats st{};
};

namespace {

// Close a block: zero what never arrived and make it deliverable, or -- if
// copies are still landing -- mark it so that the last copy finishes it.
void close_segment(pk_ring* r, Segment& s) {
  if (s.inflight > 0) {
    s.state = kClosing;
    return;
  }
  const pk_layout& L = r->L;
  if (s.count < r->per_block && (r->flags & PK_F_PACKET_ORDER)) {
    for (size_t q = 0; q < (size_t)r->per_block; ++q)
      if (!s.received[q]) memset(s.data + q * r->payload, 0, r->payload);
  } else if (s.count < r->per_block) {  // zero what never arrived
    for (int slot = 0; slot < r->slots; ++slot)
      for (int f = 0; f < L.n_fids; ++f)
        for (int x = 0; x < L.n_xids; ++x) {
          if (s.received[((size_t)slot * L.n_fids + f) * L.n_xids + x]) continue;
          for (int tt = 0; tt < 8; ++tt)
            for (int cc = 0; cc < L.n_chans_pkt; ++cc)
              memset(s.data + (((size_t)slot * 8 + tt) * r->C + (size_t)x * L.n_chans_pkt + cc) * r->N +
                         (size_t)f * L.n_inputs_pkt,
                     0, L.n_inputs_pkt);
        }
  }
  s.missing = r->per_block - s.count;
  s.state = kClosed;
  ++r->st.blocks;
  r->st.missing += s.missing;
  if (s.missing) ++r->st.blocks_with_loss;
  r->cv.notify_all();
}

// The lowest-index segment that is open or closed (the next to hand out).
int lowest_pending(pk_ring* r) {
  int best = -1;
  for (int k = 0; k < r->n_seg; ++k) {
    const Segment& s = r->seg[k];
    if ((s.state == kOpen || s.state == kClosing || s.state == kClosed) &&
        (best < 0 || s.index < r->seg[best].index))
      best = k;
  }
  return best;
}

bool deliverable(pk_ring* r) {
  const int k = lowest_pending(r);
  return k >= 0 && r->seg[k].state == kClosed;
}

void free_ring(pk_ring* r) {
  for (Segment& s : r->seg) {
    if (!s.data) continue;
    if (s.pinned)
      cudaFreeHost(s.data);
    else
      free(s.data);
  }
  delete r;
}

// ---------------------------------------------------------------- push steps
// A packet whose slot is claimed: what its copy and its finish need.
struct Claim {
  const uint8_t* src;
  Segment* seg;
  uint8_t* dst;
  int slot, fid, xid;
};

// Length and CRC, without the lock.
int precheck(pk_ring* r, const uint8_t* p, size_t len) {
  if (len != r->pkt_len) return CORR_EINVAL;
  if (!(r->flags & PK_F_NO_CRC)) {
    const uint8_t* t = p + 8 + r->payload;
    const uint32_t want = (uint32_t)t[4] << 24 | (uint32_t)t[5] << 16 | (uint32_t)t[6] << 8 | t[7];
    if (t[0] | t[1] | t[2] | t[3] || crc32(p, 8 + r->payload) != want) return CORR_ECORRUPT;
  }
  return CORR_OK;
}

// Under the lock: count a packet that failed precheck.
int count_bad(pk_ring* r, int st, size_t len) {
  if (st == CORR_ECORRUPT)
    ++r->st.bad_crc;
  else if (len != r->pkt_len)
    ++r->st.bad_length;
  return st;
}

// Under the lock: ids, MCNT gaps, the block's segment (opening or closing
// blocks as the ring policy says), and the packet's slot.
int claim_locked(pk_ring* r, const uint8_t* p, Claim* c) {
  const pk_layout& L = r->L;
  uint64_t mcnt = 0;
  for (int k = 0; k < 6; ++k) mcnt = mcnt << 8 | p[k];
  const int fid = p[6], xid = p[7];
  if (fid >= L.n_fids || xid >= L.n_xids) {
    ++r->st.bad_id;
    return CORR_EINVAL;
  }
  int64_t& last = r->last_mcnt[(size_t)fid * L.n_xids + xid];
  if (last >= 0 && (int64_t)mcnt > last + 1) {
    ++r->st.mcnt_gaps;
    r->st.mcnt_skipped += (uint64_t)((int64_t)mcnt - last - 1);
  }
  if (last < 0 || (int64_t)mcnt > last) last = (int64_t)mcnt;

  const uint64_t b = mcnt / (uint64_t)r->slots;
  const int slot = (int)(mcnt % (uint64_t)r->slots);
  if (b < r->next_deliver) {
    ++r->st.late;
    return CORR_ESEQ;
  }
  int si = -1;
  for (int k = 0; k < r->n_seg; ++k)
    if (r->seg[k].state != kFree && r->seg[k].index == b) si = k;
  if (si >= 0 && r->seg[si].state != kOpen) {
    ++r->st.late;
    return CORR_ESEQ;
  }
  if (si < 0) {
    // blocks n_seg or more older than this one stop filling
    for (Segment& s : r->seg)
      if (s.state == kOpen && s.index + (uint64_t)r->n_seg <= b) close_segment(r, s);
    for (int k = 0; k < r->n_seg && si < 0; ++k)
      if (r->seg[k].state == kFree) si = k;
    if (si < 0) {
      // no room: give up on the oldest open block older than this one so
      // that the consumer can take it and free a segment
      int old = -1;
      for (int k = 0; k < r->n_seg; ++k)
        if (r->seg[k].state == kOpen && r->seg[k].index < b &&
            (old < 0 || r->seg[k].index < r->seg[old].index))
          old = k;
      if (old >= 0) close_segment(r, r->seg[old]);
      ++r->st.busy;
      return CORR_EBUSY;
    }
    Segment& s = r->seg[si];
    s.state = kOpen;
    s.index = b;
    s.count = 0;
    s.missing = 0;
    std::fill(s.received.begin(), s.received.end(), 0);
  }
  Segment& s = r->seg[si];
  uint8_t& got = s.received[((size_t)slot * L.n_fids + fid) * L.n_xids + xid];
  if (got) {
    ++r->st.duplicate;
    return CORR_ESEQ;
  }
  // claimed: the segment cannot be handed out or reused while the copy is
  // in flight
  got = 1;
  ++s.count;
  ++s.inflight;
  ++r->st.packets;
  *c = Claim{p, &s, s.data, slot, fid, xid};
  return CORR_OK;
}

// Without the lock: the payload into its place in the block.
void copy_payload(pk_ring* r, const uint8_t* p, const Claim& c) {
  const pk_layout& L = r->L;
  const uint8_t* pay = p + 8;
  if (r->flags & PK_F_PACKET_ORDER) {
    memcpy(c.dst + (((size_t)c.slot * L.n_fids + c.fid) * L.n_xids + c.xid) * r->payload, pay,
           r->payload);
  } else {
    for (int tt = 0; tt < 8; ++tt)
      for (int cc = 0; cc < L.n_chans_pkt; ++cc)
        memcpy(c.dst + (((size_t)c.slot * 8 + tt) * r->C + (size_t)c.xid * L.n_chans_pkt + cc) * r->N +
                   (size_t)c.fid * L.n_inputs_pkt,
               pay + ((size_t)tt * L.n_chans_pkt + cc) * L.n_inputs_pkt, L.n_inputs_pkt);
  }
}

// Under the lock: the copy has landed; the last copy of a complete or given-up
// block closes it.
void finish_locked(pk_ring* r, const Claim& c) {
  Segment& s = *c.seg;
  --s.inflight;
  if (s.inflight == 0 && (s.state == kClosing || (s.state == kOpen && s.count == r->per_block)))
    close_segment(r, s);
}

}  // namespace

extern "C" {

uint32_t pk_crc32(const void* data, size_t n) {
  return crc32(static_cast<const uint8_t*>(data), n);
}

int pk_create(const pk_layout* L, int n_segments, unsigned flags, pk_ring** out) {
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (!L || L->n_fids < 1 || L->n_fids > 256 || L->n_xids < 1 || L->n_xids > 256 ||
      L->n_inputs_pkt < 1 || L->n_chans_pkt < 1 || L->n_time < 8 || L->n_time % 8 ||
      n_segments < 2 || n_segments > 64 || (flags & ~(PK_F_NO_CRC | PK_F_PACKET_ORDER)))
    return CORR_EINVAL;
  pk_ring* r = new (std::nothrow) pk_ring;
  if (!r) return CORR_ENOMEM;
  r->L = *L;
  r->n_seg = n_segments;
  r->flags = flags;
  r->C = L->n_xids * L->n_chans_pkt;
  r->N = L->n_fids * L->n_inputs_pkt;
  r->slots = L->n_time / 8;
  r->per_block = r->slots * L->n_fids * L->n_xids;
  r->payload = (size_t)8 * L->n_chans_pkt * L->n_inputs_pkt;
  r->pkt_len = 8 + r->payload + 8;
  r->block_bytes = (size_t)L->n_time * r->C * r->N;
  r->last_mcnt.assign((size_t)L->n_fids * L->n_xids, -1);
  r->seg.resize(n_segments);
  for (Segment& s : r->seg) {
    // page-locked when a device is present, so corr_push copies it
    // asynchronously; plain memory otherwise
    if (cudaMallocHost(&s.data, r->block_bytes) == cudaSuccess) {
      s.pinned = true;
    } else {
      cudaGetLastError();
      s.data = static_cast<uint8_t*>(aligned_alloc(64, (r->block_bytes + 63) / 64 * 64));
    }
    if (!s.data) {
      free_ring(r);
      return CORR_ENOMEM;
    }
    s.received.assign((size_t)r->per_block, 0);
  }
  *out = r;
  return CORR_OK;
}

int pk_push(pk_ring* r, const void* packet, size_t len) {
  if (!r || !packet) return CORR_EINVAL;
  const uint8_t* p = static_cast<const uint8_t*>(packet);
  const int pre = precheck(r, p, len);  // outside the lock: producers may run in parallel
  std::unique_lock<std::mutex> g(r->mu);
  if (pre != CORR_OK) return count_bad(r, pre, len);
  Claim c;
  const int st = claim_locked(r, p, &c);
  if (st != CORR_OK) return st;
  g.unlock();
  copy_payload(r, p, c);
  g.lock();
  finish_locked(r, c);
  return CORR_OK;
}

size_t pk_push_many(pk_ring* r, const void* packets, size_t n, size_t stride, size_t len,
                    int* codes) {
  if (!r || !packets) return 0;
  const uint8_t* base = static_cast<const uint8_t*>(packets);
  constexpr size_t kBatch = 64;  // packets per lock acquisition
  int pre[kBatch];
  Claim claims[kBatch];
  for (size_t k0 = 0; k0 < n; k0 += kBatch) {
    const size_t nb = std::min(kBatch, n - k0);
    for (size_t i = 0; i < nb; ++i) pre[i] = precheck(r, base + (k0 + i) * stride, len);
    size_t nc = 0, stop = nb;
    {
      std::lock_guard<std::mutex> g(r->mu);
      for (size_t i = 0; i < nb; ++i) {
        const uint8_t* p = base + (k0 + i) * stride;
        int st = pre[i] != CORR_OK ? count_bad(r, pre[i], len) : claim_locked(r, p, &claims[nc]);
        if (st == CORR_EBUSY) {
          stop = i;
          break;
        }
        if (st == CORR_OK) claims[nc++].src = p;
        if (codes) codes[k0 + i] = st;
      }
    }
    for (size_t i = 0; i < nc; ++i) copy_payload(r, claims[i].src, claims[i]);
    {
      std::lock_guard<std::mutex> g(r->mu);
      for (size_t i = 0; i < nc; ++i) finish_locked(r, claims[i]);
    }
    if (stop < nb) return k0 + stop;
  }
  return n;
}

int pk_next(pk_ring* r, int timeout_ms, pk_block* out) {
  if (!r || !out) return CORR_EINVAL;
  std::unique_lock<std::mutex> g(r->mu);
  if (r->handed >= 0) return CORR_ESTATE;
  auto ready = [r] { return deliverable(r); };
  if (timeout_ms < 0)
    r->cv.wait(g, ready);
  else if (!r->cv.wait_for(g, std::chrono::milliseconds(timeout_ms), ready))
    return CORR_ETIMEDOUT;
  const int k = lowest_pending(r);
  Segment& s = r->seg[k];
  s.state = kHanded;
  r->handed = k;
  r->next_deliver = s.index + 1;
  out->data = s.data;
  out->index = s.index;
  out->mcnt0 = s.index * (uint64_t)r->slots;
  out->n_packets = r->per_block;
  out->n_missing = s.missing;
  out->received = s.received.data();
  return CORR_OK;
}

int pk_release(pk_ring* r) {
  if (!r) return CORR_EINVAL;
  std::lock_guard<std::mutex> g(r->mu);
  if (r->handed < 0) return CORR_ESTATE;
  r->seg[r->handed].state = kFree;
  r->handed = -1;
  r->cv.notify_all();
  return CORR_OK;
}

int pk_flush(pk_ring* r) {
  if (!r) return CORR_EINVAL;
  std::lock_guard<std::mutex> g(r->mu);
  for (Segment& s : r->seg)
    if (s.state == kOpen) close_segment(r, s);
  return CORR_OK;
}

int pk_get_stats(pk_ring* r, pk_stats* out) {
  if (!r || !out) return CORR_EINVAL;
  std::lock_guard<std::mutex> g(r->mu);
  *out = r->st;
  return CORR_OK;
}

int pk_turn(const pk_layout* L, const void* packets, void* out, long long out_stride,
            void* stream) {
  if (!L || !packets || !out || L->n_fids < 1 || L->n_xids < 1 || L->n_inputs_pkt < 1 ||
      L->n_chans_pkt < 1 || L->n_time < 8 || L->n_time % 8 || (long long)L->n_fids * L->n_xids > 65535 ||
      out_stride < L->n_time)
    return CORR_EINVAL;
  for (const void* p : {packets, (const void*)out}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return CORR_EINVAL;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return CORR_EINVAL;
  }
  const cudaError_t e = xe::pkt_turn_launch(static_cast<const uint8_t*>(packets),
                                            static_cast<uint8_t*>(out), L->n_fids, L->n_inputs_pkt,
                                            L->n_xids, L->n_chans_pkt, L->n_time, out_stride,
                                            (cudaStream_t)stream);
  return e == cudaSuccess ? CORR_OK : CORR_ECUDA;
}

void pk_destroy(pk_ring* r) {
  if (r) free_ring(r);
}

}  // extern "C"
