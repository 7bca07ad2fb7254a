// CRC-32 steps by the ARMv8 CRC instructions, for the packet assembler's
// checks (Sec. 2.3 packets carry a CRC) on hosts that have them.  The
// instructions advance the raw CRC register (no initial or final inversion)
// by the reflected IEEE 802.3 polynomial 0xEDB88320: CRC32X over 8 bytes,
// CRC32B over one.  Host code, kept out of the CUDA sources because the
// compiler's ACLE header and CUDA's headers declare the same names.
#include <cstddef>
#include <cstdint>
#include <cstring>

#include "xe_crc.h"

#if defined(__aarch64__)
#include <arm_acle.h>
#include <sys/auxv.h>
#ifndef HWCAP_CRC32
#define HWCAP_CRC32 (1 << 7)
#endif

namespace xe {

bool crc32_hw_available() {
  static const bool ok = (getauxval(AT_HWCAP) & HWCAP_CRC32) != 0;
  return ok;
}

namespace {
__attribute__((target("+crc"))) inline uint32_t step8(uint32_t c, const uint8_t* p) {
  uint64_t v;
  std::memcpy(&v, p, 8);  // little endian: the CRC consumes the bytes in address order
  return __crc32d(c, v);
}
}  // namespace

__attribute__((target("+crc"))) uint32_t crc32_raw_hw(uint32_t c, const uint8_t* p, size_t n) {
  for (; n >= 8; p += 8, n -= 8) c = step8(c, p);
  for (; n; --n, ++p) c = __crc32b(c, *p);
  return c;
}

__attribute__((target("+crc"))) void crc32_raw4_hw(const uint8_t* p, size_t L, uint32_t c[4]) {
  const uint8_t *p1 = p + L, *p2 = p1 + L, *p3 = p2 + L;
  uint32_t c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
  for (size_t k = 0; k + 8 <= L; k += 8) {
    c0 = step8(c0, p + k);
    c1 = step8(c1, p1 + k);
    c2 = step8(c2, p2 + k);
    c3 = step8(c3, p3 + k);
  }
  c[0] = c0, c[1] = c1, c[2] = c2, c[3] = c3;
}

}  // namespace xe

#else  // no CRC instructions on this architecture: the table version runs

namespace xe {
bool crc32_hw_available() { return false; }
uint32_t crc32_raw_hw(uint32_t c, const uint8_t*, size_t) { return c; }
void crc32_raw4_hw(const uint8_t*, size_t, uint32_t*) {}
}  // namespace xe

#endif
