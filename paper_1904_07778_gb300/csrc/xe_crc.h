// CRC-32 steps by the ARMv8 CRC instructions (xe_crc.cpp).  Host code.
#pragma once
#include <cstddef>
#include <cstdint>

namespace xe {
// True on a host whose CPU has the CRC instructions (aarch64 with CRC32).
bool crc32_hw_available();
// The raw CRC register c after the n bytes at p (only if crc32_hw_available()).
uint32_t crc32_raw_hw(uint32_t c, const uint8_t* p, size_t n);
// Four raw registers c[0..3] advanced in lockstep over the four consecutive
// segments of L bytes (L a multiple of 8) starting at p.
void crc32_raw4_hw(const uint8_t* p, size_t L, uint32_t c[4]);
}  // namespace xe
