// Per-pixel arithmetic of the u8 image stages, shared by the chain and stencil kernels.
//
// Noise stage: p' = clamp(p + (h mod 41) - 20, 0, 255) with h = F(F(F(seed) ^ x) ^ y) and F the
// MurmurHash3 32-bit finaliser; x, y are the global column and row of the stage's input. The
// kernels hoist the column part: colpre = c ^ (c >> 16) with c = F(F(seed) ^ x), and
// ypre = y ^ (y >> 16), so that F(c ^ y) = fmix32_tail(colpre ^ ypre).
// Solarise: p < 128 ? p : 255 - p. Threshold: (p >= t0) + (p >= t1).
// Byte arithmetic is SIMD within 32-bit words (byte k of a word = pixel k).
#pragma once

#include <stdint.h>

namespace mrw {

constexpr uint32_t kHi = 0x80808080u;
constexpr uint32_t kLo7 = 0x7F7F7F7Fu;

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// fmix32(v) with its first xor-shift already applied to v (the caller passes v ^ (v >> 16)).
__device__ __forceinline__ uint32_t fmix32_tail(uint32_t h) {
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Byte k of the result is 0xFF if byte k of w has its top bit set, else 0: prmt's default mode
// with the sign-replicate bit set in every selector nibble (selectors 8 + k).
__device__ __forceinline__ uint32_t sign_bytes(uint32_t w) {
  uint32_t d;
  asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(d) : "r"(w));
  return d;
}

__device__ __forceinline__ uint32_t solarise4(uint32_t w) {
  // p >= 128 -> 255 - p == p ^ 0xFF; the top bit of each byte selects the flip
  return w ^ sign_bytes(w);
}

// Per byte: 0x80 if a >= t, else 0. Setting a's top bits and clearing t's makes the subtraction
// borrow-free across bytes; its top bit then compares the low 7 bits, and the top bits of a and t
// decide the rest. tlo = t & 0x7F7F7F7F.
__device__ __forceinline__ uint32_t ge4(uint32_t a, uint32_t t, uint32_t tlo) {
  const uint32_t d = (a | kHi) - tlo;
  return ((a & ~t) | (~(a ^ t) & d)) & kHi;
}

// Labels (a >= t0) + (a >= t1) of the 4 bytes of a (t0, t1 replicated into every byte).
__device__ __forceinline__ uint32_t thresh4(uint32_t a, uint32_t t0, uint32_t t1) {
  return (ge4(a, t0, t0 & kLo7) >> 7) + (ge4(a, t1, t1 & kLo7) >> 7);
}

// (z ^ (z >> 16)) mod 41: the finaliser's last xor-shift and the modulo together. With zh = z >> 16
// the value is zh 2^16 + ((z ^ zh) & 0xFFFF) and 2^16 = 18 (mod 41), so it is congruent to
// s = 18 zh + ((z ^ zh) & 0xFFFF) < 2^21. The quotient s / 41 is mulhi(s, 104755328), where
// 104755328 = 32 ceil(2^27 / 41): division by an invariant integer as a multiplication
// (Granlund and Montgomery, 1994), exact for every s below 2^21 (checked exhaustively). Only the
// shift and the xor use the integer ALU pipe; the rest runs on the multiply pipe.
__device__ __forceinline__ uint32_t mix_tail_mod41(uint32_t z) {
  const uint32_t zh = z >> 16;
  const uint32_t s = 18u * zh + ((z ^ zh) & 0xFFFFu);
  return s - 41u * __umulhi(s, 104755328u);
}

// h mod 41 of one pixel's hash h = F(colpre ^ ypre).
__device__ __forceinline__ uint32_t noise_r(uint32_t colpre, uint32_t ypre) {
  uint32_t h = (colpre ^ ypre) * 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  return mix_tail_mod41(h);
}

// The noise stage on the 4 pixels of a word (pixel k's colpre in ck), as
// max(min(p + r, 275) - 20, 0): pixels 0, 2 and 1, 3 go through the clamp two at a time in
// 16-bit lanes (an add-and-compare instruction per bound and pair).
__device__ __forceinline__ uint32_t noise4(uint32_t q, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t ypre) {
  const uint32_t r02 = noise_r(c0, ypre) + noise_r(c2, ypre) * 0x10000u;
  const uint32_t r13 = noise_r(c1, ypre) + noise_r(c3, ypre) * 0x10000u;
  const uint32_t p02 = __byte_perm(q, 0, 0x4240), p13 = __byte_perm(q, 0, 0x4341);
  const uint32_t t02 = __viaddmax_s16x2(__viaddmin_s16x2(p02, r02, 0x01130113u), 0xFFECFFECu, 0u);
  const uint32_t t13 = __viaddmax_s16x2(__viaddmin_s16x2(p13, r13, 0x01130113u), 0xFFECFFECu, 0u);
  return t02 + t13 * 0x100u;  // bytes 0, 2 and 1, 3: the add does not carry
}

__device__ __forceinline__ uint32_t noise4(uint32_t q, const uint32_t (&c)[4], uint32_t ypre) {
  return noise4(q, c[0], c[1], c[2], c[3], ypre);
}

}  // namespace mrw
