// Rules of the library encoder that its CPU and GPU implementations share,
// so that both write the same archive for the same input and parameters:
// the level schedule, the match-finder hash, the chain window and the
// table normalisation. (The format itself does not fix any of these; any
// encoder whose archive satisfies version 1 of the archive format is valid.)
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define ACE_HD __host__ __device__ __forceinline__
#else
#define ACE_HD inline
#endif

namespace aceapex {

constexpr uint32_t kChainDepth = 16;    // candidates tried per position
constexpr uint64_t kGoodEnough = 256;   // a match this long ends the chain walk
constexpr uint64_t kDistWindow = uint64_t(1) << 30;  // positions parsed per window when D > 0

// Level schedule: segment s may read segment q < s only if
// ruler_target(q) < ruler_target(s); then level(s) <= ruler_target(s) <= cap
// whatever the other segments' parses are (a "ruler": cap minus the number
// of trailing zero bits of s + 1, floored at 0).
ACE_HD uint32_t ruler_target(uint64_t s, uint32_t cap) {
#if defined(__CUDA_ARCH__)
  const uint32_t tz = (uint32_t)(__ffsll((long long)(s + 1)) - 1);
#else
  const uint32_t tz = (uint32_t)__builtin_ctzll(s + 1);
#endif
  return cap - (tz < cap ? tz : cap);
}

// Hash width for a chain window of len positions: 16..28 bits, at least
// twice as many buckets as positions while below 28 bits.
ACE_HD int hash_bits_for(uint64_t len) {
  int k = 16;
  while (k < 28 && (uint64_t(1) << k) < 2 * len) ++k;
  return k;
}

// Hash of up to 16 bytes given as two little-endian words (a = bytes 0..7,
// b = bytes 8..15, missing bytes zero), `bits` wide.
ACE_HD uint32_t hash_words(uint64_t a, uint64_t b, int bits) {
  const uint64_t v = a * 0x9E3779B97F4A7C15ull ^ (b + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
  return (uint32_t)((v ^ (v >> 29)) * 0xBF58476D1CE4E5B9ull >> (64 - bits));
}

// Hashed prefix length and sampling mask for a minimum match length: long
// minimum matches index and probe only positions whose hash has two zero
// low bits (content-defined anchors, then backward extension).
ACE_HD uint32_t hash_len_for(uint32_t min_match) { return min_match < 16 ? min_match : 16; }
ACE_HD uint32_t sample_mask_for(uint32_t min_match) {
  return min_match >= hash_len_for(min_match) + 16 ? 3u : 0u;
}

// Normalise symbol counts to frequencies summing to 4096 (every present
// symbol >= 1): rounding, then the sum is fixed on the most frequent symbols
// (ties: lowest symbol first). All zero when the class is empty.
void normalize_counts(const uint64_t *cnt, uint16_t *f);

}  // namespace aceapex
