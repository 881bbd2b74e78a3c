// Layout constants and records of the archive format (version 1), as
// seen by the library's host code and kernels.
#pragma once
#include <cstdint>

namespace aceapex {

constexpr uint32_t kMaxSym = 16384;    // symbols per segment (rule R-sym)
constexpr uint32_t kLanes = 32;        // interleaved rANS lanes per segment
constexpr uint32_t kScaleBits = 12;    // rANS scale M = 4096
constexpr uint32_t kScale = 1u << kScaleBits;
constexpr uint32_t kRansL = 1u << 16;  // state interval [2^16, 2^32)
constexpr uint32_t kHeaderBytes = 128;
constexpr uint32_t kTablesBytes = 2048;
constexpr uint32_t kMaxLog2S = 14;     // segments are at most 16 KiB

// Segment directory record as stored in the archive (24 bytes).
struct SegRec {
  uint64_t payload_off;
  uint32_t n_words;
  uint32_t n_cmd;
  uint32_t n_lit;
  uint16_t level;
  uint16_t zero;
};
static_assert(sizeof(SegRec) == 24, "directory record is 24 bytes");

// Parsed header (the format's 128-byte header).
struct Header {
  uint64_t n;
  uint32_t log2_B, log2_S, W, min_match, max_level, flags;
  uint64_t D, n_seg, n_deps, n_reads;
  uint64_t off_tables, off_dir, off_dep_ptr, off_deps, off_reads, off_payload, payload_bytes, total_bytes;
};

inline uint64_t round16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

// smallest w >= 1 with 256^w >= n
inline uint32_t offset_width(uint64_t n) {
  uint32_t w = 1;
  while (w < 8 && n > (uint64_t(1) << (8 * w))) ++w;
  return w;
}

}  // namespace aceapex
