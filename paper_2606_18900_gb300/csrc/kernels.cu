// GB300 (sm_103a) kernels of the device-resident decode path.
//
// decode_kernel — one persistent launch decodes a list of segments (paper
// §3.3 full pipeline; §4 range decode; §5 chunked range decode). Each warp
// repeatedly takes the next work item from a global counter; the list is in
// level order, so every segment a warp waits for was taken earlier by a warp
// that is running (no deadlock, every source segment has a lower dependency level). Per segment (details at
// decode_segment):
//   1. rANS over the three command classes (the format's rANS coding): the 32 lanes run
//      the 32 interleaved states; each step's renormalisation words are handed
//      out in ascending lane order with a ballot + popc, from a shared-memory
//      ring that cp.async keeps filled ahead of the reader.
//   2. command parse: 32 commands at a time, positions from warp scans, every
//      command rule checked, source segments checked (level below
//      ours, present in the view).
//   3. rANS over the literal class, each literal stored straight to its
//      output position.
//   4. bounded waits on the ready flags of source segments, then match copies
//      in hazard-free rounds spread over the lanes.
//   5. publish: the warp synchronises (which orders every lane's output
//      stores before what lane 0 does next), then lane 0 stores the level and
//      epoch into the segment's flag with release semantics, a release that
//      covers the other lanes' stores through that ordering.
// Errors latch the first code into a device word; waits give up at a time
// limit (globaltimer) or as soon as another warp has latched an error.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace aceapex {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ void latch(uint32_t *err, uint32_t code) { atomicCAS(err, 0u, code); }

// address of absolute position p in view v; nullptr when p's page is absent
__device__ __forceinline__ uint8_t *at(const OutView &v, uint64_t p, uint32_t log2_S) {
  if (v.page) {
    uint32_t slot = v.page[p >> log2_S];
    if (slot == 0xFFFFFFFFu) return nullptr;
    return v.slot_base + ((uint64_t)slot << log2_S) + (p & ((uint64_t(1) << log2_S) - 1));
  }
  return v.base + ((p - v.origin) & v.mask);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
// with an L2 cache policy
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol) : "memory");
}
// L2 policy for data read once (the payload): evicted first, so that the
// output, which matches read back, stays longer
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// inclusive warp scan of a 32-bit value
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

// Wait until every lane with `need` sees *flag == epoch. False on timeout or
// when another warp has latched an error. Lane 0 reads the error word and
// the clock and decides for the warp (see take_item).
__device__ bool wait_flags(const uint64_t *flag, bool need, uint32_t epoch, uint64_t deadline, uint32_t *err,
                           int lane) {
  for (uint32_t spin = 0;; ++spin) {
    bool ok = !need || (uint32_t)ld_acquire(flag) == epoch;
    if (__all_sync(kFull, ok)) return true;
    uint32_t why = 0;
    if (lane == 0) why = ld_relaxed(err) != 0 ? 1u : now_ns() > deadline ? 2u : 0u;
    why = __shfl_sync(kFull, why, 0);
    if (why) {
      if (why == 2 && lane == 0) latch(err, kErrTimeout);
      return false;
    }
    __nanosleep(spin < 8 ? 64 : spin < 32 ? 256 : 1024);
  }
}

// The warp's next work index (lane 0's atomic on counter) and whether the
// error word is set, both read by lane 0 and broadcast, so that every lane
// takes the same branch: lanes that read the error word themselves could see
// different values while another warp latches it, and a warp whose lanes part
// there would meet at different warp-synchronous calls.
__device__ __forceinline__ uint32_t take_item(uint32_t *counter, const uint32_t *err, int lane, bool &failed) {
  uint32_t idx = 0, e = 0;
  if (lane == 0) {
    idx = atomicAdd(counter, 1u);
    e = ld_relaxed(err);
  }
  idx = __shfl_sync(kFull, idx, 0);
  failed = __shfl_sync(kFull, e, 0) != 0;
  return idx;
}

// u16 little-endian at p (2-byte aligned)
__device__ __forceinline__ uint32_t ld16(const uint8_t *p) { return *reinterpret_cast<const uint16_t *>(p); }
__device__ __forceinline__ void st16(uint8_t *p, uint32_t v) { *reinterpret_cast<uint16_t *>(p) = (uint16_t)v; }

constexpr int kViewLinear = 0, kViewRing = 1, kViewPaged = 2;

// address of source position p in view v (its page is known to be present)
template <int kMode>
__device__ __forceinline__ const uint8_t *src_at(const OutView &v, uint64_t p, uint32_t log2_S) {
  if (kMode == kViewPaged) return at(v, p, log2_S);
  if (kMode == kViewRing) return v.base + ((p - v.origin) & v.mask);
  return v.base + (p - v.origin);
}

// r = bytes c .. c+15 of the 32 bytes X || Y (bytes past the end read as 0)
__device__ __forceinline__ void realign16(uint4 X, uint4 Y, uint32_t c, uint32_t r[4]) {
  const uint32_t w[12] = {X.x, X.y, X.z, X.w, Y.x, Y.y, Y.z, Y.w, 0u, 0u, 0u, 0u};
  const uint32_t k = c >> 2, sh = 8 * (c & 3);
  uint32_t s4[8], s2[6], s1[5];
#pragma unroll
  for (int j = 0; j < 8; ++j) s4[j] = (k & 4) ? w[j + 4] : w[j];
#pragma unroll
  for (int j = 0; j < 6; ++j) s2[j] = (k & 2) ? s4[j + 2] : s4[j];
#pragma unroll
  for (int j = 0; j < 5; ++j) s1[j] = (k & 1) ? s2[j + 1] : s2[j];
#pragma unroll
  for (int j = 0; j < 4; ++j) r[j] = __funnelshift_r(s1[j], s1[j + 1], sh);
}

// Per-warp shared table of the matches copied in one round.
struct MatchTable {
  uint64_t src[32];
  uint64_t dst[32];   // absolute positions
  uint32_t len[32];   // match length
  uint32_t start[33]; // first 16-byte unit of each lane's match in the round; start[32] = round total
  uint32_t pad[3];    // keeps the size a multiple of 16
};

// 16- and 32-bit loads through 32-bit shared-window addresses (volatile:
// they must stay behind the cp.async waits that fill the word ring)
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_u8(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_u16(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((uint16_t)v) : "memory");
}

// The command staging area of a warp: shared memory (kShared, read and
// written through its shared-window address), or a generic pointer to shared
// memory or to the warp's global slot for segments whose command streams do
// not fit. Byte offsets; the area is 4-byte aligned.
template <bool kShared>
struct Stage {
  uint8_t *p;
  uint32_t s;  // shared-window address of p (kShared)
  __device__ __forceinline__ uint32_t u16(uint32_t o) const {
    if (kShared) return lds_u16(s + o);
    return *reinterpret_cast<const uint16_t *>(p + o);
  }
  __device__ __forceinline__ uint32_t u32(uint32_t o) const {
    if (kShared) return lds_u32(s + o);
    return *reinterpret_cast<const uint32_t *>(p + o);
  }
  __device__ __forceinline__ void st8(uint32_t o, uint32_t v) const {
    if (kShared) asm volatile("st.shared.u8 [%0], %1;" ::"r"(s + o), "r"(v) : "memory");
    else p[o] = (uint8_t)v;
  }
  __device__ __forceinline__ void st16(uint32_t o, uint32_t v) const {
    if (kShared) asm volatile("st.shared.u16 [%0], %1;" ::"r"(s + o), "h"((uint16_t)v) : "memory");
    else *reinterpret_cast<uint16_t *>(p + o) = (uint16_t)v;
  }
  __device__ __forceinline__ void st32(uint32_t o, uint32_t v) const {
    if (kShared) asm volatile("st.shared.u32 [%0], %1;" ::"r"(s + o), "r"(v) : "memory");
    else *reinterpret_cast<uint32_t *>(p + o) = v;
  }
  // W-byte little-endian value at offset o (1 <= W <= 8); reads only the
  // aligned 4-byte words that hold bytes of [o, o + W), so never past the
  // word that holds byte o + W - 1
  __device__ __forceinline__ uint64_t le(uint32_t o, uint32_t W) const {
    const uint32_t a = o & ~3u, sh = 8 * (o & 3u), span = (o & 3u) + W;
    const uint32_t w0 = u32(a);
    const uint32_t w1 = span > 4 ? u32(a + 4) : 0u;
    uint64_t v = __funnelshift_r(w0, w1, sh);
    if (W > 4) {
      const uint32_t w2 = span > 8 ? u32(a + 8) : 0u;
      v |= (uint64_t)__funnelshift_r(w1, w2, sh) << 32;
    }
    return W >= 8 ? v : v & ((uint64_t(1) << (8 * W)) - 1);
  }
};

#ifdef ACEAPEX_PHASE_CLOCKS
// Warp-cycle counters per phase (instrumented build only): 0 command-class
// rANS, 1 command parse, 2 literal rANS and placement, 3 source checks of
// the match chunks,
// 4 match copies, 5 the rest of the work loop; then event counts: 6 match
// chunks, 7 copy rounds, 8 copy units, 9 segments, 10 chunks whose source
// flags were not all set at the first reading; 11 warp cycles spent waiting
// for those flags (counted apart from phase 3, the chunks' source checks).
__device__ unsigned long long g_phase_cycles[16];
#define PHASE_COUNT(i, v) \
  do {                    \
    if (lane == 0) ph[i] += (v); \
  } while (0)
#define PHASE_MARK(i)                    \
  do {                                   \
    if (lane == 0) {                     \
      const uint64_t t_ = clock64();     \
      ph[i] += t_ - ph_t;                \
      ph_t = t_;                         \
    }                                    \
  } while (0)
#else
#define PHASE_MARK(i) \
  do {                \
  } while (0)
#define PHASE_COUNT(i, v) \
  do {                    \
  } while (0)
#endif

// Decode one segment into view V and publish its ready flag.
//
// lut: the 4 x 4096-entry decode table (kSmemLut: at shared-window address
// lut_s; otherwise global lut). st: the warp's command staging area. mt: the
// warp's shared match table; ring_s: shared-window address of the warp's
// 1,280-byte renormalisation-word ring (16-byte aligned).
//
// Phases: (1) rANS over the three command classes into the staging area;
// (2) parse, scans and the checks of every command, rewriting each command's
// literal-run length in place as the inclusive literal prefix (the run's end
// in literal numbering); (3) rANS over the literal class, each literal stored
// straight to its output position: the literals of one step are consecutive
// in literal numbering, so a warp-uniform cursor walks the command boundaries
// that fall inside the step and moves the per-lane output pointers of the
// lanes past each boundary by that command's match length; (4) per 32-command
// chunk: source levels (and pages) checked, bounded waits on the source
// segments' flags, then match copies in rounds: a round copies every pending
// match whose source does not overlap the output of an earlier pending match,
// the bytes of the round spread over all lanes; (5) publish.
template <bool kSmemLut, int kMode, bool kSharedStage>
__device__ __forceinline__ void decode_segment_impl(const DecodeLaunch &L, const DevArchive &A, const OutView &V,
                                                    uint32_t seg, uint32_t epoch, const uint32_t *lut,
                                                    uint32_t lut_s, const Stage<kSharedStage> st, MatchTable *mt,
                                                    uint32_t ring_s, int lane, const SegRec &d, uint64_t *ph,
                                                    uint64_t &ph_t) {
  (void)ph;
  (void)ph_t;
  const uint32_t log2_S = A.log2_S;
  const uint64_t seg_start = (uint64_t)seg << log2_S;
  const uint64_t rem = A.n - seg_start;
  const uint32_t out_size = rem < (uint64_t(1) << log2_S) ? (uint32_t)rem : (1u << log2_S);
  const uint32_t nc = d.n_cmd, nl = d.n_lit, nw = d.n_words, W = A.W, mm = A.min_match;
  const uint32_t b1 = 2 * nc, b2 = 4 * nc, b3 = (4 + W) * nc, n_sym = b3 + nl;
  // the segment's own output is contiguous in every view
  uint8_t *const out = at(V, seg_start, log2_S);
  bool ok = out != nullptr;
  // aligned 16-byte blocks of the view never straddle a segment (hence no ring
  // wrap or page boundary either)
  const bool vec =
      log2_S >= 4 && (kMode == kViewPaged  ? (reinterpret_cast<uintptr_t>(V.slot_base) & 15) == 0
                      : kMode == kViewRing ? ((reinterpret_cast<uintptr_t>(V.base) | V.origin) & 15) == 0
                                           : ((reinterpret_cast<uintptr_t>(V.base) - V.origin) & 15) == 0);

  // ---------------------------------------------------------------- rANS
  const uint8_t *pl = A.payload + d.payload_off;
  uint32_t x = __ldg(reinterpret_cast<const uint32_t *>(pl) + lane);
  if (!__all_sync(kFull, x >= kRansL)) ok = false;
  // Renormalisation words go through a 512-word ring in shared memory, filled
  // by cp.async in blocks of 128 words two blocks ahead of the reader, so the
  // decode never waits on a global load between block boundaries. Block slot
  // 0 is also copied to the 256 bytes after the ring (lanes 16..31 make that
  // copy), so the words of the next four steps are always contiguous from
  // the read address wr: no step masks its address. A lane copies a 16-byte
  // chunk only if it starts before the segment's last word; the payload is
  // padded to 16 bytes, so no copy leaves the archive.
  const uint8_t *wsrc = pl + 128;
  const uint64_t pol = policy_evict_first();
  auto fetch = [&](uint32_t blk) {
    const uint32_t wi = blk * 128 + (uint32_t)(lane & 15) * 8;
    const uint32_t to = ring_s + (lane < 16 ? (blk & 3) * 256 : 1024u) + (lane & 15) * 16;
    if ((lane < 16 || (blk & 3) == 0) && wi < nw) cp_async16(to, wsrc + (size_t)wi * 2, pol);
    cp_async_commit();
  };
  fetch(0);
  fetch(1);
  fetch(2);
  fetch(3);
  cp_async_wait<2>();
  __syncwarp();
  // blk: the block being read; wr: shared address of the next word; bnd: end
  // of blk's slot (wr moves on into the next slot, or into the copy of slot
  // 0, which it leaves for slot 0 itself when blk advances)
  uint32_t blk = 0, wr = ring_s, bnd = ring_s + 256;
  const uint32_t lt = lanemask_lt();
  // after the step that consumed the last word of a block: reuse its slot
  auto advance = [&]() {
    if (wr >= bnd) {
      ++blk;
      bnd += 256;
      if (bnd > ring_s + 1024) {
        wr -= 1024;
        bnd -= 1024;
      }
      __syncwarp();
      fetch(blk + 3);
      cp_async_wait<2>();
      __syncwarp();
    }
  };
  // table entry of slot (class << 12 | x mod 4096)
  auto entry = [&](uint32_t idx) -> uint32_t {
    if (kSmemLut) return lds_u32(lut_s + 4 * idx);
    return __ldg(lut + idx);
  };
  // lanes whose state fell below 2^16 read the next words in ascending lane
  // order (every lane reads a ring word; only those lanes use it)
  auto renorm = [&](bool need) {
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t w = lds_u16(wr + 2 * __popc(m & lt));
    if (need) x = __byte_perm(w, x, 0x5410);  // x << 16 | w
    wr += 2 * __popc(m);
  };
  // one interleaved step of the command classes: lane j decodes symbol q
  auto cmd_step = [&](uint32_t q) -> uint32_t {
    const bool active = q < n_sym;
    const uint32_t cls = (uint32_t)(q >= b1) + (uint32_t)(q >= b2) + (uint32_t)(q >= b3);
    uint32_t sym = 0;
    if (active) {
      const uint32_t e = entry((cls << kScaleBits) | (x & (kScale - 1)));
      sym = e & 0xFFu;
      x = ((e >> 20) + 1u) * (x >> kScaleBits) + ((e >> 8) & 0xFFFu);
    }
    renorm(active && x < kRansL);
    return sym;
  };

  // Stage layout: command c's literal-run length and match length less
  // min_match as one 32-bit record (u16, u16) at 4 c, which the parse
  // replaces by the run's end in literal numbering and the match bytes of
  // commands 0..c (both below 2^16: a segment holds at most 16 KiB); at 4 nc
  // a sentinel record whose run end (65535) lies beyond every literal; the
  // W-byte offsets from 4 nc + 4. Symbol q of the command classes goes to
  // stage_off(q).
  auto stage_off = [&](uint32_t q) -> uint32_t {
    if (q < b1) return 4 * (q >> 1) + (q & 1);
    if (q < b2) return 4 * ((q - b1) >> 1) + 2 + ((q - b1) & 1);
    return q + 4;
  };
  const uint32_t offs = b2 + 4;  // the offsets' start

  // (1) command classes; the step that crosses into the literals keeps its
  // literal symbol in `pend` until the command prefixes exist. Four steps take
  // at most 128 words, so after an advance() (blocks blk and blk + 1 complete,
  // wr inside blk's slot) four steps read only those two blocks.
  uint32_t t0 = 0, pend = 0;
  if (ok) {
    // four steps inside one class: the table row is known for all lanes
    auto cls_step = [&](uint32_t row) -> uint32_t {
      const uint32_t e = entry(row | (x & (kScale - 1)));
      x = ((e >> 20) + 1u) * (x >> kScaleBits) + ((e >> 8) & 0xFFFu);
      renorm(x < kRansL);
      return e & 0xFFu;
    };
    for (; t0 + 128 <= b3; t0 += 128) {
      const uint32_t c_lo = (uint32_t)(t0 >= b1) + (uint32_t)(t0 >= b2);
      const uint32_t c_hi = (uint32_t)(t0 + 127 >= b1) + (uint32_t)(t0 + 127 >= b2);
      if (c_lo == c_hi) {
        const uint32_t base = c_lo == 0 ? 0u : c_lo == 1 ? b1 : b2;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t k = t0 + 32 * u + lane - base;  // symbol number within the class
          st.st8(c_lo == 2 ? b2 + 4 + k : 4 * (k >> 1) + 2 * c_lo + (k & 1), cls_step(c_lo << kScaleBits));
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) st.st8(stage_off(t0 + 32 * u + lane), cmd_step(t0 + 32 * u + lane));
      }
      advance();
    }
    for (; t0 < b3; t0 += 32) {
      const uint32_t q = t0 + lane;
      const uint32_t sym = cmd_step(q);
      if (q < b3) st.st8(stage_off(q), sym);
      else pend = sym;
      advance();
    }
  }
  __syncwarp();
  PHASE_MARK(0);

  // (2) parse, prefixes, checks
  uint32_t tot_l = 0, tot_m = 0;
  for (uint32_t c0 = 0; ok && c0 < nc; c0 += 32) {
    const uint32_t c = c0 + lane;
    const bool valid = c < nc;
    uint32_t ll = 0, ml = 0;
    uint64_t src = 0;
    if (valid) {
      const uint32_t rec = st.u32(4 * c);
      ll = rec & 0xFFFFu;
      ml = (rec >> 16) + mm;
      src = W == 4 ? (uint64_t)st.u32(offs + 4 * c) : st.le(offs + W * c, W);  // (4-byte offsets are aligned)
    }
    const uint32_t inc_l = warp_incl_scan(ll, lane), inc_m = warp_incl_scan(ml, lane);
    const uint32_t lit_end = tot_l + inc_l, msum = tot_m + inc_m - ml;
    const uint32_t cend = lit_end + msum + ml;  // end of the command in the segment
    const uint64_t dst = seg_start + lit_end + msum;
    const bool bad = valid && ((uint64_t)cend > out_size || lit_end > nl || src + ml > dst || src + ml < src ||
                               (A.D && dst - src > A.D));
    if (__any_sync(kFull, bad)) {
      ok = false;
      break;
    }
    if (valid) st.st32(4 * c, lit_end | (msum + ml) << 16);
    tot_l += __shfl_sync(kFull, inc_l, 31);
    tot_m += __shfl_sync(kFull, inc_m, 31);
  }
  if (ok && (tot_l + tot_m > out_size || out_size - tot_m != nl)) ok = false;
  if (ok && lane == 0) st.st32(4 * nc, 0xFFFFu);
  __syncwarp();
  PHASE_MARK(1);

  // (3) literals. K0: literal number of lane 0 in the current step; E: end of
  // the literal run of command cu (literal number), the next boundary; Sc:
  // match bytes before the literals from the current boundary on (the
  // cumulative match length through command cu - 1); outK: the output
  // address of literal K0 before any match byte.
  if (ok) {
    int K0 = (b3 & 31u) ? (int)(b3 & ~31u) - (int)b3 : 0;
    uint32_t cu = 0, rec = st.u32(0), Sc = 0;
    int E = (int)(rec & 0xFFFFu);
    uint8_t *outK = out + K0;
    // The lane's offset for this step: lanes at or after a run end that lies
    // inside [K0, K0 + 32) take that command's cumulative match length.
    auto bound = [&]() -> uint32_t {
      uint32_t sl = Sc;
      while (E - K0 < 32) {
        Sc = rec >> 16;
        if (lane >= E - K0) sl = Sc;
        rec = st.u32(4 * ++cu);
        E = (int)(rec & 0xFFFFu);
      }
      return sl + (uint32_t)lane;
    };
    auto lit_rans = [&]() -> uint32_t {
      const uint32_t e = entry((3u << kScaleBits) | (x & (kScale - 1)));
      x = ((e >> 20) + 1u) * (x >> kScaleBits) + ((e >> 8) & 0xFFFu);
      renorm(x < kRansL);
      return e;
    };
    if (b3 & 31u) {  // the crossing step, decoded in (1)
      const uint32_t o = bound();
      if (lane >= -K0 && t0 - 32 + lane < n_sym) outK[o] = (uint8_t)pend;
      outK += 32;
      K0 += 32;
    }
    for (; t0 + 128 <= n_sym; t0 += 128) {
      if (E - K0 >= 128) {  // no run ends inside these four steps
        uint8_t *p = outK + (Sc + (uint32_t)lane);
#pragma unroll
        for (int u = 0; u < 4; ++u) p[32 * u] = (uint8_t)lit_rans();
      } else {
        // the same walk as bound(), with the next run end kept relative to
        // the block (D) and each lane's offset (ol) changed only at run ends,
        // so that a step without one costs a compare and its store
        int D = E - K0;
        uint32_t ol = Sc + (uint32_t)lane;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          uint32_t o = ol;
          while (D < 32 * (u + 1)) {  // a run end inside step u, at lane D - 32 u
            Sc = rec >> 16;
            ol = Sc + (uint32_t)lane;
            if (lane >= D - 32 * u) o = ol;
            rec = st.u32(4 * ++cu);
            E = (int)(rec & 0xFFFFu);
            D = E - K0;
          }
          outK[32 * u + o] = (uint8_t)lit_rans();
        }
      }
      K0 += 128;
      outK += 128;
      advance();
    }
    for (; t0 + 32 <= n_sym; t0 += 32) {
      const uint32_t o = bound();
      outK[o] = (uint8_t)lit_rans();
      outK += 32;
      K0 += 32;
      advance();
    }
    if (t0 < n_sym) {
      const bool active = t0 + lane < n_sym;
      const uint32_t o = bound();
      uint32_t e = 0;
      if (active) {
        e = entry((3u << kScaleBits) | (x & (kScale - 1)));
        x = ((e >> 20) + 1u) * (x >> kScaleBits) + ((e >> 8) & 0xFFFu);
      }
      renorm(active && x < kRansL);
      if (active) outK[o] = (uint8_t)e;
      t0 += 32;
    }
  }
  // words consumed: the blocks before the current ring cycle plus the offset
  // of wr in the ring (and its copy of slot 0)
  const uint32_t wb = (blk & ~3u) * 256 + (wr - ring_s);
  if (!__all_sync(kFull, x == kRansL) || wb != 2 * nw) ok = false;
  __syncwarp();
  PHASE_MARK(2);

  // (4) matches
  const uint32_t my_level = d.level;
  const uint64_t deadline = now_ns() + L.wait_ns;
  uint32_t mbase = 0;  // match bytes before the chunk
  for (uint32_t c0 = 0; ok && c0 < nc; c0 += 32) {
    const uint32_t c = c0 + lane;
    const bool valid = c < nc;
    uint32_t ml = 0, lend = 0, cum = 0;
    uint64_t src = 0;
    if (valid) {
      const uint32_t rec = st.u32(4 * c);
      cum = rec >> 16;
      lend = rec & 0xFFFFu;
      src = W == 4 ? (uint64_t)st.u32(offs + 4 * c) : st.le(offs + W * c, W);  // (4-byte offsets are aligned)
    }
    // match bytes of the commands before c (the previous lane's sum, or the
    // last sum of the previous chunk); this command's length is the difference
    const uint32_t up = __shfl_up_sync(kFull, cum, 1);
    const uint32_t before = lane ? up : mbase;
    if (valid) ml = cum - before;
    const uint64_t dst = valid ? seg_start + lend + before : ~uint64_t(0);
    mbase = __shfl_sync(kFull, cum, min(nc - 1 - c0, 31u));
    const uint64_t q0 = src >> log2_S, q1 = valid ? (src + ml - 1) >> log2_S : q0;
    // start moving the chunk's source bytes (the first and the last 128-byte
    // line of each match's) toward L2 while the checks and hazards run
    if (kMode != kViewPaged && valid) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(src_at<kMode>(V, src, log2_S)));
      if (((src ^ (src + ml - 1)) >> 7) != 0)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(src_at<kMode>(V, src + ml - 1, log2_S)));
    }
    const bool need0 = valid && q0 != seg;
    const bool need1 = valid && q1 != q0 && q1 != seg;
    // A source segment must have a lower level than ours (a wait on any other
    // could not end) and, in a paged view, be present. Its level is the high
    // half of its flag word, read in the same load as its epoch.
    bool bad = false;
    uint32_t f0 = epoch, f1 = epoch;
    if (need0) {
      const uint64_t f = ld_acquire(A.flags + q0);
      bad |= (uint32_t)(f >> 32) >= my_level;
      if (kMode == kViewPaged) bad |= V.page[q0] == 0xFFFFFFFFu;
      f0 = (uint32_t)f;
    }
    if (need1) {
      const uint64_t f = ld_acquire(A.flags + q1);
      bad |= (uint32_t)(f >> 32) >= my_level;
      if (kMode == kViewPaged) bad |= V.page[q1] == 0xFFFFFFFFu;
      f1 = (uint32_t)f;
    }
    // (the hazard ranges need no flag: they are found while the loads above
    // are in flight, and the loaded values are used only after them)
    // linear view: the table holds each match's source address
    mt->src[lane] = kMode == kViewLinear ? (uint64_t)reinterpret_cast<uintptr_t>(V.base + (src - V.origin)) : src;
    mt->dst[lane] = dst;
    __syncwarp();
    // The earlier matches of this chunk whose outputs overlap this match's
    // source: outputs are disjoint and ascending, so they are the lanes j with
    // dst_j < src + ml and dst_j + ml_j > src, a contiguous range [jlo, jhi]
    // found by two binary searches (offsets from the segment start; a source
    // that ends before the segment overlaps nothing); all lie below this lane
    // because src + ml <= dst.
    uint32_t hmask = 0;
    {
      const uint64_t se = src + ml;
      const uint32_t se_rel = valid && se > seg_start ? (uint32_t)(se - seg_start) : 0u;
      const uint32_t s_rel = valid && src > seg_start ? (uint32_t)(src - seg_start) : 0u;
      const uint32_t d_off = valid ? (uint32_t)(dst - seg_start) : 0xFFFFFFFFu;
      const uint32_t d_end = valid ? d_off + ml : 0xFFFFFFFFu;
      // (no search when every source ends before the chunk's first output)
      if (__any_sync(kFull, se_rel > __shfl_sync(kFull, d_off, 0))) {
        uint32_t jh = 0, jl = 0;
#pragma unroll
        for (int s = 16; s; s >>= 1) {
          if (__shfl_sync(kFull, d_off, jh + s) < se_rel) jh += s;
          if (__shfl_sync(kFull, d_end, jl + s) <= s_rel) jl += s;
        }
        const bool any_h = __shfl_sync(kFull, d_off, jh) < se_rel;  // some output starts before the source ends
        const bool any_l = __shfl_sync(kFull, d_end, jl) <= s_rel;  // some output ends before the source starts
        const uint32_t jlo = any_l ? jl + 1 : 0;
        if (any_h && jlo <= jh) hmask = ((2u << jh) - 1u) & ~((1u << jlo) - 1u);
      }
    }
    if (__any_sync(kFull, bad)) {
      ok = false;
      break;
    }
    if (!__all_sync(kFull, f0 == epoch && f1 == epoch)) {
      PHASE_COUNT(10, 1);
      PHASE_MARK(3);
      if (!wait_flags(A.flags + (need0 ? q0 : 0), need0, epoch, deadline, L.err, lane) ||
          !wait_flags(A.flags + (need1 ? q1 : 0), need1, epoch, deadline, L.err, lane)) {
        ok = false;
        break;
      }
      PHASE_MARK(11);
    }
    PHASE_MARK(3);
    PHASE_COUNT(6, 1);
    bool pending = valid;
    for (int round = 0;; ++round) {
      const uint32_t pm = __ballot_sync(kFull, pending);
      if (!pm) break;
      // a match waits while its source overlaps the output of an earlier
      // pending match
      const bool haz = (pm & hmask) != 0;
      const bool ready = pending && !haz;
      // Units: with vec, the 16-byte-aligned blocks of each match's output
      // (a block's source bytes span at most two aligned source blocks, read
      // with two 16-byte loads and realigned in registers; a whole block is
      // stored with one 16-byte store, a partial one byte by byte); otherwise
      // 16-byte pieces copied byte by byte. Lane j copies units j, j+32, ...
      // of the round. With vec an aligned source block never leaves its
      // segment, and a segment is only read after its flag was acquired.
      const uint32_t nu = !ready ? 0 : vec ? (((uint32_t)(dst - seg_start) & 15u) + ml + 15) >> 4 : (ml + 15) >> 4;
      const uint32_t incl = warp_incl_scan(nu, lane);
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      PHASE_COUNT(7, 1);
      PHASE_COUNT(8, total);
      mt->start[lane] = incl - nu;
      mt->len[lane] = ml;
      if (lane == 31) mt->start[32] = incl;
      __syncwarp();
      for (uint32_t uu = lane; uu < total; uu += 32) {
        uint32_t m = 0;
#pragma unroll
        for (int s = 16; s; s >>= 1)
          if (mt->start[m + s] <= uu) m += s;
        if (vec) {
          const uint32_t doff = (uint32_t)(mt->dst[m] - seg_start);
          const uint32_t b16 = (doff & ~15u) + ((uu - mt->start[m]) << 4);
          const uint32_t a0 = max(doff, b16), a1 = min(doff + mt->len[m], b16 + 16);
          const uint32_t o = a0 - b16, n = a1 - a0;
          uint4 X = make_uint4(0, 0, 0, 0), Y = X;
          uint32_t cc;
          if (kMode == kViewLinear) {
            const uint8_t *pa = reinterpret_cast<const uint8_t *>(mt->src[m] + (a0 - doff));
            const uint32_t dl = (uint32_t)reinterpret_cast<uintptr_t>(pa) & 15u;
            const uint4 *pb = reinterpret_cast<const uint4 *>(pa - dl);
            if (dl >= o) {
              X = pb[0];
              if (dl + n > 16) Y = pb[1];
              cc = dl - o;
            } else {
              Y = pb[0];
              cc = 16 + dl - o;
            }
          } else {
            const uint64_t P = mt->src[m] + (a0 - doff);
            const uint8_t *pa = src_at<kMode>(V, P, log2_S);
            const uint32_t dl = (uint32_t)reinterpret_cast<uintptr_t>(pa) & 15u;
            if (dl >= o) {
              X = *reinterpret_cast<const uint4 *>(pa - dl);
              if (dl + n > 16) Y = *reinterpret_cast<const uint4 *>(src_at<kMode>(V, P + (16 - dl), log2_S));
              cc = dl - o;
            } else {
              Y = *reinterpret_cast<const uint4 *>(pa - dl);
              cc = 16 + dl - o;
            }
          }
          // cc < 16 in both cases (dl, o < 16): the mask tells the compiler,
          // which drops the selection level that a shift of 16 or more needs
          uint32_t r[4];
          realign16(X, Y, cc & 15u, r);
          uint8_t *to = out + b16;
          if (n == 16) {
            *reinterpret_cast<uint4 *>(to) = make_uint4(r[0], r[1], r[2], r[3]);
          } else {
            // bytes [o, o + n) of the block as naturally aligned pieces of
            // 1, 2, 4 and 8 bytes (a scattered store costs the memory
            // pipeline one pass per line it touches, whatever its width)
            auto wd = [&](uint32_t i) { return i & 2 ? (i & 1 ? r[3] : r[2]) : (i & 1 ? r[1] : r[0]); };
            if (o == 0 || o + n == 16) {
              // the first or last block of a match: one end of the bytes is
              // an end of the block, and the pieces are the set bits of n,
              // rising in size from o when the bytes end at the block's end,
              // falling from 0 when they start at its start (four store
              // instructions per warp)
              const bool rise = o != 0;
              if (n & 8) *reinterpret_cast<uint2 *>(to + (rise ? 8 : 0)) = rise ? make_uint2(r[2], r[3]) : make_uint2(r[0], r[1]);
              if (n & 4) {
                const uint32_t a = rise ? o + (n & 3) : (n & 8);
                *reinterpret_cast<uint32_t *>(to + a) = wd(a >> 2);
              }
              if (n & 2) {
                const uint32_t a = rise ? o + (n & 1) : (n & 12);
                *reinterpret_cast<uint16_t *>(to + a) = (uint16_t)(wd(a >> 2) >> (8 * (a & 2)));
              }
              if (n & 1) {
                const uint32_t a = rise ? o : (n & 14);
                to[a] = (uint8_t)(wd(a >> 2) >> (8 * (a & 3)));
              }
            } else {
              // both ends inside the block (a match shorter than 16 bytes):
              // rising in size up to the first boundary that the next piece
              // would cross, then falling (eight store instructions)
              uint32_t a = o;
              const uint32_t e = o + n;
              if ((a & 1) && a < e) { to[a] = (uint8_t)(wd(a >> 2) >> (8 * (a & 3))); a += 1; }
              if ((a & 2) && a + 2 <= e) { *reinterpret_cast<uint16_t *>(to + a) = (uint16_t)(wd(a >> 2) >> (8 * (a & 2))); a += 2; }
              if ((a & 4) && a + 4 <= e) { *reinterpret_cast<uint32_t *>(to + a) = wd(a >> 2); a += 4; }
              if ((a & 8) && a + 8 <= e) { *reinterpret_cast<uint2 *>(to + a) = make_uint2(r[2], r[3]); a += 8; }
              if (a + 8 <= e) { *reinterpret_cast<uint2 *>(to + a) = (a & 8) ? make_uint2(r[2], r[3]) : make_uint2(r[0], r[1]); a += 8; }
              if (a + 4 <= e) { *reinterpret_cast<uint32_t *>(to + a) = wd(a >> 2); a += 4; }
              if (a + 2 <= e) { *reinterpret_cast<uint16_t *>(to + a) = (uint16_t)(wd(a >> 2) >> (8 * (a & 2))); a += 2; }
              if (a < e) to[a] = (uint8_t)(wd(a >> 2) >> (8 * (a & 3)));
            }
          }
        } else {
          const uint32_t o = (uu - mt->start[m]) << 4;
          const uint32_t n = min(16u, mt->len[m] - o);
          const uint64_t pp = mt->src[m] + o;
          uint8_t *to = out + (mt->dst[m] - seg_start) + o;
          uint8_t v[16];
          if (kMode == kViewLinear) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if ((uint32_t)j < n) v[j] = reinterpret_cast<const uint8_t *>(pp)[j];
          } else
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if ((uint32_t)j < n) v[j] = *src_at<kMode>(V, pp + j, log2_S);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if ((uint32_t)j < n) to[j] = v[j];
        }
      }
      __syncwarp();
      pending = pending && !ready;
    }
    PHASE_MARK(4);
  }
  if (!ok && lane == 0 && ld_relaxed(L.err) == 0) latch(L.err, kErrCorrupt);

  PHASE_COUNT(9, 1);
  // ------------------------------------------------------------- publish
  // (no fence per lane: the warp barrier orders every lane's stores before
  // lane 0's release store, and release is cumulative)
  __syncwarp();
  if (lane == 0 && ok && !(A.blocked && A.blocked[seg])) st_release(A.flags + seg, (uint64_t)d.level << 32 | epoch);
}

// Decode one segment: its command streams are staged in the warp's shared
// area when they fit (scap bytes), else in its global slot gstage. With
// kSharedStage every segment of the launch fits (the host checked the
// archive's largest command stream), and the stage is read and written with
// shared-memory instructions.
template <bool kSmemLut, int kMode, bool kSharedStage>
__device__ __forceinline__ void decode_segment(const DecodeLaunch &L, const DevArchive &A, const OutView &V,
                                               uint32_t seg, uint32_t epoch, const uint32_t *lut, uint8_t *sstage,
                                               uint32_t scap, uint8_t *gstage, MatchTable *mt, uint16_t *ring,
                                               int lane, uint64_t *ph, uint64_t &ph_t) {
  const SegRec d = A.dir[seg];
  const uint32_t b3 = (4 + A.W) * d.n_cmd;
  uint8_t *stage = kSharedStage || b3 + 4 <= scap ? sstage : gstage;
  decode_segment_impl<kSmemLut, kMode, kSharedStage>(L, A, V, seg, epoch, lut, kSmemLut ? smem_addr(lut) : 0u,
                                                     Stage<kSharedStage>{stage, kSharedStage ? smem_addr(stage) : 0u},
                                                     mt, smem_addr(ring), lane, d, ph, ph_t);
}

// Dynamic shared memory of a decode CTA: the decode table (64 KiB), then a
// 1,280-byte word ring per warp (the 1 KiB ring and a copy of its first 256
// bytes), then a match table and a command stage per warp.
struct WarpSmem {
  uint32_t *lut;
  uint16_t *ring;
  MatchTable *mt;
  uint8_t *stage;
};
__device__ __forceinline__ WarpSmem warp_smem(uint8_t *smem, int wid) {
  constexpr uint32_t nw = kDecodeThreads / 32;
  WarpSmem w;
  w.lut = reinterpret_cast<uint32_t *>(smem);
  uint8_t *rings = smem + kLutBytes;
  w.ring = reinterpret_cast<uint16_t *>(rings + wid * 1280);
  w.mt = reinterpret_cast<MatchTable *>(rings + nw * 1280) + wid;
  w.stage = rings + nw * (1280 + sizeof(MatchTable)) + (size_t)wid * kSmemStage;
  return w;
}

#ifdef ACEAPEX_PHASE_CLOCKS
#define PHASE_DECL        \
  uint64_t ph[12] = {};   \
  uint64_t ph_t = clock64()
#define PHASE_FLUSH()                                                                               \
  do {                                                                                              \
    if (lane == 0)                                                                                  \
      for (int i_ = 0; i_ < 12; ++i_) atomicAdd(&g_phase_cycles[i_], (unsigned long long)ph[i_]); \
  } while (0)
#else
#define PHASE_DECL            \
  uint64_t *ph = nullptr;     \
  uint64_t ph_t = 0
#define PHASE_FLUSH() \
  do {                \
  } while (0)
#endif

// Persistent decode of one archive: its decode table is copied to shared
// memory once per CTA, and every warp takes the next work item.
// kMode: how the view maps positions (linear output, ring, or page table).
template <int kMode, bool kSharedStage>
__global__ void __launch_bounds__(kDecodeThreads, 1) decode_kernel(DecodeLaunch L) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const WarpSmem ws = warp_smem(smem, wid);
  {
    const uint4 *g = reinterpret_cast<const uint4 *>(L.arc0.lut);
    uint4 *s4 = reinterpret_cast<uint4 *>(ws.lut);
    for (uint32_t i = threadIdx.x; i < kLutBytes / 16; i += blockDim.x) s4[i] = g[i];
    __syncthreads();
  }
  const uint32_t gwarp = blockIdx.x * (blockDim.x >> 5) + wid;
  if (gwarp >= L.scratch_warps || (uint32_t)wid >= L.active_warps) return;
  uint8_t *gstage = L.scratch + (size_t)gwarp * kStageBytes;
  const uint32_t epoch = ld_relaxed(L.epoch);
  PHASE_DECL;
  for (;;) {
    bool failed;
    const uint32_t idx = take_item(L.counter, L.err, lane, failed);
    if (idx >= L.n_work) break;
    if (failed) continue;  // drain the list quickly after an error
    PHASE_MARK(5);
    decode_segment<true, kMode, kSharedStage>(L, L.arc0, L.view0, L.work[idx].seg, epoch, ws.lut, ws.stage,
                                              L.stage_cap, gstage, ws.mt, ws.ring, lane, ph, ph_t);
  }
  PHASE_FLUSH();
}

// Batch decode, one archive per CTA at a time (see launch_batch).
__global__ void __launch_bounds__(kDecodeThreads, 1) batch_kernel(DecodeLaunch L, uint32_t n_arcs) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_arc, s_next;
  __shared__ DevArchive s_A;
  __shared__ OutView s_V;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const WarpSmem ws = warp_smem(smem, wid);
  const uint32_t gwarp = blockIdx.x * (blockDim.x >> 5) + wid;
  uint8_t *gstage = L.scratch + (size_t)gwarp * kStageBytes;
  const uint32_t epoch = ld_relaxed(L.epoch);
  PHASE_DECL;
  for (;;) {
    if (threadIdx.x == 0) {
      s_arc = atomicAdd(L.counter, 1u);
      s_next = 0;
    }
    __syncthreads();
    const uint32_t a = s_arc;
    if (a >= n_arcs) break;
    if (threadIdx.x == 0) {
      s_A = L.arcs[a];
      s_V = L.views[a];
    }
    __syncthreads();
    const DevArchive &A = s_A;
    const uint4 *g = reinterpret_cast<const uint4 *>(A.lut);
    uint4 *s4 = reinterpret_cast<uint4 *>(ws.lut);
    for (uint32_t i = threadIdx.x; i < kLutBytes / 16; i += blockDim.x) s4[i] = g[i];
    __syncthreads();
    for (; (uint32_t)wid < L.active_warps;) {
      bool failed;
      const uint32_t idx = take_item(&s_next, L.err, lane, failed);
      if (idx >= A.n_seg) break;
      if (failed) continue;
      PHASE_MARK(5);
      decode_segment<true, kViewLinear, false>(L, A, s_V, A.order[idx].seg, epoch, ws.lut, ws.stage, L.stage_cap,
                                               gstage, ws.mt, ws.ring, lane, ph, ph_t);
    }
    __syncthreads();  // the table is replaced only after every warp left this archive
  }
  PHASE_FLUSH();
}

// One warp per window of `per` segments: the window's segments in level
// order, index order within a level (one pass over the window per level, a
// ballot placing each pass's members), into out[s0 .. s1) of the window.
__global__ void window_order_kernel(const SegRec *dir, uint64_t n_seg, uint64_t per, uint32_t max_level,
                                    WorkItem *out) {
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t s0 = w * per;
  if (s0 >= n_seg) return;  // (the whole warp)
  const uint64_t s1 = min(n_seg, s0 + per);
  const uint32_t lt = lanemask_lt();
  uint64_t pos = s0;
  for (uint32_t l = 0; l <= max_level; ++l)
    for (uint64_t b = s0; b < s1; b += 32) {
      const uint64_t s = b + lane;
      const bool take = s < s1 && dir[s].level == l;
      const uint32_t m = __ballot_sync(kFull, take);
      if (take) out[pos + __popc(m & lt)] = WorkItem{0u, (uint32_t)s};
      pos += __popc(m);
    }
}

__global__ void init_flags_kernel(uint64_t *flags, const SegRec *dir, uint64_t n) {
  const uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (s < n) flags[s] = (uint64_t)dir[s].level << 32;
}

__global__ void begin_kernel(uint32_t *global_epoch, uint32_t *epoch, uint32_t *counter) {
  *epoch = atomicAdd(global_epoch, 1u) + 1u;
  *counter = 0;
}

__global__ void clear_pages_kernel(uint32_t *page, const WorkItem *work, uint32_t n) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) page[work[i].seg] = 0xFFFFFFFFu;
}

__global__ void copy_view_kernel(OutView src, OutView dst, uint32_t log2_S, uint64_t lo, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint8_t *p = at(src, lo + i, log2_S);
    uint8_t *q = at(dst, lo + i, log2_S);
    if (p && q) *q = *p;
  }
}

__global__ void gather_kernel(OutView v, uint32_t log2_S, uint64_t lo, uint64_t n, uint8_t *dst) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint8_t *p = at(v, lo + i, log2_S);
    dst[i] = p ? *p : 0;
  }
}

// bases [0, n) of a FASTA region whose first base sits at lo with line phase
// `phase` (its position within a line of L bases): base i is at
// lo + i + (phase + i) / L, the newline after every L bases skipped
__global__ void gather_bases_kernel(OutView v, uint32_t log2_S, uint64_t lo, uint32_t phase, uint32_t L, uint64_t n,
                                    uint8_t *dst) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint8_t *p = at(v, lo + i + (phase + i) / L, log2_S);
    dst[i] = p ? *p : 0;
  }
}

constexpr uint64_t kGatherChunk = 65536;

__global__ void multi_gather_kernel(const GatherJob *jobs, uint32_t n_jobs, uint64_t n_chunks) {
  for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    // the job holding chunk c: largest j with jobs[j].chunk0 <= c
    uint32_t lo = 0, hi = n_jobs;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (jobs[mid].chunk0 <= c) lo = mid;
      else hi = mid;
    }
    const GatherJob &J = jobs[lo];
    const uint64_t a = (c - J.chunk0) * kGatherChunk, b = min(J.n, a + kGatherChunk);
    for (uint64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
      const uint8_t *p = at(J.v, J.lo + i, J.log2_S);
      J.dst[i] = p ? *p : 0;
    }
  }
}

__global__ void set_pages_kernel(uint32_t *page, const WorkItem *work, uint32_t n) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) page[work[i].seg] = i;
}

// -------------------------------------------------------- device closures
__global__ void closure_seed_kernel(ClosureDev C, uint32_t s_lo, uint32_t n, uint32_t gen) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    C.mark[s_lo + i] = gen;
    C.list[i] = s_lo + i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *C.cnt = n;
}

// One warp per member of the given level (grid-stride over the list); its
// lanes walk the member's dependency list. A dependency joins the closure
// when this warp is the first to tag it with gen; the warp reserves the list
// slots of its new members with one atomic. Members added here have lower
// levels, so the entries a warp sees beyond its first reading of cnt are
// skipped by the level test.
__global__ void closure_expand_kernel(ClosureDev C, uint32_t level, uint32_t gen) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  const uint32_t n = ld_relaxed(C.cnt);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const uint32_t s = C.list[i];
    if (C.dir[s].level != level) continue;
    const uint64_t b = C.dep_ptr[s], e = C.dep_ptr[s + 1];
    for (uint64_t k0 = b; k0 < e; k0 += 32) {
      const uint64_t k = k0 + lane;
      uint32_t d = 0;
      bool fresh = false;
      if (k < e) {
        d = C.deps[k];
        fresh = atomicExch(C.mark + d, gen) != gen;
      }
      const uint32_t m = __ballot_sync(kFull, fresh);
      if (!m) continue;
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(C.cnt, (uint32_t)__popc(m));
      base = __shfl_sync(kFull, base, 0);
      if (fresh) C.list[base + __popc(m & lanemask_lt())] = d;
    }
  }
}

// one CTA: counting sort of the members by level (levels < 65536)
constexpr int kClosureLevels = 256;
__global__ void __launch_bounds__(1024) closure_order_kernel(ClosureDev C, WorkItem *work, uint32_t *page,
                                                             uint32_t *n_out) {
  __shared__ uint32_t off[kClosureLevels];
  const uint32_t n = *C.cnt;
  for (int l = threadIdx.x; l < kClosureLevels; l += blockDim.x) off[l] = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
    atomicAdd(&off[min((uint32_t)C.dir[C.list[i]].level, (uint32_t)(kClosureLevels - 1))], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int l = 0; l < kClosureLevels; ++l) {
      const uint32_t c = off[l];
      off[l] = run;
      run += c;
    }
    *n_out = n;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t s = C.list[i];
    const uint32_t pos = atomicAdd(&off[min((uint32_t)C.dir[s].level, (uint32_t)(kClosureLevels - 1))], 1u);
    work[pos] = WorkItem{0u, s};
    page[s] = pos;
  }
}

// ------------------------------------------------------------------- CRC-32
// Standard CRC-32 (reflected polynomial 0xEDB88320, init and xorout ~0).
// A register r advanced over a message M from r0 is shift(r0, |M|) ^ raw(M),
// where raw is the register from r0 = 0 and shift(r, n) multiplies r by
// x^(8n) mod P (n zero bytes). So raw(A||B) = shift(raw(A), |B|) ^ raw(B),
// and crc(M) = raw(M) ^ shift(~0, |M|) ^ ~0. Everything is GF(2)-linear in
// the bytes, which the kernels below use to hash pieces in any order.
//
// Table words (g_crc_tabs, filled once per device from the host):
//   [0, 4096)                slice tables T_k[b] = raw(b followed by k zero
//                            bytes), k = 0..15 (T_0 is the usual byte table)
//   4096 + 1024 k + 256 i    byte tables of shift by 2^k bytes, k = 0..47:
//                            entry v = shift(v << 8i, 2^k)
constexpr int kCrcOps = 48;
constexpr int kCrcTabWords = 4096 + kCrcOps * 1024;
constexpr int kCrcSmemOps = 10;  // shifts by 2^0 .. 2^9 bytes kept in shared memory
constexpr int kCrcSmemWords = 4096 + kCrcSmemOps * 1024;
constexpr int kCrcThreads = 512;
__device__ uint32_t g_crc_tabs[kCrcTabWords];

__device__ __forceinline__ uint32_t crc_op(const uint32_t *t, uint32_t r) {
  return t[r & 0xFFu] ^ t[256 + ((r >> 8) & 0xFFu)] ^ t[512 + ((r >> 16) & 0xFFu)] ^ t[768 + (r >> 24)];
}

// shift(r, n) with the byte tables of 2^k bytes at ops + 1024 k
__device__ __forceinline__ uint32_t crc_shift(const uint32_t *ops, uint32_t r, uint64_t n) {
  for (int k = 0; n; ++k, n >>= 1)
    if (n & 1) r = crc_op(ops + 1024 * k, r);
  return r;
}

// raw CRC of 16 bytes held little-endian in w
__device__ __forceinline__ uint32_t crc_raw16(const uint32_t *T, uint4 w) {
  const uint32_t v[4] = {w.x, w.y, w.z, w.w};
  uint32_t r = 0;
#pragma unroll
  for (int m = 0; m < 16; ++m) r ^= T[256 * (15 - m) + ((v[m >> 2] >> (8 * (m & 3))) & 0xFFu)];
  return r;
}

// Raw CRC of each segment piece [max(lo, seg), min(hi, seg_end)) of the ring
// view. One warp per piece,
// persistent grid. The piece is read in rows of 512 bytes, lane j taking the
// 16 bytes at 512 i + 16 j of row i (coalesced), and folds its 16-byte pieces
// Horner-style with a shift of 512 bytes between rows; bytes after the last
// full row are folded per lane. Each lane then shifts its register past the
// bytes that follow its own last piece, and the warp XORs the 32 registers.
__global__ void __launch_bounds__(kCrcThreads, 3) seg_crc_kernel(OutView v, uint32_t log2_S, uint64_t lo, uint64_t hi,
                                                                  uint32_t *seg_crc) {
  __shared__ uint32_t tab[kCrcSmemWords];
  for (int i = threadIdx.x; i < kCrcSmemWords; i += blockDim.x) tab[i] = g_crc_tabs[i];
  __syncthreads();
  const uint32_t *ops = tab + 4096;
  const uint32_t *op512 = ops + 1024 * 9;
  const int lane = threadIdx.x & 31;
  const uint64_t S = uint64_t(1) << log2_S;
  const uint64_t first = lo >> log2_S, last = (hi - 1) >> log2_S;
  const uint64_t nseg = last - first + 1;
  for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < nseg;
       i += (uint64_t)gridDim.x * (blockDim.x >> 5)) {
    const uint64_t s = first + i;
    const uint64_t a = (s << log2_S) > lo ? (s << log2_S) : lo;
    const uint64_t b = ((s << log2_S) + S) < hi ? ((s << log2_S) + S) : hi;
    const uint32_t len = (uint32_t)(b - a);
    const uint8_t *p = v.base + ((a - v.origin) & v.mask);
    // a piece with a full row has S >= 512 and starts at a multiple of S in a
    // ring of a multiple of S bytes, so p is 16-byte aligned
    const uint32_t rows = len >> 9;
    uint32_t acc = 0;
    const uint4 *p16 = reinterpret_cast<const uint4 *>(p) + lane;
    uint32_t row = 0;
    for (; row + 4 <= rows; row += 4) {
      uint4 w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) w[u] = __ldcs(p16 + 32 * (row + u));
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = crc_op(op512, acc) ^ crc_raw16(tab, w[u]);
    }
    for (; row < rows; ++row) acc = crc_op(op512, acc) ^ crc_raw16(tab, __ldcs(p16 + 32 * row));
    uint32_t r = rows ? crc_shift(ops, acc, (len - 512u * rows) + 496u - 16u * lane) : 0u;
    // bytes after the full rows: lane j takes [16 j, 16 j + 16) of the rest
    const uint32_t t = len - 512u * rows, t0 = 16u * lane;
    if (t0 < t) {
      const uint32_t tj = min(16u, t - t0);
      uint32_t x = 0;
      for (uint32_t k = 0; k < tj; ++k) x = (x >> 8) ^ tab[(x ^ p[512u * rows + t0 + k]) & 0xFFu];
      r ^= crc_shift(ops, x, t - t0 - tj);
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) r ^= __shfl_xor_sync(kFull, r, d);
    if (lane == 0) seg_crc[i] = r;
  }
}

// One block per window: the window's CRC from its pieces' raw CRCs. Thread t
// folds a contiguous run of pieces, then a tree joins neighbouring runs.
__global__ void __launch_bounds__(1024) window_crc_kernel(const uint32_t *seg_crc, uint64_t lo, uint64_t hi,
                                                          uint64_t window, uint32_t log2_S, uint32_t *out) {
  __shared__ uint32_t opS[1024];
  __shared__ uint32_t part[1024];
  __shared__ uint64_t plen[1024];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) opS[i] = g_crc_tabs[4096 + 1024 * log2_S + i];
  __syncthreads();
  const uint32_t *gops = g_crc_tabs + 4096;
  const uint64_t k = blockIdx.x;
  const uint64_t wa = lo + k * window, wb = wa + window < hi ? wa + window : hi;
  const uint64_t first = lo >> log2_S;
  const uint64_t s0 = wa >> log2_S, s1 = (wb - 1) >> log2_S;  // pieces of this window
  const uint64_t np = s1 - s0 + 1;
  const uint64_t per = (np + blockDim.x - 1) / blockDim.x;
  const uint64_t i0 = threadIdx.x * per, i1 = i0 + per < np ? i0 + per : np;
  uint32_t acc = 0;
  uint64_t alen = 0;
  for (uint64_t i = i0; i < i1; ++i) {
    const uint64_t s = s0 + i;
    const uint64_t a = (s << log2_S) > wa ? (s << log2_S) : wa;
    const uint64_t e = ((s + 1) << log2_S) < wb ? ((s + 1) << log2_S) : wb;
    acc = (e - a == (uint64_t(1) << log2_S) ? crc_op(opS, acc) : crc_shift(gops, acc, e - a)) ^ seg_crc[s - first];
    alen += e - a;
  }
  part[threadIdx.x] = acc;
  plen[threadIdx.x] = alen;
  __syncthreads();
  for (uint32_t d = 1; d < blockDim.x; d <<= 1) {
    const uint32_t t = threadIdx.x;
    if (t % (2 * d) == 0 && t + d < blockDim.x && plen[t + d]) {
      part[t] = crc_shift(gops, part[t], plen[t + d]) ^ part[t + d];
      plen[t] += plen[t + d];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = part[0] ^ crc_shift(gops, 0xFFFFFFFFu, plen[0]) ^ 0xFFFFFFFFu;
}


// ------------------------------------------------- FASTQ stream separation
// A FASTQ split into its four line streams (headers, sequences, '+' lines,
// qualities) is put back together on the device: the newlines of each
// decoded stream are indexed (count per chunk, scan, positions), then one warp
// per record copies line r of every stream to its place. Record r starts at
// the sum over the streams of the start of their line r, since every earlier
// line of every stream precedes it in the FASTQ.
constexpr uint32_t kNlChunk = 65536;

// counts[c] = newlines in chunk c of buf[0, n); one CTA of 256 threads per chunk
__global__ void nl_count_kernel(const uint8_t *buf, uint64_t n, uint32_t *counts) {
  const uint64_t c0 = (uint64_t)blockIdx.x * kNlChunk, c1 = c0 + kNlChunk < n ? c0 + kNlChunk : n;
  uint32_t k = 0;
  for (uint64_t p = c0 + threadIdx.x; p < c1; p += blockDim.x) k += buf[p] == '\n';
  for (int d = 16; d; d >>= 1) k += __shfl_xor_sync(kFull, k, d);
  __shared__ uint32_t part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = k;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += part[w];
    counts[blockIdx.x] = t;
  }
}

// offs[c] = newlines before chunk c; offs[n_chunks] = total (one CTA)
__global__ void nl_scan_kernel(const uint32_t *counts, uint32_t n_chunks, uint64_t *offs) {
  __shared__ uint64_t part[1024];
  const uint32_t per = (n_chunks + blockDim.x - 1) / blockDim.x;
  const uint32_t i0 = threadIdx.x * per, i1 = i0 + per < n_chunks ? i0 + per : n_chunks;
  uint64_t t = 0;
  for (uint32_t i = i0; i < i1; ++i) t += counts[i];
  part[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t run = 0;
    for (uint32_t w = 0; w < blockDim.x; ++w) {
      const uint64_t v = part[w];
      part[w] = run;
      run += v;
    }
    offs[n_chunks] = run;
  }
  __syncthreads();
  uint64_t run = part[threadIdx.x];
  for (uint32_t i = i0; i < i1; ++i) {
    offs[i] = run;
    run += counts[i];
  }
}

// nl[j] = position of the j-th newline of buf (j < cap; err set beyond)
__global__ void nl_positions_kernel(const uint8_t *buf, uint64_t n, const uint64_t *offs, uint32_t *nl, uint64_t cap,
                                    uint32_t *err) {
  const uint64_t c0 = (uint64_t)blockIdx.x * kNlChunk, c1 = c0 + kNlChunk < n ? c0 + kNlChunk : n;
  // each warp takes 32-byte windows in order; a ballot places the window's
  // newlines after those of the earlier windows of the chunk
  __shared__ uint32_t wcount[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t span = (c1 - c0 + 7) / 8, w0 = c0 + wid * span, w1 = w0 + span < c1 ? w0 + span : c1;
  uint32_t mine = 0;
  for (uint64_t p = w0 + lane; p < w1 + lane; p += 32) mine += (p < w1 && buf[p] == '\n');
  for (int d = 16; d; d >>= 1) mine += __shfl_xor_sync(kFull, mine, d);
  if (lane == 0) wcount[wid] = mine;
  __syncthreads();
  uint64_t base = offs[blockIdx.x];
  for (int w = 0; w < wid; ++w) base += wcount[w];
  for (uint64_t p = w0; p < w1; p += 32) {
    const bool is_nl = p + lane < w1 && buf[p + lane] == '\n';
    const uint32_t m = __ballot_sync(kFull, is_nl);
    if (is_nl) {
      const uint64_t j = base + __popc(m & ((1u << lane) - 1u));
      if (j < cap) nl[j] = (uint32_t)(p + lane);
      else latch(err, kErrCorrupt);
    }
    base += __popc(m);
  }
}

struct LineStreams {
  const uint8_t *base[4];
  const uint32_t *nl[4];
  const uint64_t *count[4];  // device: newlines of each stream
  uint64_t len[4];
};

// one warp per record (grid-stride): line r of stream k is [s, e) with
// s = nl_k[r - 1] + 1 (0 for r = 0) and e = nl_k[r] + 1, or the stream end
// for a last line without newline
__global__ void interleave_kernel(LineStreams S, uint8_t *out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  uint64_t cnt[4], R = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) cnt[k] = *S.count[k];
  R = cnt[0] + (S.len[0] && (cnt[0] == 0 || S.nl[0][cnt[0] - 1] != S.len[0] - 1) ? 1 : 0);
  for (uint64_t r = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += warps) {
    uint64_t s[4], e[4], o = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      s[k] = r == 0 ? 0 : (r - 1 < cnt[k] ? (uint64_t)S.nl[k][r - 1] + 1 : S.len[k]);
      e[k] = r < cnt[k] ? (uint64_t)S.nl[k][r] + 1 : S.len[k];
      if (e[k] < s[k]) e[k] = s[k];
      o += s[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint8_t *src = S.base[k] + s[k];
      const uint64_t len = e[k] - s[k];
      for (uint64_t i = lane; i < len; i += 32) out[o + i] = src[i];
      o += len;
    }
  }
}
}  // namespace

// ------------------------------------------------------------------ launchers

constexpr size_t kWarpSmem = sizeof(MatchTable) + 1280 + kSmemStage;
static_assert(sizeof(MatchTable) % 16 == 0, "keeps the stages aligned");
constexpr size_t kSmemLutBytes = kLutBytes + (size_t)(kDecodeThreads / 32) * kWarpSmem;

int decode_grid(int device, int block) {
  (void)block;
  int sms = 0, a = 0, b = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const auto smem = [](const void *k) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLutBytes);
  };
  smem((const void *)decode_kernel<kViewLinear, false>);
  smem((const void *)decode_kernel<kViewRing, false>);
  smem((const void *)decode_kernel<kViewPaged, false>);
  smem((const void *)decode_kernel<kViewLinear, true>);
  smem((const void *)decode_kernel<kViewRing, true>);
  smem((const void *)decode_kernel<kViewPaged, true>);
  cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLutBytes);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, decode_kernel<kViewLinear, false>, kDecodeThreads, kSmemLutBytes);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_kernel, kDecodeThreads, kSmemLutBytes);
  int per_sm = a < b ? a : b;
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

cudaError_t launch_decode(const DecodeLaunch &L, int grid, int block, cudaStream_t st) {
  (void)block;
  if (L.n_work == 0) return cudaSuccess;
  // every segment's command streams fit the shared stage: the stage-in-shared kernel
  const bool sh = L.max_stage <= L.stage_cap;
  if (L.view0.page) {
    if (sh) decode_kernel<kViewPaged, true><<<grid, kDecodeThreads, kSmemLutBytes, st>>>(L);
    else decode_kernel<kViewPaged, false><<<grid, kDecodeThreads, kSmemLutBytes, st>>>(L);
  } else if (L.view0.mask != ~uint64_t(0)) {
    if (sh) decode_kernel<kViewRing, true><<<grid, kDecodeThreads, kSmemLutBytes, st>>>(L);
    else decode_kernel<kViewRing, false><<<grid, kDecodeThreads, kSmemLutBytes, st>>>(L);
  } else {
    if (sh) decode_kernel<kViewLinear, true><<<grid, kDecodeThreads, kSmemLutBytes, st>>>(L);
    else decode_kernel<kViewLinear, false><<<grid, kDecodeThreads, kSmemLutBytes, st>>>(L);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch(const DecodeLaunch &L, uint32_t n_arcs, int grid, cudaStream_t st) {
  if (n_arcs == 0) return cudaSuccess;
  cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLutBytes);
  batch_kernel<<<grid, kDecodeThreads, kSmemLutBytes, st>>>(L, n_arcs);
  return cudaGetLastError();
}

cudaError_t launch_window_order(const SegRec *dir, uint64_t n_seg, uint64_t per, uint32_t max_level, WorkItem *out,
                                cudaStream_t st) {
  if (!n_seg || !per) return cudaSuccess;
  const uint64_t warps = (n_seg + per - 1) / per;
  window_order_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(dir, n_seg, per, max_level, out);
  return cudaGetLastError();
}

cudaError_t launch_init_flags(uint64_t *flags, const SegRec *dir, uint64_t n, cudaStream_t st) {
  if (!n) return cudaSuccess;
  init_flags_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(flags, dir, n);
  return cudaGetLastError();
}

cudaError_t launch_begin(uint32_t *global_epoch, uint32_t *epoch, uint32_t *counter, cudaStream_t st) {
  begin_kernel<<<1, 1, 0, st>>>(global_epoch, epoch, counter);
  return cudaGetLastError();
}

cudaError_t launch_clear_pages(uint32_t *page, const WorkItem *work, uint32_t n, cudaStream_t st) {
  if (!n) return cudaSuccess;
  clear_pages_kernel<<<(n + 255) / 256, 256, 0, st>>>(page, work, n);
  return cudaGetLastError();
}

cudaError_t launch_copy_view(OutView src, OutView dst, uint32_t log2_S, uint64_t lo, uint64_t hi, cudaStream_t st) {
  if (hi <= lo) return cudaSuccess;
  uint64_t n = hi - lo;
  int grid = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  copy_view_kernel<<<grid, 256, 0, st>>>(src, dst, log2_S, lo, n);
  return cudaGetLastError();
}

cudaError_t launch_gather(OutView v, uint32_t log2_S, uint64_t lo, uint64_t hi, uint8_t *dst, cudaStream_t st) {
  if (hi <= lo) return cudaSuccess;
  uint64_t n = hi - lo;
  int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  gather_kernel<<<grid, 256, 0, st>>>(v, log2_S, lo, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_gather_bases(OutView v, uint32_t log2_S, uint64_t lo, uint32_t phase, uint32_t line_width,
                                uint64_t n, uint8_t *dst, cudaStream_t st) {
  if (!n) return cudaSuccess;
  int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  gather_bases_kernel<<<grid, 256, 0, st>>>(v, log2_S, lo, phase, line_width, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_fastq_interleave(const uint8_t *const base[4], const uint64_t len[4], uint32_t *counts,
                                    uint64_t *offs, uint32_t *const nl[4], const uint64_t cap[4], uint32_t *err,
                                    uint8_t *out, cudaStream_t st) {
  LineStreams S{};
  uint64_t off_at = 0;
  for (int k = 0; k < 4; ++k) {
    const uint32_t chunks = (uint32_t)((len[k] + kNlChunk - 1) / kNlChunk);
    uint64_t *o = offs + off_at;
    if (chunks) {
      nl_count_kernel<<<chunks, 256, 0, st>>>(base[k], len[k], counts);
      nl_scan_kernel<<<1, 1024, 0, st>>>(counts, chunks, o);
      nl_positions_kernel<<<chunks, 256, 0, st>>>(base[k], len[k], o, nl[k], cap[k], err);
    } else if (cudaMemsetAsync(o, 0, sizeof(uint64_t), st) != cudaSuccess) {
      return cudaGetLastError();
    }
    S.base[k] = base[k];
    S.nl[k] = nl[k];
    S.count[k] = o + chunks;
    S.len[k] = len[k];
    off_at += chunks + 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  interleave_kernel<<<8 * sms, 256, 0, st>>>(S, out);
  return cudaGetLastError();
}

cudaError_t launch_multi_gather(const GatherJob *jobs, uint32_t n_jobs, uint64_t n_chunks, cudaStream_t st) {
  if (!n_jobs || !n_chunks) return cudaSuccess;
  const int grid = (int)(n_chunks < 4096 ? n_chunks : 4096);
  multi_gather_kernel<<<grid, 256, 0, st>>>(jobs, n_jobs, n_chunks);
  return cudaGetLastError();
}

cudaError_t launch_set_pages(uint32_t *page, const WorkItem *work, uint32_t n, cudaStream_t st) {
  if (!n) return cudaSuccess;
  set_pages_kernel<<<(n + 255) / 256, 256, 0, st>>>(page, work, n);
  return cudaGetLastError();
}

cudaError_t launch_closure_seed(ClosureDev C, uint32_t s_lo, uint32_t n, uint32_t gen, cudaStream_t st) {
  closure_seed_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(C, s_lo, n, gen);
  return cudaGetLastError();
}

cudaError_t launch_closure_expand(ClosureDev C, uint32_t level, uint32_t gen, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  closure_expand_kernel<<<2 * sms, 512, 0, st>>>(C, level, gen);
  return cudaGetLastError();
}

cudaError_t launch_closure_order(ClosureDev C, WorkItem *work, uint32_t *page, uint32_t *n_out, cudaStream_t st) {
  closure_order_kernel<<<1, 1024, 0, st>>>(C, work, page, n_out);
  return cudaGetLastError();
}

static bool g_crc_ready[64] = {};

// Fills g_crc_tabs on the current device (once per device).
static cudaError_t ensure_crc_constants() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && g_crc_ready[dev]) return cudaSuccess;
  static std::vector<uint32_t> tabs;
  static std::once_flag once;
  std::call_once(once, [] {
    tabs.assign(kCrcTabWords, 0);
    auto byte_step = [](uint32_t c) {
      for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
      return c;
    };
    uint32_t *T = tabs.data();
    for (uint32_t b = 0; b < 256; ++b) T[b] = byte_step(b);
    for (int k = 1; k < 16; ++k)
      for (uint32_t b = 0; b < 256; ++b) {
        const uint32_t c = T[256 * (k - 1) + b];
        T[256 * k + b] = (c >> 8) ^ T[c & 0xFFu];
      }
    // col[k][i]: register 1 << i shifted by 2^k zero bytes (repeated squaring)
    std::vector<uint32_t> col(32 * kCrcOps);
    for (int i = 0; i < 32; ++i) col[i] = byte_step(1u << i);
    for (int k = 1; k < kCrcOps; ++k)
      for (int i = 0; i < 32; ++i) {
        uint32_t v = col[32 * (k - 1) + i], r = 0;
        for (int j = 0; j < 32; ++j)
          if (v >> j & 1u) r ^= col[32 * (k - 1) + j];
        col[32 * k + i] = r;
      }
    for (int k = 0; k < kCrcOps; ++k)
      for (int i = 0; i < 4; ++i)
        for (uint32_t v = 0; v < 256; ++v) {
          uint32_t r = 0;
          for (int j = 0; j < 8; ++j)
            if (v >> j & 1u) r ^= col[32 * k + 8 * i + j];
          T[4096 + 1024 * k + 256 * i + v] = r;
        }
  });
  cudaError_t e = cudaMemcpyToSymbol(g_crc_tabs, tabs.data(), tabs.size() * sizeof(uint32_t));
  if (e == cudaSuccess && dev >= 0 && dev < 64) g_crc_ready[dev] = true;
  return e;
}

cudaError_t launch_window_crc(OutView v, uint64_t lo, uint64_t hi, uint64_t window, uint32_t *crc, uint32_t *seg_crc,
                              uint32_t log2_S, cudaStream_t st) {
  if (hi <= lo) return cudaSuccess;
  cudaError_t e = ensure_crc_constants();
  if (e != cudaSuccess) return e;
  const uint64_t nseg = ((hi - 1) >> log2_S) - (lo >> log2_S) + 1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = (nseg + kCrcThreads / 32 - 1) / (kCrcThreads / 32);
  const int grid = (int)(want < (uint64_t)(3 * sms) ? want : (uint64_t)(3 * sms));
  seg_crc_kernel<<<grid, kCrcThreads, 0, st>>>(v, log2_S, lo, hi, seg_crc);
  const uint64_t nwin = (hi - lo + window - 1) / window;
  window_crc_kernel<<<(unsigned)nwin, 1024, 0, st>>>(seg_crc, lo, hi, window, log2_S, crc);
  return cudaGetLastError();
}

// ===================================================================
// Allocation-free whole-file decode (aceapex_decode_all_noalloc).
//
// Some callers cannot allocate device memory at decode time: a host program
// that hands the whole device to its own memory pool at start-up and forbids
// libraries from calling cudaMalloc afterwards, or a real-time pipeline that
// only permits allocation during initialisation. For them this entry point
// decodes an archive that the caller already holds in device memory into the
// caller's output buffer and allocates nothing: the scratch it needs (decode
// tables, ready flags, control words and per-warp staging) lives in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
//
// Limits: at most kNoAllocMaxSegments segments (1 GiB of output at 16 KiB
// segments); larger archives are rejected with ACEAPEX_ERANGE. The decode
// runs on kNoAllocWarps warps only, so it is slower than
// aceapex_decode_all. All calls share the array and it keeps the last
// call's contents: each call clears the words that must start at zero and
// takes a fresh epoch, but calls that overlap on the GPU (on different
// streams, or from different threads) race and must not be issued.
namespace {

constexpr uint32_t kNoAllocMaxSegments = 65536;
constexpr uint32_t kNoAllocWarps = 256;
constexpr size_t kNoAllocCtlBytes = 256;                       // counter, epoch, err
constexpr size_t kNoAllocLutBytes = 4 * kScale * sizeof(uint32_t);
constexpr size_t kNoAllocFlagBytes = kNoAllocMaxSegments * sizeof(uint64_t);
constexpr size_t kNoAllocStageBytes = (size_t)kNoAllocWarps * kStageBytes;
constexpr size_t kNoAllocBytes = kNoAllocCtlBytes + kNoAllocLutBytes + kNoAllocFlagBytes + kNoAllocStageBytes;

// about 4.3 MiB per device
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

// control words at the start of the array
constexpr size_t kCtlCounter = 0, kCtlEpoch = 4, kCtlErr = 8, kCtlEmpty = 12;

// builds the decode table from the archive's tables, checks their sums,
// clears the counter and the error word, and takes the next epoch
__global__ void noalloc_setup_kernel(const uint8_t *tables) {
  uint8_t *base = g_noalloc_scratch;
  uint32_t *ctl = reinterpret_cast<uint32_t *>(base);
  uint32_t *lut = reinterpret_cast<uint32_t *>(base + kNoAllocCtlBytes);
  __shared__ uint32_t cum[4][257];
  __shared__ uint32_t bad;
  __shared__ uint32_t empty;
  if (threadIdx.x == 0) {
    bad = 0;
    empty = 0;
    for (int c = 0; c < 4; ++c) {
      uint32_t s = 0;
      cum[c][0] = 0;
      for (int x = 0; x < 256; ++x) {
        s += (uint32_t)tables[512 * c + 2 * x] | ((uint32_t)tables[512 * c + 2 * x + 1] << 8);
        cum[c][x + 1] = s;
      }
      if (s != 0 && s != kScale) bad = 1;
      if (s == 0) empty |= 1u << c;
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
    const uint32_t c = i >> 8, x = i & 255, f = cum[c][x + 1] - cum[c][x];
    for (uint32_t k = 0; k < f && !bad; ++k) lut[c * kScale + cum[c][x] + k] = x | (k << 8) | ((f - 1) << 20);
  }
  if (threadIdx.x == 0) {
    ctl[kCtlCounter / 4] = 0;
    ctl[kCtlErr / 4] = bad ? kErrCorrupt : 0u;
    ctl[kCtlEmpty / 4] = empty;
    ctl[kCtlEpoch / 4] = ctl[kCtlEpoch / 4] + 1u;
  }
}

// segments in index order (every source segment precedes its reader, so a
// warp only waits for segments that running warps took earlier)
__global__ void __launch_bounds__(256) noalloc_decode_kernel(DecodeLaunch L, uint64_t payload_bytes,
                                                             uint32_t max_level) {
  const int lane = threadIdx.x & 31;
  const uint32_t gwarp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gwarp >= kNoAllocWarps) return;
  uint8_t *stage = g_noalloc_scratch + kNoAllocCtlBytes + kNoAllocLutBytes + kNoAllocFlagBytes +
                   (size_t)gwarp * kStageBytes;
  __shared__ MatchTable mts[8];
  __shared__ __align__(16) uint16_t rings_raw[8][640];
  uint16_t *ring = rings_raw[threadIdx.x >> 5];
  const uint32_t epoch = ld_relaxed(L.epoch);
  PHASE_DECL;
  const uint32_t empty = reinterpret_cast<const uint32_t *>(g_noalloc_scratch)[kCtlEmpty / 4];
  const DevArchive &A = L.arc0;
  for (;;) {
    bool failed;
    const uint32_t seg = take_item(L.counter, L.err, lane, failed);
    if (seg >= A.n_seg) break;
    if (failed) continue;
    // the directory was not validated on the host: check what the shared
    // segment decoder relies on before calling it
    const SegRec d = A.dir[seg];
    // (the payload test is written so that no sum can wrap)
    const uint64_t n_sym = (uint64_t)d.n_cmd * (4 + A.W) + d.n_lit;
    const bool sane = n_sym <= kMaxSym && (d.payload_off & 15) == 0 && d.payload_off <= payload_bytes &&
                      payload_bytes - d.payload_off >= 128 &&
                      d.n_words <= (payload_bytes - d.payload_off - 128) / 2 && d.level <= max_level &&
                      !(d.n_cmd && (empty & 7u)) && !(d.n_lit && (empty & 8u));
    if (!sane) {
      if (lane == 0) latch(L.err, kErrCorrupt);
      continue;
    }
    decode_segment<false, kViewLinear, false>(L, A, L.view0, seg, epoch, A.lut, stage, 0, stage,
                                              &mts[threadIdx.x >> 5], ring, lane, ph, ph_t);
  }
}

__global__ void noalloc_status_kernel(uint32_t *status) {
  *status = reinterpret_cast<const uint32_t *>(g_noalloc_scratch)[kCtlErr / 4];
}

std::mutex g_noalloc_mu;
uint8_t *g_noalloc_addr[64] = {};

}  // namespace

extern "C" int aceapex_decode_all_noalloc(const void *d_archive, uint64_t nbytes, void *d_out, uint64_t out_cap,
                                          uint32_t *d_status, void *stream) {
  if (!d_archive || !d_status || nbytes < kHeaderBytes + kTablesBytes ||
      (reinterpret_cast<uintptr_t>(d_archive) & 15))
    return 1;  // ACEAPEX_EINVAL
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 4;  // ACEAPEX_ECUDA
  // set-up, once per device with that device current: the device address of
  // the scratch array (its name in host code is only a stand-in)
  uint8_t *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return 4;
      g_noalloc_addr[dev] = static_cast<uint8_t *>(p);
    }
    base = g_noalloc_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the header, read into host stack memory
  uint8_t h[kHeaderBytes];
  if (cudaMemcpyAsync(h, d_archive, kHeaderBytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return 4;
  auto u64 = [&](int o) { uint64_t v; std::memcpy(&v, h + o, 8); return v; };
  auto u32 = [&](int o) { uint32_t v; std::memcpy(&v, h + o, 4); return v; };
  const uint64_t n = u64(16), n_seg = u64(40), n_deps = u64(48), n_reads = u64(56);
  const uint32_t log2_B = h[24], log2_S = h[25], W = h[26], min_match = h[27], flags = h[31];
  if (std::memcmp(h, "ACEAPEX1", 8) != 0 || u32(8) != 1 || u32(12) != kHeaderBytes || h[28] != kScaleBits ||
      h[29] != kLanes || (flags & ~1u) || (!(flags & 1u) && n_reads) || log2_B < 2 || log2_B > 30 ||
      log2_S != (log2_B < kMaxLog2S ? log2_B : kMaxLog2S) || W != offset_width(n) || min_match < 1)
    return 2;  // ACEAPEX_ECORRUPT
  // counts bounded by the archive length first, so that the section offsets
  // below cannot wrap
  if (n_seg > nbytes / 24 || n_deps > nbytes / 4 || n_reads > nbytes / 8) return 2;
  const uint64_t S = uint64_t(1) << log2_S;
  const uint64_t off_dir = u64(72), off_dep_ptr = u64(80), off_deps = u64(88), off_reads = u64(96);
  const uint64_t off_payload = u64(104), payload_bytes = u64(112), total = u64(120);
  if (off_payload > nbytes || payload_bytes > nbytes || (payload_bytes & 15)) return 2;
  if (n_seg != (n + S - 1) / S || u64(64) != kHeaderBytes || off_dir != kHeaderBytes + kTablesBytes ||
      off_dep_ptr != round16(off_dir + 24 * n_seg) || off_deps != round16(off_dep_ptr + 8 * (n_seg + 1)) ||
      off_reads != round16(off_deps + 4 * n_deps) || off_payload != round16(off_reads + 8 * n_reads) ||
      total != off_payload + payload_bytes || total != nbytes)
    return 2;
  if (n_seg > kNoAllocMaxSegments) return 6;  // ACEAPEX_ERANGE: beyond the fixed scratch
  if (out_cap < n || (n && !d_out)) return 6;
  if (n == 0) return cudaMemsetAsync(d_status, 0, 4, st) == cudaSuccess ? 0 : 4;

  const uint8_t *arc = static_cast<const uint8_t *>(d_archive);
  DecodeLaunch L{};
  DevArchive &A = L.arc0;
  A.payload = arc + off_payload;
  A.dir = reinterpret_cast<const SegRec *>(arc + off_dir);
  A.lut = reinterpret_cast<const uint32_t *>(base + kNoAllocCtlBytes);
  A.flags = reinterpret_cast<uint64_t *>(base + kNoAllocCtlBytes + kNoAllocLutBytes);
  A.blocked = nullptr;
  A.n = n;
  A.D = u64(32);
  A.log2_S = log2_S;
  A.W = W;
  A.min_match = min_match;
  A.n_seg = (uint32_t)n_seg;
  L.view0.base = static_cast<uint8_t *>(d_out);
  L.view0.origin = 0;
  L.view0.mask = ~uint64_t(0);
  L.counter = reinterpret_cast<uint32_t *>(base + kCtlCounter);
  L.epoch = reinterpret_cast<const uint32_t *>(base + kCtlEpoch);
  L.err = reinterpret_cast<uint32_t *>(base + kCtlErr);
  L.scratch = nullptr;
  L.scratch_warps = kNoAllocWarps;
  L.wait_ns = 2000000000ull;
  noalloc_setup_kernel<<<1, 256, 0, st>>>(arc + kHeaderBytes);
  // (a corrupt record's level is caught by that segment's own checks, and a
  // reader that waits for it gives up once that segment latches the error)
  launch_init_flags(A.flags, A.dir, n_seg, st);
  noalloc_decode_kernel<<<kNoAllocWarps / 8, 256, 0, st>>>(L, payload_bytes, h[30]);
  noalloc_status_kernel<<<1, 1, 0, st>>>(d_status);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

}  // namespace aceapex

#ifdef ACEAPEX_PHASE_CLOCKS
// Instrumented build only: copies the warp cycles that the decode kernels
// spent in each phase (command-class rANS, command parse, literal rANS and
// placement, source checks, match copies, the rest of the work loop), the
// event counts (match chunks, copy rounds, copy units, segments, chunks that
// waited) and the cycles spent waiting for source segments, in that order,
// since the last reset into out[0 .. n) (n <= 12), and zeroes them when
// reset != 0.
// Synchronises the current device. Returns 0, or 4 on a CUDA error.
extern "C" int aceapex_phase_cycles(uint64_t *out, int n, int reset) {
  unsigned long long h[16] = {};
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpyFromSymbol(h, aceapex::g_phase_cycles, sizeof(h)) != cudaSuccess)
    return 4;
  for (int i = 0; i < n && i < 12; ++i) out[i] = h[i];
  if (reset) {
    const unsigned long long z[16] = {};
    if (cudaMemcpyToSymbol(aceapex::g_phase_cycles, z, sizeof(z)) != cudaSuccess) return 4;
  }
  return 0;
}
#endif
