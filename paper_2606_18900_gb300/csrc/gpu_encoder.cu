// GPU encoder of the library: the match search of paper §2 (global search
// over the whole decompressed history, absolute offsets, fixed-size blocks)
// run on the device. The paper's encoder is CPU-only and names its speed as
// the pipeline's bottleneck (§8, Limitations). This one applies the rules of
// the host encoder (encoder_rules.h) and writes the same archive, byte for
// byte, in four phases:
//
//  1. chains: hash every position of the chain window and sort the (hash,
//     position) pairs stably (LSD radix sort); the positions with the same
//     hash then sit in ascending order, so the slots before a position's
//     slot are its hash chain, latest first, equal to the chains of a
//     sequential insertion pass over a hash table.
//  2. match and parse: one thread per sorted slot finds the longest legal
//     match of its position among the preceding slots (coalesced reads, no
//     dependent walk; a candidate whose 8 bytes ending at the current best
//     length differ cannot win and is not compared further) into a table
//     indexed by position, with a bitmask of the usable ones; then one
//     thread per segment (the ruler level schedule makes segments
//     independent) parses greedily with one-step lazy matching, jumping
//     between mask bits, applies the symbol budget, flattens intra-segment
//     chains and lists the segment's source segments.
//  3. symbols: one warp per segment writes the segment's symbol message
//     (the format's symbol message) and counts symbols per class; levels follow tier by tier
//     of the schedule (a segment only reads lower tiers); dependency lists
//     are packed into CSR form.
//  4. entropy: the 1024 class counts are normalised on the host (4 x 256
//     values); rANS runs twice, one warp per segment, first counting the
//     words of each segment and then writing them at their final offsets;
//     the directory and the other sections are written in place.
//
// Device memory is kept by the encoder object between calls and grows on
// demand. Every kernel is a bounded loop: no kernel waits for another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "aceapex.h"
#include "encoder_rules.h"
#include "format.h"

namespace aceapex {
namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kInPad = 64;          // readable bytes past the input's end
constexpr uint32_t kBatchSegs = 65536;   // segments parsed per launch
constexpr uint32_t kErrCmdCap = 1, kErrLevel = 2, kErrSchedule = 4, kErrSymbols = 8;

// ------------------------------------------------------------ shared helpers

ACE_HD uint32_t ctz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return (uint32_t)(__ffsll((long long)x) - 1);
#else
  return (uint32_t)__builtin_ctzll(x);
#endif
}

// 8 little-endian bytes at any address (the buffer is padded past its end)
ACE_HD uint64_t load_le64(const uint8_t *p) {
#if defined(__CUDA_ARCH__)
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint64_t *q = reinterpret_cast<const uint64_t *>(a & ~uintptr_t(7));
  const uint32_t sh = (uint32_t)(a & 7) * 8;
  const uint64_t lo = q[0];
  return sh ? (lo >> sh) | (q[1] << (64 - sh)) : lo;
#else
  uint64_t v;
  std::memcpy(&v, p, 8);
  return v;
#endif
}

ACE_HD uint64_t min64(uint64_t a, uint64_t b) { return a < b ? a : b; }

ACE_HD uint64_t common_len(const uint8_t *a, const uint8_t *b, uint64_t lim) {
  uint64_t L = 0;
  while (L + 8 <= lim) {
    const uint64_t x = load_le64(a + L), y = load_le64(b + L);
    if (x != y) return L + (ctz64(x ^ y) >> 3);
    L += 8;
  }
  while (L < lim && a[L] == b[L]) ++L;
  return L;
}

// What the match search and the parse read.
struct ParseCtx {
  const uint8_t *in;
  uint64_t n;
  uint64_t base;  // first position of the chain window (sorted values are relative to it)
  uint64_t S, D;
  uint32_t log2_S, W, min_match, cap, sample_mask;
};

// Longest legal match at position p = base + V[j], sorted slot j. The
// positions with the same hash sit in the slots just before j, latest first
// (the sort is stable), so they are p's hash chain: at most kChainDepth of
// them are tried. A candidate is clipped at the distance bound, at the
// segment end, at p itself (src + len <= p) and at the first source segment
// that the level schedule forbids.
ACE_HD uint64_t match_at_slot(const ParseCtx &g, const uint32_t *K, const uint32_t *V, uint64_t j, uint64_t p,
                              uint64_t *src_out) {
  const uint64_t s = p >> g.log2_S, seg_end = min64(g.n, (s + 1) << g.log2_S);
  const uint32_t Ts = ruler_target(s, g.cap), key = K[j];
  uint64_t best = 0, best_src = 0;
  for (uint32_t k = 0; k < kChainDepth && k < j; ++k) {
    const uint64_t jj = j - 1 - k;
    if (K[jj] != key) break;
    const uint64_t c = g.base + V[jj];
    if (g.D && p - c > g.D) break;
    uint64_t lim = min64(p - c, seg_end - p);
    const uint64_t q0 = c >> g.log2_S, q1 = (c + lim - 1) >> g.log2_S;
    for (uint64_t q = q0; q <= q1; ++q) {
      if (q != s && ruler_target(q, g.cap) >= Ts) {
        const uint64_t start = q << g.log2_S;
        lim = min64(lim, start > c ? start - c : 0);
        break;
      }
    }
    if (lim <= best) continue;
    // a longer match than best agrees on bytes [0, best]: test the 8 bytes
    // ending at best first (the outcome is the same, most losers cost one load)
    if (best >= 7 && load_le64(g.in + c + best - 7) != load_le64(g.in + p + best - 7)) continue;
    const uint64_t L = common_len(g.in + c, g.in + p, lim);
    if (L > best) {
      best = L;
      best_src = c;
      if ((L == lim && lim == seg_end - p) || L >= kGoodEnough) break;
    }
  }
  *src_out = best_src;
  return best;
}

// Match table of a window's positions (enc_match_kernel): t[p - p0] =
// len << 32 | (p - src), 0 where the parse finds nothing; mask bit p - p0 is
// set where the parse can use the match (length >= min_match, or any length
// in sampled mode, where backward extension may lengthen it).
struct TableFinder {
  const uint64_t *t;
  const uint64_t *mask;
  uint64_t p0;
  ACE_HD uint64_t operator()(uint64_t p, uint64_t *src) const {
    const uint64_t v = t[p - p0];
    const uint64_t len = v >> 32;
    *src = len ? p - (uint32_t)v : 0;
    return len;
  }
  // first position in [p, end) whose mask bit is set, else end
  ACE_HD uint64_t next(uint64_t p, uint64_t end) const {
    const uint64_t r = p - p0;
    uint64_t w = r >> 6, bits = mask[w] & (~0ull << (r & 63));
    while (!bits) {
      ++w;
      if (p0 + (w << 6) >= end) return end;
      bits = mask[w];
    }
    const uint64_t q = p0 + (w << 6) + ctz64(bits);
    return q < end ? q : end;
  }
};

// Greedy parse of segment s with one-step lazy matching (content-defined
// anchors with backward extension in sampled mode); find(p, &src) gives the
// match at p and find.next(p, end) skips the positions where the parse
// can only emit a literal. Commands go to
// lm[k] = lit_len | mlen << 16, srcs[k], dst[k] = destination - segment
// start. Returns the command count; *overflow is set if cap_cmd would be
// exceeded (the symbol budget makes that impossible).
template <class Find>
ACE_HD uint32_t parse_segment(const ParseCtx &g, uint64_t s, const Find &find, uint32_t *lm, uint64_t *srcs,
                              uint16_t *dst, uint32_t cap_cmd, bool *overflow) {
  const uint64_t seg_start = s << g.log2_S, seg_end = min64(g.n, seg_start + g.S);
  const uint32_t Ts = ruler_target(s, g.cap);
  const uint64_t cs = 4 + g.W;
  uint64_t p = seg_start, lit_start = seg_start, mlen_sum = 0;
  uint32_t ncmd = 0;
  bool have_next = false;
  uint64_t next_len = 0, next_src = 0;
  const bool sparse = g.sample_mask != 0;
  while (p < seg_end) {
    if (!have_next) {
      p = find.next(p, seg_end);
      if (p >= seg_end) break;
    }
    const uint64_t p0 = p;
    uint64_t src = 0, len = 0;
    if (sparse) {
      {
        len = find(p, &src);
        if (len) {
          uint64_t back = 0;
          const uint64_t max_back = p - (src + len);
          while (back < max_back && p - back > lit_start && src - back > 0 &&
                 g.in[src - back - 1] == g.in[p - back - 1]) {
            const uint64_t q = (src - back - 1) >> g.log2_S;
            if (q != s && ruler_target(q, g.cap) >= Ts) break;
            ++back;
          }
          p -= back;
          src -= back;
          len += back;
        }
      }
    } else if (have_next) {
      len = next_len;
      src = next_src;
      have_next = false;
    } else {
      len = find(p, &src);
    }
    if (!sparse && len >= g.min_match && p + 1 < seg_end) {
      next_len = find(p + 1, &next_src);
      if (next_len > len) {
        len = 0;
        have_next = true;
      }
    }
    if (len >= g.min_match) {
      const uint64_t lits = (p - seg_start) - mlen_sum;
      const uint64_t v_now = ncmd * cs + lits + (seg_end - p);
      if (v_now + cs > kMaxSym + len) len = 0;
      if (ncmd >= cap_cmd) {
        *overflow = true;
        len = 0;
      }
    }
    if (len < g.min_match) p = p0;
    if (len >= g.min_match) {
      lm[ncmd] = (uint32_t)(p - lit_start) | ((uint32_t)len << 16);
      srcs[ncmd] = src;
      dst[ncmd] = (uint16_t)(p - seg_start);
      ++ncmd;
      mlen_sum += len;
      p += len;
      lit_start = p;
    } else {
      ++p;
    }
  }
  return ncmd;
}

// Redirect a source that lies inside an earlier match's destination of the
// same segment to that match's source (same bytes, no new dependency,
// shorter chains for the decoder).
ACE_HD void flatten(const ParseCtx &g, uint64_t seg_start, uint32_t ncmd, const uint32_t *lm, uint64_t *srcs,
                    const uint16_t *dst) {
  for (uint32_t i = 0; i < ncmd; ++i) {
    const uint64_t mi = lm[i] >> 16;
    for (int guard = 0; guard < 64; ++guard) {
      const uint64_t a = srcs[i], b = a + mi;
      if (a < seg_start) break;
      const uint64_t rel = a - seg_start;
      uint32_t lo = 0, hi = i;  // first j < i with dst[j] > rel
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)dst[mid] <= rel) lo = mid + 1;
        else hi = mid;
      }
      if (lo == 0) break;
      const uint32_t j = lo - 1;
      const uint64_t dj = seg_start + dst[j];
      if (b > dj + (lm[j] >> 16)) break;
      const uint64_t ns = srcs[j] + (a - dj);
      if (g.D && seg_start + dst[i] - ns > g.D) break;
      srcs[i] = ns;
    }
  }
}

ACE_HD void sift_down(uint32_t *a, uint32_t i, uint32_t n) {
  for (;;) {
    uint32_t c = 2 * i + 1;
    if (c >= n) return;
    if (c + 1 < n && a[c + 1] > a[c]) ++c;
    if (a[i] >= a[c]) return;
    const uint32_t t = a[i];
    a[i] = a[c];
    a[c] = t;
    i = c;
  }
}

// Distinct source segments other than s, ascending, into tmp (room for two
// per command: a match is at most one segment long). Returns their count.
ACE_HD uint32_t collect_deps(uint64_t s, uint32_t log2_S, uint32_t ncmd, const uint32_t *lm, const uint64_t *srcs,
                             uint32_t *tmp) {
  uint32_t m = 0;
  for (uint32_t i = 0; i < ncmd; ++i) {
    const uint64_t src = srcs[i], ml = lm[i] >> 16;
    for (uint64_t q = src >> log2_S; q <= (src + ml - 1) >> log2_S; ++q)
      if (q != s) tmp[m++] = (uint32_t)q;
  }
  if (m > 1) {
    for (uint32_t i = m / 2; i-- > 0;) sift_down(tmp, i, m);
    for (uint32_t e = m - 1; e > 0; --e) {
      const uint32_t t = tmp[0];
      tmp[0] = tmp[e];
      tmp[e] = t;
      sift_down(tmp, 0, e);
    }
  }
  uint32_t u = 0;
  for (uint32_t i = 0; i < m; ++i)
    if (u == 0 || tmp[u - 1] != tmp[i]) tmp[u++] = tmp[i];
  return u;
}

// ------------------------------------------------------------ phase 1: chains

__global__ void __launch_bounds__(256) enc_hash_kernel(const uint8_t *in, uint64_t base, uint64_t lim, uint32_t hlen,
                                                       int bits, uint32_t sample_mask, uint32_t *keys,
                                                       uint32_t *vals) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t ma = hlen >= 8 ? ~0ull : (1ull << (8 * hlen)) - 1;
  const uint64_t mb = hlen <= 8 ? 0 : hlen >= 16 ? ~0ull : (1ull << (8 * (hlen - 8))) - 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lim; i += stride) {
    const uint8_t *p = in + base + i;
    const uint64_t a = load_le64(p) & ma;
    const uint64_t b = mb ? load_le64(p + 8) & mb : 0;
    const uint32_t h = hash_words(a, b, bits);
    // in sampled mode, unsampled positions get a key above every hash: they
    // sort last and are nobody's candidate
    keys[i] = (sample_mask && (h & sample_mask) != 0) ? (1u << bits) : h;
    vals[i] = (uint32_t)i;
  }
}

constexpr int kRsWarps = 8, kRsItems = 16, kRsTile = kRsWarps * 32 * kRsItems;  // 4096 pairs per tile
constexpr int kRsSmem = 4 * kRsTile * 4;  // scatter: the tile in input order and in digit order (keys, values)

__global__ void __launch_bounds__(256) rs_hist_kernel(const uint32_t *keys, uint64_t n, int shift, uint32_t ntiles,
                                                      uint32_t *hist) {
  __shared__ uint32_t c[256];
  c[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kRsTile;
  for (int k = 0; k < kRsTile / 256; ++k) {
    const uint64_t idx = base + (uint64_t)k * 256 + threadIdx.x;
    if (idx < n) atomicAdd(&c[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = c[threadIdx.x];
}

// Stable scatter of one tile: warp w owns pairs [tile + 512w, tile + 512w +
// 512), visited in index order (item k of lane l is 32k + l); the rank of a
// pair among equal digits is the count in earlier warps + earlier items of
// its warp + earlier lanes of its item (match_any groups equal digits). The
// tile is first ordered by digit in shared memory, so that each digit's run
// leaves as consecutive stores. The pairs wait in shared memory in input
// order meanwhile (only their ranks stay in registers).
__global__ void __launch_bounds__(256) rs_scatter_kernel(const uint32_t *kin, const uint32_t *vin, uint64_t n,
                                                         int shift, uint32_t ntiles, const uint32_t *offs,
                                                         uint32_t *kout, uint32_t *vout) {
  extern __shared__ uint32_t rs_dyn[];
  uint32_t *ink = rs_dyn, *inv = rs_dyn + kRsTile, *sk = rs_dyn + 2 * kRsTile, *sv = rs_dyn + 3 * kRsTile;
  __shared__ uint32_t toff[256], tstart[256], wsum[kRsWarps];
  __shared__ uint32_t wc[kRsWarps][256];
  const uint32_t tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  toff[tid] = offs[(uint64_t)tid * ntiles + blockIdx.x];
  for (uint32_t j = tid; j < kRsWarps * 256; j += 256) (&wc[0][0])[j] = 0;
  __syncthreads();
  const uint64_t tbase = (uint64_t)blockIdx.x * kRsTile;
  const uint64_t wbase = tbase + (uint64_t)w * 32 * kRsItems;
  const uint32_t lt = (1u << lane) - 1;
  const uint32_t lbase = w * 32 * kRsItems + lane;  // tile-local index of item 0
  uint32_t rk[kRsItems];
#pragma unroll
  for (int k = 0; k < kRsItems; ++k) {
    const uint64_t idx = wbase + (uint64_t)k * 32 + lane;
    const bool valid = idx < n;
    const uint32_t key = valid ? kin[idx] : 0;
    if (valid) {
      ink[lbase + 32 * k] = key;
      inv[lbase + 32 * k] = vin[idx];
    }
    const uint32_t d = valid ? (key >> shift) & 255u : 256u;
    const uint32_t peers = __match_any_sync(kFull, d);
    const uint32_t before = valid ? wc[w][d] : 0;
    __syncwarp();
    if (valid && lane == (uint32_t)(__ffs(peers) - 1)) wc[w][d] = before + __popc(peers);
    __syncwarp();
    rk[k] = before + __popc(peers & lt);
  }
  __syncthreads();
  // thread tid = digit: per-warp prefix of its count, then the tile's
  // exclusive prefix over digits (start of the digit's run in the tile)
  uint32_t cnt = 0;
  for (int v = 0; v < kRsWarps; ++v) {
    const uint32_t c = wc[v][tid];
    wc[v][tid] = cnt;
    cnt += c;
  }
  uint32_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  uint32_t wpre = 0;
  for (uint32_t v = 0; v < w; ++v) wpre += wsum[v];
  tstart[tid] = wpre + inc - cnt;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kRsItems; ++k) {
    const uint64_t idx = wbase + (uint64_t)k * 32 + lane;
    if (idx < n) {
      const uint32_t key = ink[lbase + 32 * k], d = (key >> shift) & 255u;
      const uint32_t at = tstart[d] + wc[w][d] + rk[k];
      sk[at] = key;
      sv[at] = inv[lbase + 32 * k];
    }
  }
  __syncthreads();
  const uint32_t tile_n = (uint32_t)min64(kRsTile, n - tbase);
  for (uint32_t i = tid; i < tile_n; i += 256) {
    const uint32_t k = sk[i], d = (k >> shift) & 255u;
    const uint64_t dest = (uint64_t)toff[d] + (i - tstart[d]);
    kout[dest] = k;
    vout[dest] = sv[i];
  }
}

// The match of every position of [a, b) that lies in the sorted window, one
// thread per sorted slot: candidates are the preceding slots (coalesced
// reads instead of a dependent walk), the result goes to t[p - a].
__global__ void __launch_bounds__(256) enc_match_kernel(ParseCtx g, const uint32_t *K, const uint32_t *V, uint64_t m,
                                                        uint32_t sentinel, uint64_t a, uint64_t b, uint64_t *table) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const uint64_t p = g.base + V[j];
    if (p < a || p >= b) continue;  // history before the window: a candidate only
    uint64_t v = 0;
    if (K[j] != sentinel) {
      uint64_t src;
      const uint64_t len = match_at_slot(g, K, V, j, p, &src);
      if (len) v = (len << 32) | (p - src);
    }
    table[p - a] = v;
  }
}

// One 64-bit mask word per warp iteration: bit q set when the match at
// position q of the table is usable (length >= min_len).
__global__ void __launch_bounds__(256) enc_mask_kernel(const uint64_t *table, uint64_t np, uint64_t min_len,
                                                       uint64_t *mask) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nwords = (np + 63) >> 6;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t w = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nwords; w += nwarps) {
    const uint64_t i0 = (w << 6) + lane, i1 = i0 + 32;
    const bool b0 = i0 < np && (table[i0] >> 32) >= min_len;
    const bool b1 = i1 < np && (table[i1] >> 32) >= min_len;
    const uint32_t lo = __ballot_sync(kFull, b0), hi = __ballot_sync(kFull, b1);
    if (lane == 0) mask[w] = (uint64_t)lo | ((uint64_t)hi << 32);
  }
}

// ------------------------------------------------------------ scans (1024 threads, 8 items each)

constexpr int kScThreads = 1024, kScItems = 8, kScTile = kScThreads * kScItems;

template <class T>
__device__ T block_exclusive_scan(T x, T *total) {
  __shared__ unsigned long long ws_raw[32];
  T *ws = reinterpret_cast<T *>(ws_raw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(kFull, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T v = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(kFull, v, o);
      if (lane >= (uint32_t)o) v += y;
    }
    ws[lane] = v;
  }
  __syncthreads();
  const T wpre = warp ? ws[warp - 1] : T(0);
  *total = ws[31];
  __syncthreads();
  return wpre + incl - x;
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(kScThreads) scan_reduce_kernel(const Tin *in, uint64_t n, Tout *part) {
  const uint64_t base = (uint64_t)blockIdx.x * kScTile;
  Tout sum = 0;
  for (int k = 0; k < kScItems; ++k) {
    const uint64_t idx = base + (uint64_t)k * kScThreads + threadIdx.x;
    if (idx < n) sum += (Tout)in[idx];
  }
  Tout total;
  block_exclusive_scan<Tout>(sum, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// one block: exclusive scan of part[0..nb) in place, starting at *init (0 when null)
template <class Tout>
__global__ void __launch_bounds__(kScThreads) scan_top_kernel(Tout *part, uint64_t nb, const Tout *init) {
  Tout carry = init ? *init : Tout(0);
  for (uint64_t base = 0; base < nb; base += kScTile) {
    Tout v[kScItems], t = 0;
    for (int k = 0; k < kScItems; ++k) {
      const uint64_t idx = base + (uint64_t)threadIdx.x * kScItems + k;
      v[k] = idx < nb ? part[idx] : Tout(0);
      t += v[k];
    }
    Tout total;
    Tout run = carry + block_exclusive_scan<Tout>(t, &total);
    for (int k = 0; k < kScItems; ++k) {
      const uint64_t idx = base + (uint64_t)threadIdx.x * kScItems + k;
      if (idx < nb) part[idx] = run;
      run += v[k];
    }
    carry += total;
  }
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(kScThreads) scan_down_kernel(const Tin *in, uint64_t n, const Tout *part, Tout *out,
                                                             int inclusive) {
  const uint64_t base = (uint64_t)blockIdx.x * kScTile;
  Tout v[kScItems], t = 0;
  for (int k = 0; k < kScItems; ++k) {
    const uint64_t idx = base + (uint64_t)threadIdx.x * kScItems + k;
    v[k] = idx < n ? (Tout)in[idx] : Tout(0);
    t += v[k];
  }
  Tout total;
  Tout run = part[blockIdx.x] + block_exclusive_scan<Tout>(t, &total);
  for (int k = 0; k < kScItems; ++k) {
    const uint64_t idx = base + (uint64_t)threadIdx.x * kScItems + k;
    if (inclusive) run += v[k];
    if (idx < n) out[idx] = run;
    if (!inclusive) run += v[k];
  }
}

// ------------------------------------------------------------ phases 2 and 3

struct BatchBufs {
  uint32_t *lm;
  uint64_t *srcs;
  uint16_t *dst;
  uint32_t *deptmp;
  uint32_t *ncmd;
  uint32_t *ndep;
  uint32_t cap_cmd;
};

__global__ void __launch_bounds__(128) enc_parse_kernel(ParseCtx g, uint64_t s0, uint32_t nb, TableFinder find,
                                                        BatchBufs b, uint32_t *err) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const uint64_t s = s0 + i, cmd0 = (uint64_t)i * b.cap_cmd;  // the segment's first command slot
  bool overflow = false;
  const uint32_t nc = parse_segment(g, s, find, b.lm + cmd0, b.srcs + cmd0, b.dst + cmd0, b.cap_cmd, &overflow);
  if (overflow) atomicOr(err, kErrCmdCap);
  flatten(g, s << g.log2_S, nc, b.lm + cmd0, b.srcs + cmd0, b.dst + cmd0);
  b.ncmd[i] = nc;
  b.ndep[i] = collect_deps(s, g.log2_S, nc, b.lm + cmd0, b.srcs + cmd0, b.deptmp + 2 * cmd0);
}

// One warp per segment: the symbol message (the format's symbol message) into
// sym[s * slot ...] and the per-class symbol counts.
__global__ void __launch_bounds__(256) enc_symbols_kernel(const uint8_t *in, uint64_t n, uint64_t s0, uint32_t nb,
                                                          uint32_t log2_S, uint32_t W, uint32_t min_match,
                                                          BatchBufs b, uint8_t *sym, uint32_t slot,
                                                          uint32_t *n_cmd, uint32_t *n_lit,
                                                          unsigned long long *counts, uint32_t *err) {
  __shared__ uint32_t hist[1024];
  for (uint32_t j = threadIdx.x; j < 1024; j += blockDim.x) hist[j] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t wpb = blockDim.x >> 5;
  for (uint32_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nb; i += gridDim.x * wpb) {
    const uint64_t s = s0 + i, cmd0 = (uint64_t)i * b.cap_cmd;
    const uint32_t nc = b.ncmd[i];
    const uint32_t *lm = b.lm + cmd0;
    const uint64_t *srcs = b.srcs + cmd0;
    uint8_t *out = sym + s * slot;
    const uint64_t seg_start = s << log2_S;
    const uint64_t seg_len = min64(n - seg_start, uint64_t(1) << log2_S);
    uint64_t mlen_sum = 0;  // the symbol count is n_cmd (4 + W) + seg_len - sum of match lengths
    for (uint32_t k = lane; k < nc; k += 32) mlen_sum += lm[k] >> 16;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mlen_sum += __shfl_xor_sync(kFull, mlen_sum, o);
    if ((uint64_t)(4 + W) * nc + seg_len - mlen_sum > slot) {  // cannot happen: the parse keeps n_sym <= slot
      if (lane == 0) atomicOr(err, kErrSymbols);
      continue;
    }
    for (uint32_t k = lane; k < nc; k += 32) {
      const uint32_t v = lm[k], ll = v & 0xffffu, mv = (v >> 16) - min_match;
      out[2 * k] = (uint8_t)ll;
      out[2 * k + 1] = (uint8_t)(ll >> 8);
      atomicAdd(&hist[ll & 255u], 1u);
      atomicAdd(&hist[ll >> 8], 1u);
      out[2 * nc + 2 * k] = (uint8_t)mv;
      out[2 * nc + 2 * k + 1] = (uint8_t)(mv >> 8);
      atomicAdd(&hist[256 + (mv & 255u)], 1u);
      atomicAdd(&hist[256 + (mv >> 8)], 1u);
      const uint64_t src = srcs[k];
      for (uint32_t by = 0; by < W; ++by) {
        const uint32_t x = (uint32_t)(src >> (8 * by)) & 255u;
        out[4 * (uint64_t)nc + (uint64_t)k * W + by] = (uint8_t)x;
        atomicAdd(&hist[512 + x], 1u);
      }
    }
    uint8_t *lit = out + (uint64_t)(4 + W) * nc;
    uint64_t lit_carry = 0, pos_carry = 0;
    for (uint32_t k0 = 0; k0 < nc; k0 += 32) {
      const uint32_t k = k0 + lane;
      const uint32_t v = k < nc ? lm[k] : 0u;
      const uint32_t ll = v & 0xffffu, adv = ll + (v >> 16);
      uint32_t il = ll, ia = adv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yl = __shfl_up_sync(kFull, il, o), ya = __shfl_up_sync(kFull, ia, o);
        if (lane >= (uint32_t)o) il += yl, ia += ya;
      }
      const uint64_t lo = lit_carry + il - ll, po = pos_carry + ia - adv;
      for (uint32_t t = 0; t < ll; ++t) {
        const uint8_t x = in[seg_start + po + t];
        lit[lo + t] = x;
        atomicAdd(&hist[768 + x], 1u);
      }
      lit_carry += __shfl_sync(kFull, il, 31);
      pos_carry += __shfl_sync(kFull, ia, 31);
    }
    const uint64_t ntr = seg_len - pos_carry;
    for (uint64_t t = lane; t < ntr; t += 32) {
      const uint8_t x = in[seg_start + pos_carry + t];
      lit[lit_carry + t] = x;
      atomicAdd(&hist[768 + x], 1u);
    }
    if (lane == 0) {
      n_cmd[s] = nc;
      n_lit[s] = (uint32_t)(lit_carry + ntr);
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < 1024; j += blockDim.x)
    if (hist[j]) atomicAdd(&counts[j], (unsigned long long)hist[j]);
}

// Levels of the batch's segments of one schedule tier (their sources lie in
// lower tiers, whose levels are final).
__global__ void __launch_bounds__(256) enc_levels_kernel(uint64_t s0, uint32_t nb, uint32_t cap, uint32_t tier,
                                                         BatchBufs b, uint16_t *level, uint32_t *err) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const uint64_t s = s0 + i;
  if (ruler_target(s, cap) != tier) return;
  const uint32_t *d = b.deptmp + 2 * (uint64_t)i * b.cap_cmd;
  uint32_t lv = 0;
  for (uint32_t k = 0; k < b.ndep[i]; ++k) {
    if (ruler_target(d[k], cap) >= tier) atomicOr(err, kErrSchedule);
    lv = max(lv, (uint32_t)level[d[k]] + 1u);
  }
  if (lv > cap) atomicOr(err, kErrLevel);
  level[s] = (uint16_t)lv;
}

__global__ void __launch_bounds__(256) enc_deps_copy_kernel(uint64_t s0, uint32_t nb, BatchBufs b,
                                                            const uint64_t *dep_ptr, uint32_t *deps) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const uint32_t *d = b.deptmp + 2 * (uint64_t)i * b.cap_cmd;
  uint32_t *o = deps + dep_ptr[s0 + i];
  for (uint32_t k = 0; k < b.ndep[i]; ++k) o[k] = d[k];
}

// ------------------------------------------------------------ phase 4: entropy coding and layout

// One warp per segment: the format's rANS encoder, 32 lanes, symbols in
// reverse order. Pass 1 (payload == nullptr) counts the words; pass 2
// writes the 32 initial states and the words in decode order.
__global__ void __launch_bounds__(256) enc_rans_kernel(const uint8_t *sym, uint32_t slot, const uint32_t *n_cmd,
                                                       const uint32_t *n_lit, uint64_t n_seg, uint32_t W,
                                                       const uint16_t *tabs, uint32_t *n_words, uint8_t *payload,
                                                       const uint64_t *poff) {
  __shared__ uint16_t f[1024], cum[1024];
  for (uint32_t j = threadIdx.x; j < 1024; j += blockDim.x) {
    f[j] = tabs[j];
    cum[j] = tabs[1024 + j];
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, gt = ~((2u << lane) - 1u);
  const uint32_t wpb = blockDim.x >> 5;
  for (uint64_t s = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5); s < n_seg; s += (uint64_t)gridDim.x * wpb) {
    const uint32_t nc = n_cmd[s];
    const uint32_t ns = nc * (4 + W) + n_lit[s];
    const uint32_t b1 = 2 * nc, b2 = 4 * nc, b3 = (4 + W) * nc;
    const uint8_t *m = sym + s * slot;
    uint32_t x = kRansL;
    uint32_t tail = payload ? n_words[s] : 0, count = 0;
    uint8_t *wbase = payload ? payload + poff[s] + 128 : nullptr;
    for (int64_t t = ((int64_t)ns + 31) / 32 - 1; t >= 0; --t) {
      const uint32_t q = (uint32_t)t * 32 + lane;
      bool emit = false;
      uint32_t word = 0;
      if (q < ns) {
        const uint32_t c = q < b1 ? 0u : q < b2 ? 1u : q < b3 ? 2u : 3u;
        const uint32_t e = c * 256 + m[q];
        const uint32_t fv = f[e];
        if ((uint64_t)x >= ((uint64_t)fv << 20)) {
          emit = true;
          word = x & 0xffffu;
          x >>= 16;
        }
        x = (x / fv) * kScale + (x % fv) + cum[e];
      }
      const uint32_t bal = __ballot_sync(kFull, emit);
      if (payload) {
        if (emit) {
          const uint32_t idx = tail - 1 - __popc(bal & gt);
          reinterpret_cast<uint16_t *>(wbase)[idx] = (uint16_t)word;
        }
        tail -= __popc(bal);
      } else {
        count += __popc(bal);
      }
    }
    if (payload) reinterpret_cast<uint32_t *>(payload + poff[s])[lane] = x;
    else if (lane == 0) n_words[s] = count;
  }
}

__global__ void __launch_bounds__(256) enc_sizes_kernel(const uint32_t *n_words, uint64_t n_seg, uint64_t *sz) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n_seg) sz[s] = (128 + 2 * (uint64_t)n_words[s] + 15) & ~uint64_t(15);  // round16
}

__global__ void __launch_bounds__(256) enc_dir_kernel(const uint64_t *poff, const uint32_t *n_words,
                                                      const uint32_t *n_cmd, const uint32_t *n_lit,
                                                      const uint16_t *level, uint64_t n_seg, uint8_t *dir) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_seg) return;
  uint64_t *r = reinterpret_cast<uint64_t *>(dir + 24 * s);
  r[0] = poff[s];
  r[1] = (uint64_t)n_words[s] | ((uint64_t)n_cmd[s] << 32);
  r[2] = (uint64_t)n_lit[s] | ((uint64_t)level[s] << 32);
}

// ------------------------------------------------------------ host side

struct Buf {
  void *p = nullptr;
  uint64_t cap = 0;
  cudaError_t reserve(uint64_t bytes) {  // contents are not kept
    if (bytes <= cap && p) return cudaSuccess;
    release();
    const cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e == cudaSuccess) cap = bytes ? bytes : 16;
    else p = nullptr;
    return e;
  }
  cudaError_t grow_keep(uint64_t bytes, uint64_t used, cudaStream_t st) {  // first `used` bytes kept
    if (bytes <= cap && p) return cudaSuccess;
    void *q = nullptr;
    const uint64_t nb = std::max<uint64_t>(bytes, cap + cap / 2);
    cudaError_t e = cudaMalloc(&q, nb);
    if (e != cudaSuccess) return e;
    if (used) e = cudaMemcpyAsync(q, p, used, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(q);
      return e;
    }
    if (p) cudaFree(p);
    p = q;
    cap = nb;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T>
  T *as() const {
    return static_cast<T *>(p);
  }
};

}  // namespace
}  // namespace aceapex

struct aceapex_gpu_encoder {
  int device = 0;
  int sms = 152;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[6] = {};
  uint64_t launches = 0;  // kernels launched by the current call
  aceapex::Buf in, kA, vA, kB, vB, hist, part;
  aceapex::Buf lm, srcs, dst, deptmp, bncmd, bndep, mtab, mask;
  aceapex::Buf sym, n_cmd, n_lit, n_words, level, dep_ptr, deps, poff, sz;
  aceapex::Buf counts, tabs, err, arc;
  ~aceapex_gpu_encoder() {
    aceapex::Buf *all[] = {&in, &kA, &vA, &kB, &vB, &hist, &part, &lm, &srcs, &dst,
                           &deptmp, &bncmd, &bndep, &mtab, &mask, &sym, &n_cmd, &n_lit, &n_words, &level, &dep_ptr, &deps,
                           &poff, &sz, &counts, &tabs, &err, &arc};
    for (auto *b : all) b->release();
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    if (st) cudaStreamDestroy(st);
  }
};

namespace aceapex {
namespace {

inline int cuda_rc(cudaError_t e) { return e == cudaSuccess ? ACEAPEX_OK : (e == cudaErrorMemoryAllocation ? ACEAPEX_ENOMEM : ACEAPEX_ECUDA); }

#define ENC_TRY(x)                      \
  do {                                  \
    const cudaError_t e_ = (x);         \
    if (e_ != cudaSuccess) return cuda_rc(e_); \
  } while (0)

// Scan of n elements of `in` into `out` (exclusive or inclusive), starting at
// *d_init (device; 0 when null). Tout is uint32_t or uint64_t.
template <class Tin, class Tout>
int device_scan(aceapex_gpu_encoder *E, const Tin *in, uint64_t n, Tout *out, const Tout *d_init, bool inclusive) {
  if (n == 0) return ACEAPEX_OK;
  const uint64_t nb = (n + kScTile - 1) / kScTile;
  ENC_TRY(E->part.reserve(nb * sizeof(Tout)));
  Tout *part = E->part.as<Tout>();
  scan_reduce_kernel<Tin, Tout><<<(unsigned)nb, kScThreads, 0, E->st>>>(in, n, part);
  scan_top_kernel<Tout><<<1, kScThreads, 0, E->st>>>(part, nb, d_init);
  scan_down_kernel<Tin, Tout><<<(unsigned)nb, kScThreads, 0, E->st>>>(in, n, part, out, inclusive ? 1 : 0);
  E->launches += 3;
  return cuda_rc(cudaGetLastError());
}

// Phase 1 for the window [base, end): the hashed positions [base, base +
// lim) sorted stably by hash; *K, *V receive the sorted keys and positions
// (relative to base).
int sort_window(aceapex_gpu_encoder *E, uint64_t n, uint64_t base, uint64_t end, uint32_t hlen, uint32_t smask,
                uint64_t *lim_out, const uint32_t **K, const uint32_t **V, uint32_t *sentinel) {
  const uint64_t len = end - base;
  const int bits = hash_bits_for(len);
  const uint64_t lim = (base + hlen <= n) ? std::min<uint64_t>(len, n - hlen + 1 - base) : 0;
  *lim_out = lim;
  *sentinel = smask ? (1u << bits) : 0xffffffffu;
  *K = *V = nullptr;
  if (lim == 0) return ACEAPEX_OK;
  ENC_TRY(E->kA.reserve(4 * lim));
  ENC_TRY(E->vA.reserve(4 * lim));
  ENC_TRY(E->kB.reserve(4 * lim));
  ENC_TRY(E->vB.reserve(4 * lim));
  const unsigned grid = (unsigned)E->sms * 8;
  enc_hash_kernel<<<grid, 256, 0, E->st>>>(E->in.as<uint8_t>(), base, lim, hlen, bits, smask, E->kA.as<uint32_t>(),
                                          E->vA.as<uint32_t>());
  ++E->launches;
  ENC_TRY(cudaGetLastError());
  const int key_bits = bits + (smask ? 1 : 0);
  const uint64_t ntiles = (lim + kRsTile - 1) / kRsTile;
  ENC_TRY(E->hist.reserve(4 * 256 * ntiles));
  uint32_t *ki = E->kA.as<uint32_t>(), *vi = E->vA.as<uint32_t>(), *ko = E->kB.as<uint32_t>(),
           *vo = E->vB.as<uint32_t>();
  for (int shift = 0; shift < key_bits; shift += 8) {
    rs_hist_kernel<<<(unsigned)ntiles, 256, 0, E->st>>>(ki, lim, shift, (uint32_t)ntiles, E->hist.as<uint32_t>());
    ++E->launches;
    ENC_TRY(cudaGetLastError());
    const int rc = device_scan<uint32_t, uint32_t>(E, E->hist.as<uint32_t>(), 256 * ntiles, E->hist.as<uint32_t>(),
                                                   nullptr, false);
    if (rc) return rc;
    rs_scatter_kernel<<<(unsigned)ntiles, 256, kRsSmem, E->st>>>(ki, vi, lim, shift, (uint32_t)ntiles,
                                                                E->hist.as<uint32_t>(), ko, vo);
    ++E->launches;
    ENC_TRY(cudaGetLastError());
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  *K = ki;
  *V = vi;
  return ACEAPEX_OK;
}

inline void put32(uint8_t *p, uint32_t v) { std::memcpy(p, &v, 4); }
inline void put64(uint8_t *p, uint64_t v) { std::memcpy(p, &v, 8); }

int gpu_encode_steps(aceapex_gpu_encoder *E, const uint8_t *in, int in_on_device, uint64_t n, uint32_t log2_B,
                     uint32_t min_match, uint32_t cap, uint64_t D, const uint64_t *reads, uint64_t n_reads,
                     uint8_t **out, uint64_t *out_len, aceapex_encode_stats *stats) {
  if (log2_B < 2 || log2_B > 30 || cap > 255 || (n && !in) || !out || !out_len || (n_reads && !reads))
    return ACEAPEX_EINVAL;
  const uint32_t log2_S = std::min<uint32_t>(log2_B, kMaxLog2S);
  const uint64_t S = uint64_t(1) << log2_S, n_seg = (n + S - 1) >> log2_S;
  const uint32_t W = offset_width(n);
  const uint32_t mm = min_match ? min_match : 4 + W;
  if (mm > 255) return ACEAPEX_EINVAL;
  for (uint64_t r = 0; r < n_reads; ++r)
    if (reads[r] >= n || (r && reads[r] <= reads[r - 1])) return ACEAPEX_EINVAL;
  if (D == 0 && n >= (uint64_t(1) << 32)) return ACEAPEX_EINVAL;
  if (D >= (uint64_t(1) << 31)) return ACEAPEX_EINVAL;
  if (n_seg >= (uint64_t(1) << 32)) return ACEAPEX_EINVAL;
  ENC_TRY(cudaSetDevice(E->device));
  cudaStream_t st = E->st;
  E->launches = 0;
  const uint32_t hlen = hash_len_for(mm), smask = sample_mask_for(mm);
  // a segment has at most S commands (every match is at least one byte) and
  // kMaxSym / (4 + W) of them (rule R-sym); its symbols number at most
  // kMaxSym and at most (4 + W) per byte
  const uint32_t cap_cmd = (uint32_t)std::min<uint64_t>(kMaxSym / (4 + W) + 1, S);
  const uint32_t slot = (uint32_t)std::min<uint64_t>(kMaxSym, S * (4 + W));

  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> chain_ev, parse_ev, match_ev;
  auto fresh_event = [](cudaEvent_t *e) { return cudaEventCreate(e); };
  struct EvGuard {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *a, *b, *c;
    ~EvGuard() {
      for (auto *v : {a, b, c})
        for (auto &pr : *v) {
          if (pr.first) cudaEventDestroy(pr.first);
          if (pr.second) cudaEventDestroy(pr.second);
        }
    }
  } guard{&chain_ev, &parse_ev, &match_ev};

  ENC_TRY(cudaEventRecord(E->ev[0], st));
  ENC_TRY(E->in.reserve(n + kInPad));
  ENC_TRY(cudaMemsetAsync(E->in.as<uint8_t>() + n, 0, kInPad, st));
  if (n) ENC_TRY(cudaMemcpyAsync(E->in.p, in, n, in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  ENC_TRY(cudaEventRecord(E->ev[1], st));

  ENC_TRY(E->err.reserve(4));
  ENC_TRY(cudaMemsetAsync(E->err.p, 0, 4, st));
  ENC_TRY(E->counts.reserve(8 * 1024));
  ENC_TRY(cudaMemsetAsync(E->counts.p, 0, 8 * 1024, st));
  const uint64_t segs = std::max<uint64_t>(n_seg, 1);
  ENC_TRY(E->sym.reserve(segs * slot));
  ENC_TRY(E->n_cmd.reserve(4 * segs));
  ENC_TRY(E->n_lit.reserve(4 * segs));
  ENC_TRY(E->n_words.reserve(4 * segs));
  ENC_TRY(E->level.reserve(2 * segs));
  ENC_TRY(E->dep_ptr.reserve(8 * (segs + 1)));
  ENC_TRY(E->poff.reserve(8 * (segs + 1)));
  ENC_TRY(E->sz.reserve(8 * segs));
  ENC_TRY(cudaMemsetAsync(E->dep_ptr.p, 0, 8, st));
  ENC_TRY(cudaMemsetAsync(E->poff.p, 0, 8, st));
  const uint32_t batch = (uint32_t)std::min<uint64_t>(kBatchSegs, segs);
  ENC_TRY(E->lm.reserve(4ull * batch * cap_cmd));
  ENC_TRY(E->srcs.reserve(8ull * batch * cap_cmd));
  ENC_TRY(E->dst.reserve(2ull * batch * cap_cmd));
  ENC_TRY(E->deptmp.reserve(8ull * batch * cap_cmd));
  ENC_TRY(E->bncmd.reserve(4ull * batch));
  ENC_TRY(E->bndep.reserve(4ull * batch));
  const uint64_t chunk = D ? std::max<uint64_t>(kDistWindow, S) : std::max<uint64_t>(n, 1);
  ENC_TRY(E->mtab.reserve(8 * std::min<uint64_t>(chunk, std::max<uint64_t>(n, 1))));
  ENC_TRY(E->mask.reserve(8 * ((std::min<uint64_t>(chunk, std::max<uint64_t>(n, 1)) + 63) / 64)));
  BatchBufs bb{E->lm.as<uint32_t>(), E->srcs.as<uint64_t>(), E->dst.as<uint16_t>(), E->deptmp.as<uint32_t>(),
               E->bncmd.as<uint32_t>(), E->bndep.as<uint32_t>(), cap_cmd};
  uint64_t deps_used = 0;  // entries of deps written so far

  // ---- phases 1-3, window by window (the host encoder's windows)
  for (uint64_t a = 0; a < n; a += chunk) {
    const uint64_t b = std::min(n, a + chunk);
    const uint64_t base = D ? (a > D ? a - D : 0) : 0;
    chain_ev.emplace_back(nullptr, nullptr);
    ENC_TRY(fresh_event(&chain_ev.back().first));
    ENC_TRY(fresh_event(&chain_ev.back().second));
    ENC_TRY(cudaEventRecord(chain_ev.back().first, st));
    uint64_t lim = 0;
    const uint32_t *K = nullptr, *V = nullptr;
    uint32_t sentinel = 0;
    int rc = sort_window(E, n, base, b, hlen, smask, &lim, &K, &V, &sentinel);
    if (rc) return rc;
    ENC_TRY(cudaEventRecord(chain_ev.back().second, st));
    // match table of [a, b) and its mask; positions past the last full hash
    // window have no match
    const ParseCtx g{E->in.as<uint8_t>(), n, base, S, D, log2_S, W, mm, cap, smask};
    uint64_t *table = E->mtab.as<uint64_t>();
    const uint64_t hashed_end = std::max(a, std::min(b, base + lim));
    if (hashed_end < b) ENC_TRY(cudaMemsetAsync(table + (hashed_end - a), 0, 8 * (b - hashed_end), st));
    match_ev.emplace_back(nullptr, nullptr);
    ENC_TRY(fresh_event(&match_ev.back().first));
    ENC_TRY(fresh_event(&match_ev.back().second));
    ENC_TRY(cudaEventRecord(match_ev.back().first, st));
    if (lim) {
      enc_match_kernel<<<(unsigned)E->sms * 16, 256, 0, st>>>(g, K, V, lim, sentinel, a, b, table);
      ++E->launches;
      ENC_TRY(cudaGetLastError());
    }
    ENC_TRY(cudaEventRecord(match_ev.back().second, st));
    parse_ev.emplace_back(nullptr, nullptr);
    ENC_TRY(fresh_event(&parse_ev.back().first));
    ENC_TRY(fresh_event(&parse_ev.back().second));
    ENC_TRY(cudaEventRecord(parse_ev.back().first, st));
    enc_mask_kernel<<<(unsigned)E->sms * 8, 256, 0, st>>>(table, b - a, smask ? 1 : mm, E->mask.as<uint64_t>());
    ++E->launches;
    ENC_TRY(cudaGetLastError());
    const TableFinder find{table, E->mask.as<uint64_t>(), a};
    const uint64_t s_lo = a >> log2_S, s_hi = (b + S - 1) >> log2_S;
    for (uint64_t s0 = s_lo; s0 < s_hi; s0 += batch) {
      const uint32_t nb = (uint32_t)std::min<uint64_t>(batch, s_hi - s0);
      enc_parse_kernel<<<(nb + 127) / 128, 128, 0, st>>>(g, s0, nb, find, bb, E->err.as<uint32_t>());
      ++E->launches;
      ENC_TRY(cudaGetLastError());
      enc_symbols_kernel<<<(unsigned)E->sms * 8, 256, 0, st>>>(
          E->in.as<uint8_t>(), n, s0, nb, log2_S, W, mm, bb, E->sym.as<uint8_t>(), slot, E->n_cmd.as<uint32_t>(),
          E->n_lit.as<uint32_t>(), E->counts.as<unsigned long long>(), E->err.as<uint32_t>());
      ++E->launches;
      ENC_TRY(cudaGetLastError());
      for (uint32_t tier = 0; tier <= cap; ++tier) {
        enc_levels_kernel<<<(nb + 255) / 256, 256, 0, st>>>(s0, nb, cap, tier, bb, E->level.as<uint16_t>(),
                                                           E->err.as<uint32_t>());
        ++E->launches;
        ENC_TRY(cudaGetLastError());
      }
      uint64_t *dp = E->dep_ptr.as<uint64_t>();
      rc = device_scan<uint32_t, uint64_t>(E, bb.ndep, nb, dp + s0 + 1, dp + s0, true);
      if (rc) return rc;
      uint64_t total = 0;
      ENC_TRY(cudaMemcpyAsync(&total, dp + s0 + nb, 8, cudaMemcpyDeviceToHost, st));
      ENC_TRY(cudaStreamSynchronize(st));
      ENC_TRY(E->deps.grow_keep(4 * std::max<uint64_t>(total, 1), 4 * deps_used, st));
      deps_used = total;
      enc_deps_copy_kernel<<<(nb + 255) / 256, 256, 0, st>>>(s0, nb, bb, dp, E->deps.as<uint32_t>());
      ++E->launches;
      ENC_TRY(cudaGetLastError());
    }
    ENC_TRY(cudaEventRecord(parse_ev.back().second, st));
  }

  // ---- phase 4: tables, rANS, layout
  uint64_t cnt[1024];
  uint32_t err = 0;
  ENC_TRY(cudaMemcpyAsync(cnt, E->counts.p, sizeof(cnt), cudaMemcpyDeviceToHost, st));
  ENC_TRY(cudaMemcpyAsync(&err, E->err.p, 4, cudaMemcpyDeviceToHost, st));
  ENC_TRY(cudaStreamSynchronize(st));
  if (err) return ACEAPEX_ECORRUPT;  // an encoder invariant failed (never expected)
  uint16_t f[4][256], tabs[2048];
  for (int c = 0; c < 4; ++c) {
    normalize_counts(cnt + 256 * c, f[c]);
    uint32_t acc = 0;
    for (int x = 0; x < 256; ++x) {
      tabs[256 * c + x] = f[c][x];
      tabs[1024 + 256 * c + x] = (uint16_t)acc;
      acc += f[c][x];
    }
  }
  ENC_TRY(E->tabs.reserve(sizeof(tabs)));
  ENC_TRY(cudaMemcpyAsync(E->tabs.p, tabs, sizeof(tabs), cudaMemcpyHostToDevice, st));
  const unsigned rgrid = (unsigned)E->sms * 8;
  uint64_t payload = 0;
  if (n_seg) {
    enc_rans_kernel<<<rgrid, 256, 0, st>>>(E->sym.as<uint8_t>(), slot, E->n_cmd.as<uint32_t>(), E->n_lit.as<uint32_t>(),
                                          n_seg, W, E->tabs.as<uint16_t>(), E->n_words.as<uint32_t>(), nullptr,
                                          nullptr);
    ENC_TRY(cudaGetLastError());
    enc_sizes_kernel<<<(unsigned)((n_seg + 255) / 256), 256, 0, st>>>(E->n_words.as<uint32_t>(), n_seg,
                                                                     E->sz.as<uint64_t>());
    E->launches += 2;
    ENC_TRY(cudaGetLastError());
    const int rc = device_scan<uint64_t, uint64_t>(E, E->sz.as<uint64_t>(), n_seg, E->poff.as<uint64_t>() + 1,
                                                   E->poff.as<uint64_t>(), true);
    if (rc) return rc;
    ENC_TRY(cudaMemcpyAsync(&payload, E->poff.as<uint64_t>() + n_seg, 8, cudaMemcpyDeviceToHost, st));
    ENC_TRY(cudaStreamSynchronize(st));
  }
  const uint64_t n_deps = deps_used;
  const uint64_t off_dir = kHeaderBytes + kTablesBytes;
  const uint64_t off_dep_ptr = round16(off_dir + 24 * n_seg);
  const uint64_t off_deps = round16(off_dep_ptr + 8 * (n_seg + 1));
  const uint64_t off_reads = round16(off_deps + 4 * n_deps);
  const uint64_t off_payload = round16(off_reads + 8 * n_reads);
  const uint64_t total = off_payload + payload;
  uint8_t head[kHeaderBytes + kTablesBytes];
  std::memset(head, 0, sizeof(head));
  std::memcpy(head, "ACEAPEX1", 8);
  put32(head + 8, 1);
  put32(head + 12, kHeaderBytes);
  put64(head + 16, n);
  head[24] = (uint8_t)log2_B;
  head[25] = (uint8_t)log2_S;
  head[26] = (uint8_t)W;
  head[27] = (uint8_t)mm;
  head[28] = (uint8_t)kScaleBits;
  head[29] = (uint8_t)kLanes;
  head[30] = (uint8_t)cap;
  head[31] = n_reads ? 1 : 0;
  put64(head + 32, D);
  put64(head + 40, n_seg);
  put64(head + 48, n_deps);
  put64(head + 56, n_reads);
  put64(head + 64, kHeaderBytes);
  put64(head + 72, off_dir);
  put64(head + 80, off_dep_ptr);
  put64(head + 88, off_deps);
  put64(head + 96, off_reads);
  put64(head + 104, off_payload);
  put64(head + 112, payload);
  put64(head + 120, total);
  std::memcpy(head + kHeaderBytes, f, sizeof(f));
  ENC_TRY(E->arc.reserve(total));
  uint8_t *A = E->arc.as<uint8_t>();
  ENC_TRY(cudaMemsetAsync(A, 0, total, st));
  ENC_TRY(cudaMemcpyAsync(A, head, sizeof(head), cudaMemcpyHostToDevice, st));
  if (n_seg) {
    enc_dir_kernel<<<(unsigned)((n_seg + 255) / 256), 256, 0, st>>>(
        E->poff.as<uint64_t>(), E->n_words.as<uint32_t>(), E->n_cmd.as<uint32_t>(), E->n_lit.as<uint32_t>(),
        E->level.as<uint16_t>(), n_seg, A + off_dir);
    ++E->launches;
    ENC_TRY(cudaGetLastError());
  }
  ENC_TRY(cudaMemcpyAsync(A + off_dep_ptr, E->dep_ptr.p, 8 * (n_seg + 1), cudaMemcpyDeviceToDevice, st));
  if (n_deps) ENC_TRY(cudaMemcpyAsync(A + off_deps, E->deps.p, 4 * n_deps, cudaMemcpyDeviceToDevice, st));
  if (n_reads) ENC_TRY(cudaMemcpyAsync(A + off_reads, reads, 8 * n_reads, cudaMemcpyHostToDevice, st));
  if (n_seg) {
    enc_rans_kernel<<<rgrid, 256, 0, st>>>(E->sym.as<uint8_t>(), slot, E->n_cmd.as<uint32_t>(), E->n_lit.as<uint32_t>(),
                                          n_seg, W, E->tabs.as<uint16_t>(), E->n_words.as<uint32_t>(),
                                          A + off_payload, E->poff.as<uint64_t>());
    ++E->launches;
    ENC_TRY(cudaGetLastError());
  }
  ENC_TRY(cudaEventRecord(E->ev[2], st));
  uint8_t *h = static_cast<uint8_t *>(std::malloc(total));
  if (!h) return ACEAPEX_ENOMEM;
  cudaError_t e = cudaMemcpyAsync(h, A, total, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(E->ev[3], st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&err, E->err.p, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess || err) {
    std::free(h);
    return e != cudaSuccess ? cuda_rc(e) : ACEAPEX_ECORRUPT;
  }
  *out = h;
  *out_len = total;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    float ms = 0;
    cudaEventElapsedTime(&ms, E->ev[0], E->ev[1]);
    stats->ms_h2d = ms;
    for (auto &pr : chain_ev) {
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      stats->ms_chains += ms;
    }
    for (auto &pr : match_ev) {
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      stats->ms_match += ms;
    }
    for (auto &pr : parse_ev) {
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      stats->ms_parse += ms;
    }
    stats->kernel_launches = E->launches;
    cudaEventElapsedTime(&ms, parse_ev.empty() ? E->ev[1] : parse_ev.back().second, E->ev[2]);
    stats->ms_entropy = ms;
    cudaEventElapsedTime(&ms, E->ev[2], E->ev[3]);
    stats->ms_d2h = ms;
    cudaEventElapsedTime(&ms, E->ev[0], E->ev[3]);
    stats->ms_total = ms;
    stats->input_bytes = n;
    stats->archive_bytes = total;
    stats->n_segments = n_seg;
    stats->n_deps = n_deps;
    stats->windows = chain_ev.size();
  }
  return ACEAPEX_OK;
}

// A call that fails part-way waits for the kernels it already queued, so
// that none is still running when the caller frees or reuses memory, or
// exits.
int gpu_encode(aceapex_gpu_encoder *E, const uint8_t *in, int in_on_device, uint64_t n, uint32_t log2_B,
               uint32_t min_match, uint32_t cap, uint64_t D, const uint64_t *reads, uint64_t n_reads, uint8_t **out,
               uint64_t *out_len, aceapex_encode_stats *stats) {
  const int rc =
      gpu_encode_steps(E, in, in_on_device, n, log2_B, min_match, cap, D, reads, n_reads, out, out_len, stats);
  if (rc != ACEAPEX_OK && E->st) cudaStreamSynchronize(E->st);
  return rc;
}

}  // namespace
}  // namespace aceapex

extern "C" {

int aceapex_gpu_encoder_create(int device, aceapex_gpu_encoder **out) {
  if (!out) return ACEAPEX_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return ACEAPEX_ECUDA;
  auto *E = new (std::nothrow) aceapex_gpu_encoder;
  if (!E) return ACEAPEX_ENOMEM;
  E->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&E->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&E->st, cudaStreamNonBlocking);
  for (auto &ev : E->ev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(aceapex::rs_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, aceapex::kRsSmem);
  if (e != cudaSuccess) {
    delete E;
    return ACEAPEX_ECUDA;
  }
  *out = E;
  return ACEAPEX_OK;
}

void aceapex_gpu_encoder_destroy(aceapex_gpu_encoder *E) {
  if (!E) return;
  cudaSetDevice(E->device);
  cudaStreamSynchronize(E->st);
  delete E;
}

int aceapex_gpu_encode(aceapex_gpu_encoder *E, const void *in, int in_on_device, uint64_t n, uint32_t log2_B,
                       uint32_t min_match, uint32_t max_level, uint64_t dist_bound, const uint64_t *h_reads,
                       uint64_t n_reads, void **h_out, uint64_t *out_len, aceapex_encode_stats *stats) {
  if (!E || !h_out || !out_len) return ACEAPEX_EINVAL;
  uint8_t *o = nullptr;
  const int rc = aceapex::gpu_encode(E, static_cast<const uint8_t *>(in), in_on_device, n, log2_B, min_match,
                                     max_level, dist_bound, h_reads, n_reads, &o, out_len, stats);
  *h_out = o;
  return rc;
}

}  // extern "C"
