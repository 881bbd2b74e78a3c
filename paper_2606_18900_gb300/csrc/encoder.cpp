// Host encoder of the library (paper §2: global match search over the whole
// decompressed history, absolute offsets, fixed-size blocks; the paper's
// encoder is also CPU-only and slow, §8). It writes version-1 archives.
//
// Design, differing from a plain sequential encoder in three ways so that it
// is fast and deterministic for any thread count:
//  * Hash chains over a window are built once, then every segment is parsed
//    in parallel; a candidate for position p is found by walking prev[] from
//    p itself, so only earlier positions are seen.
//  * The level cap is met by a fixed schedule instead of a greedy test: each
//    segment s gets a target T(s) = cap - min(cap, ctz(s+1)) (a "ruler"),
//    and s may read segment q < s only if T(q) < T(s). Then
//    level(s) <= T(s) <= cap without knowing the other segments' parses, and
//    half of all segments (those with even s+1) stay referenceable.
//  * Intra-segment chains are flattened after parsing: a match whose source
//    lies inside the destination of an earlier match of the same segment is
//    redirected to that match's source. The bytes are the same, the
//    dependency set does not grow, and the decoder sees shorter chains.
#include <sys/mman.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "encoder_rules.h"
#include "format.h"

namespace aceapex {

struct Cmd {
  uint32_t lit_len;
  uint32_t mlen;
  uint64_t src;
};

namespace {

struct Geo {
  uint64_t n, S, n_seg, D;
  uint32_t log2_B, log2_S, W, min_match, cap;
};

template <class F>
void parallel_for(uint64_t n, int threads, F &&f) {
  if (threads <= 1 || n < 2) {
    for (uint64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<uint64_t> next{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&] {
      for (;;) {
        uint64_t i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto &th : pool) th.join();
}


// Uninitialised buffer of T backed by transparent huge pages when possible
// (the chain arrays are several GB; first-touch faults on 4 KiB pages cost
// more than the hashing). Reused across the windows of one encode call.
template <class T>
struct RawBuf {
  T *p = nullptr;
  uint64_t cap = 0;
  void reserve(uint64_t n) {
    if (n <= cap) return;
    std::free(p);
    const uint64_t bytes = ((n * sizeof(T)) + (2u << 20) - 1) & ~uint64_t((2u << 20) - 1);
    p = static_cast<T *>(std::aligned_alloc(2u << 20, bytes));
    if (!p) throw std::bad_alloc();
#ifdef MADV_HUGEPAGE
    madvise(p, bytes, MADV_HUGEPAGE);
#endif
    cap = n;
  }
  ~RawBuf() { std::free(p); }
  T &operator[](uint64_t i) { return p[i]; }
  const T &operator[](uint64_t i) const { return p[i]; }
};

struct Window {
  const uint8_t *in;
  uint64_t n;        // total input length
  uint64_t base;     // first position covered by the chains
  uint64_t end;      // one past the last position covered
  uint32_t hlen;
  uint32_t sample_mask;  // positions whose hash & mask != 0 are neither indexed nor probed
  uint64_t lim;          // positions [base, base + lim) have a full hash window
  RawBuf<uint32_t> prev;  // prev[p - base]: previous indexed position (relative + 1) with the same hash, 0 = none
  RawBuf<uint32_t> hv;    // hash of each position
  RawBuf<uint32_t> idx;   // positions bucketed by hash partition
  RawBuf<uint32_t> head;
  bool sampled(uint64_t p) const { return p >= base && p - base < lim && (hv[p - base] & sample_mask) == 0; }
};

// hash of the first hlen (<= 16) bytes at p, kHashBits wide
inline uint32_t hash_at(const uint8_t *p, uint32_t hlen, int kHashBits) {
  uint64_t a = 0, b = 0;
  std::memcpy(&a, p, hlen < 8 ? hlen : 8);
  if (hlen > 8) std::memcpy(&b, p + 8, hlen - 8);
  return hash_words(a, b, kHashBits);
}

// Chains equal to one sequential insertion pass, built in parallel: hash
// every position (parallel over ranges), stably bucket the positions by the
// top bits of their hash (counting sort, parallel over ranges), then each
// partition's thread inserts its positions in increasing order. A partition
// owns its head entries, so no two threads touch the same chain.
void build_chains(Window &w, int threads) {
  const uint64_t len = w.end - w.base;
  const int kHashBits = hash_bits_for(len);
  const uint64_t lim = (w.base + w.hlen <= w.n) ? std::min<uint64_t>(len, w.n - w.hlen + 1 - w.base) : 0;
  w.lim = lim;
  w.prev.reserve(len ? len : 1);
  w.hv.reserve(lim ? lim : 1);
  w.idx.reserve(lim ? lim : 1);
  const uint64_t hsize = uint64_t(1) << kHashBits;
  w.head.reserve(hsize);
  int tb = 0;
  while ((1 << (tb + 1)) <= threads && tb < 8) ++tb;
  const int parts = 1 << tb;
  const int ranges = std::max(1, threads);
  parallel_for((uint64_t)ranges, threads, [&](uint64_t r) {
    const uint64_t hs = (hsize + ranges - 1) / ranges, a = std::min(hsize, r * hs), b = std::min(hsize, a + hs);
    std::memset(w.head.p + a, 0, (b - a) * 4);
    const uint64_t ps = (len + ranges - 1) / ranges, c = std::min(len, r * ps), e = std::min(len, c + ps);
    std::memset(w.prev.p + c, 0, (e - c) * 4);
  });
  if (lim == 0) return;
  const uint64_t rs = (lim + ranges - 1) / ranges;
  std::vector<uint64_t> cnt((size_t)ranges * parts, 0);
  const uint32_t smask = w.sample_mask;
  parallel_for((uint64_t)ranges, threads, [&](uint64_t r) {
    const uint64_t a = r * rs, b = std::min(lim, a + rs);
    uint64_t *c = &cnt[r * parts];
    for (uint64_t i = a; i < b; ++i) {
      const uint32_t h = hash_at(w.in + w.base + i, w.hlen, kHashBits);
      w.hv[i] = h;
      if ((h & smask) == 0) ++c[tb ? (h >> (kHashBits - tb)) : 0];
    }
  });
  // offsets: partition-major, range-minor (keeps each partition's positions ascending)
  std::vector<uint64_t> off((size_t)ranges * parts), pstart(parts + 1, 0);
  uint64_t acc = 0;
  for (int p = 0; p < parts; ++p) {
    pstart[p] = acc;
    for (int r = 0; r < ranges; ++r) {
      off[(size_t)r * parts + p] = acc;
      acc += cnt[(size_t)r * parts + p];
    }
  }
  pstart[parts] = acc;
  parallel_for((uint64_t)ranges, threads, [&](uint64_t r) {
    const uint64_t a = r * rs, b = std::min(lim, a + rs);
    uint64_t *o = &off[r * parts];
    for (uint64_t i = a; i < b; ++i) {
      const uint32_t h = w.hv[i];
      if ((h & smask) == 0) w.idx[o[tb ? (h >> (kHashBits - tb)) : 0]++] = (uint32_t)i;
    }
  });
  parallel_for((uint64_t)parts, threads, [&](uint64_t p) {
    const uint64_t a = pstart[p], b = pstart[p + 1];
    for (uint64_t j = a; j < b; ++j) {
      if (j + 16 < b) __builtin_prefetch(&w.head[w.hv[w.idx[j + 16]]], 1, 0);  // hide the random head access
      const uint32_t i = w.idx[j], h = w.hv[i];
      w.prev[i] = w.head[h];
      w.head[h] = i + 1;
    }
  });
}

inline uint64_t common_len(const uint8_t *a, const uint8_t *b, uint64_t lim) {
  uint64_t L = 0;
  while (L + 8 <= lim) {
    uint64_t x, y;
    std::memcpy(&x, a + L, 8);
    std::memcpy(&y, b + L, 8);
    if (x != y) return L + (uint64_t)(__builtin_ctzll(x ^ y) >> 3);
    L += 8;
  }
  while (L < lim && a[L] == b[L]) ++L;
  return L;
}

struct Parser {
  const Geo &g;
  const Window &w;
  uint32_t chain;

  // longest legal match at p in segment s (see the rules in parse_segment)
  uint64_t find(uint64_t s, uint32_t Ts, uint64_t p, uint64_t seg_end, uint64_t *src_out) const {
    if (p + w.hlen > g.n || p < w.base) return 0;
    uint64_t best = 0, best_src = 0;
    uint32_t c1 = w.prev[p - w.base];
    for (uint32_t k = 0; k < chain && c1 != 0; ++k) {
      uint64_t c = w.base + c1 - 1;
      c1 = w.prev[c - w.base];
      if (g.D && p - c > g.D) break;
      uint64_t lim = std::min<uint64_t>(p - c, seg_end - p);
      // clip at the first source segment that the level schedule forbids
      uint64_t q0 = c >> g.log2_S, q1 = (c + lim - 1) >> g.log2_S;
      for (uint64_t q = q0; q <= q1; ++q) {
        if (q != s && ruler_target(q, g.cap) >= Ts) {
          uint64_t allowed = (q << g.log2_S) > c ? (q << g.log2_S) - c : 0;
          lim = std::min(lim, allowed);
          break;
        }
      }
      if (lim <= best) continue;
      // a longer match than best agrees on bytes [0, best]: the 8 bytes
      // ending at best decide most losers with one comparison
      if (best >= 7) {
        uint64_t x, y;
        std::memcpy(&x, w.in + c + best - 7, 8);
        std::memcpy(&y, w.in + p + best - 7, 8);
        if (x != y) continue;
      }
      uint64_t L = common_len(w.in + c, w.in + p, lim);
      if (L > best) {
        best = L;
        best_src = c;
        if ((L == lim && lim == seg_end - p) || L >= kGoodEnough) break;
      }
    }
    *src_out = best_src;
    return best;
  }

  // Parse segment s. Rules: mlen >= min_match, src + mlen <=
  // dst, the match stays inside its segment, dst - src <= D, and the symbol
  // budget n_cmd*(4+W) + literals + bytes still to produce stays <= kMaxSym.
  void parse_segment(uint64_t s, std::vector<Cmd> &out) const {
    uint64_t seg_start = s << g.log2_S, seg_end = std::min(g.n, seg_start + g.S);
    uint32_t Ts = ruler_target(s, g.cap);
    const uint64_t cs = 4 + g.W;
    uint64_t p = seg_start, lit_start = seg_start, ncmd = 0, mlen_sum = 0;
    bool have_next = false;
    uint64_t next_len = 0, next_src = 0;
    const bool sparse = w.sample_mask != 0;
    while (p < seg_end) {
      const uint64_t p0 = p;
      uint64_t src = 0, len = 0;
      if (sparse) {
        // content-defined anchors: probe here only if this position was
        // indexed, then extend the match backwards over the literal run
        if (w.sampled(p)) {
          len = find(s, Ts, p, seg_end, &src);
          if (len) {
            // src + len <= p - back keeps the source off the destination (R-order)
            uint64_t back = 0;
            const uint64_t max_back = p - (src + len);
            while (back < max_back && p - back > lit_start && src - back > 0 &&
                   w.in[src - back - 1] == w.in[p - back - 1]) {
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
        len = find(s, Ts, p, seg_end, &src);
      }
      if (!sparse && len >= g.min_match && p + 1 < seg_end) {
        next_len = find(s, Ts, p + 1, seg_end, &next_src);
        if (next_len > len) {  // one-step lazy: a literal now, the longer match next
          len = 0;
          have_next = true;
        }
      }
      if (len >= g.min_match) {
        uint64_t lits = (p - seg_start) - mlen_sum;
        uint64_t v_now = ncmd * cs + lits + (seg_end - p);
        if (v_now + cs > kMaxSym + len) len = 0;
      }
      if (len < g.min_match) p = p0;  // a rejected extension must not move the scan back
      if (len >= g.min_match) {
        out.push_back(Cmd{(uint32_t)(p - lit_start), (uint32_t)len, src});
        ++ncmd;
        mlen_sum += len;
        p += len;
        lit_start = p;
      } else {
        ++p;
      }
    }
    flatten(s, seg_start, out);
  }

  // redirect intra-segment sources that sit inside an earlier match's output
  void flatten(uint64_t s, uint64_t seg_start, std::vector<Cmd> &cmds) const {
    (void)s;
    std::vector<uint64_t> dst(cmds.size());
    uint64_t p = seg_start;
    for (size_t i = 0; i < cmds.size(); ++i) {
      p += cmds[i].lit_len;
      dst[i] = p;
      p += cmds[i].mlen;
    }
    for (size_t i = 0; i < cmds.size(); ++i) {
      for (int guard = 0; guard < 64; ++guard) {
        uint64_t a = cmds[i].src, b = a + cmds[i].mlen;
        if (a < seg_start) break;
        // the latest earlier match whose destination starts at or before a
        size_t j = (size_t)(std::upper_bound(dst.begin(), dst.begin() + i, a) - dst.begin());
        if (j == 0) break;
        --j;
        if (b > dst[j] + cmds[j].mlen) break;  // not fully inside match j
        uint64_t ns = cmds[j].src + (a - dst[j]);
        if (g.D && dst[i] - ns > g.D) break;
        cmds[i].src = ns;
      }
    }
  }
};

// ----------------------------------------------------------------- rANS

struct Tables {
  uint16_t f[4][256];
  uint32_t c[4][257];
};


inline int sym_class(uint64_t q, uint64_t n, uint32_t W) {
  return q < 2 * n ? 0 : q < 4 * n ? 1 : q < (4 + (uint64_t)W) * n ? 2 : 3;
}

uint64_t segment_symbols(const uint8_t *in, const Geo &g, uint64_t s, const std::vector<Cmd> &cmds,
                         uint8_t *sym) {
  uint64_t n = cmds.size(), q = 0;
  for (auto &c : cmds) { sym[q++] = (uint8_t)c.lit_len; sym[q++] = (uint8_t)(c.lit_len >> 8); }
  for (auto &c : cmds) {
    uint32_t v = c.mlen - g.min_match;
    sym[q++] = (uint8_t)v;
    sym[q++] = (uint8_t)(v >> 8);
  }
  for (auto &c : cmds)
    for (uint32_t b = 0; b < g.W; ++b) sym[q++] = (uint8_t)(c.src >> (8 * b));
  uint64_t p = s << g.log2_S, end = std::min(g.n, p + g.S);
  for (auto &c : cmds) {
    std::memcpy(sym + q, in + p, c.lit_len);
    q += c.lit_len;
    p += c.lit_len + c.mlen;
  }
  std::memcpy(sym + q, in + p, end - p);
  q += end - p;
  (void)n;
  return q;
}

struct Coded {
  uint32_t states[kLanes];
  std::vector<uint16_t> words;
  uint32_t n_lit;
};

void rans_encode(const uint8_t *sym, uint64_t n_sym, uint64_t nc, uint32_t W, const Tables &t, Coded &out) {
  uint32_t x[kLanes];
  for (uint32_t j = 0; j < kLanes; ++j) x[j] = kRansL;
  out.words.clear();
  out.words.reserve(n_sym / 2 + 16);
  for (uint64_t q = n_sym; q-- > 0;) {
    uint32_t j = (uint32_t)(q & (kLanes - 1));
    int c = sym_class(q, nc, W);
    uint32_t s = sym[q], f = t.f[c][s];
    if ((uint64_t)x[j] >= (uint64_t(1) << 20) * f) {
      out.words.push_back((uint16_t)x[j]);
      x[j] >>= 16;
    }
    x[j] = (x[j] / f) * kScale + (x[j] % f) + t.c[c][s];
  }
  std::reverse(out.words.begin(), out.words.end());
  std::memcpy(out.states, x, sizeof(x));
}

inline void put16(uint8_t *p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
inline void put32(uint8_t *p, uint32_t v) { std::memcpy(p, &v, 4); }
inline void put64(uint8_t *p, uint64_t v) { std::memcpy(p, &v, 8); }

}  // namespace

void normalize_counts(const uint64_t *cnt, uint16_t *f) {
  uint64_t total = 0;
  for (int s = 0; s < 256; ++s) total += cnt[s];
  std::memset(f, 0, 512);
  if (!total) return;
  int64_t sum = 0;
  for (int s = 0; s < 256; ++s) {
    if (!cnt[s]) continue;
    uint64_t v = (uint64_t)(((unsigned __int128)cnt[s] * kScale + total / 2) / total);
    if (v < 1) v = 1;
    f[s] = (uint16_t)v;
    sum += (int64_t)v;
  }
  // fix the sum on the symbols with the largest counts (ties: lowest symbol)
  int order[256];
  for (int s = 0; s < 256; ++s) order[s] = s;
  std::stable_sort(order, order + 256, [&](int a, int b) { return cnt[a] > cnt[b]; });
  int64_t diff = (int64_t)kScale - sum;
  for (int k = 0; diff != 0; k = (k + 1) % 256) {
    int s = order[k];
    if (!cnt[s]) { k = -1; continue; }
    if (diff > 0) { f[s]++; diff--; }
    else if (f[s] > 1) { f[s]--; diff++; }
  }
}

// Returns 0 or an aceapex_status code. *out is malloc'd.
int encode_archive(const uint8_t *in, uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t cap, uint64_t D,
                   const uint64_t *reads, uint64_t n_reads, int threads, uint8_t **out, uint64_t *out_len) {
  static_assert(__BYTE_ORDER__ == __ORDER_LITTLE_ENDIAN__, "little-endian host");
  if (log2_B < 2 || log2_B > 30 || cap > 255 || (n && !in) || !out || !out_len) return 1;
  Geo g;
  g.n = n;
  g.log2_B = log2_B;
  g.log2_S = std::min<uint32_t>(log2_B, kMaxLog2S);
  g.S = uint64_t(1) << g.log2_S;
  g.n_seg = (n + g.S - 1) >> g.log2_S;
  g.W = offset_width(n);
  g.min_match = min_match ? min_match : 4 + g.W;
  g.cap = cap;
  g.D = D;
  if (g.min_match > 255) return 1;
  for (uint64_t r = 0; r < n_reads; ++r)
    if (reads[r] >= n || (r && reads[r] <= reads[r - 1])) return 1;
  if (D == 0 && n >= (uint64_t(1) << 32)) return 1;  // unbounded history needs 32-bit chains
  if (D >= (uint64_t(1) << 31)) return 1;
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());

  // ---- parse, window by window
  std::vector<std::vector<Cmd>> cmds(g.n_seg);
  const uint64_t chunk = D ? std::max<uint64_t>(kDistWindow, g.S) : std::max<uint64_t>(n, 1);
  Window w;
  w.in = in;
  w.n = n;
  w.hlen = hash_len_for(g.min_match);
  // Long minimum matches use content-defined sampling: a position is indexed
  // and probed only when the low bits of its hash are zero (1 in 4), which
  // finds a match of length >= hlen + 15 with probability > 0.99 (a
  // sampled position falls inside its first min_match - hlen + 1 starts) and
  // cuts the indexing and probing work by four.
  w.sample_mask = sample_mask_for(g.min_match);
  for (uint64_t a = 0; a < n; a += chunk) {
    uint64_t b = std::min(n, a + chunk);
    w.base = D ? (a > D ? a - D : 0) : 0;
    w.end = b;
    build_chains(w, threads);
    Parser P{g, w, kChainDepth};
    uint64_t s0 = a >> g.log2_S, s1 = (b + g.S - 1) >> g.log2_S;
    parallel_for(s1 - s0, threads, [&](uint64_t i) { P.parse_segment(s0 + i, cmds[s0 + i]); });
  }

  // ---- deps and levels (sequential: levels of earlier segments first)
  std::vector<uint64_t> dep_ptr(g.n_seg + 1, 0);
  std::vector<uint32_t> deps;
  std::vector<uint16_t> level(g.n_seg, 0);
  {
    std::vector<uint64_t> tmp;
    for (uint64_t s = 0; s < g.n_seg; ++s) {
      tmp.clear();
      for (auto &c : cmds[s])
        for (uint64_t q = c.src >> g.log2_S; q <= (c.src + c.mlen - 1) >> g.log2_S; ++q)
          if (q != s) tmp.push_back(q);
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      uint32_t lv = 0;
      for (uint64_t q : tmp) {
        deps.push_back((uint32_t)q);
        lv = std::max<uint32_t>(lv, level[q] + 1u);
      }
      if (lv > cap) return 2;  // cannot happen under the schedule
      level[s] = (uint16_t)lv;
      dep_ptr[s + 1] = deps.size();
    }
  }

  // ---- symbol counts and tables
  Tables t;
  {
    std::vector<std::vector<uint64_t>> part(threads, std::vector<uint64_t>(4 * 256, 0));
    std::atomic<uint64_t> next{0};
    std::vector<std::thread> pool;
    for (int th = 0; th < threads; ++th)
      pool.emplace_back([&, th] {
        std::vector<uint8_t> sym(kMaxSym);
        for (;;) {
          uint64_t s = next.fetch_add(1);
          if (s >= g.n_seg) break;
          uint64_t nc = cmds[s].size(), ns = segment_symbols(in, g, s, cmds[s], sym.data());
          for (uint64_t q = 0; q < ns; ++q) part[th][sym_class(q, nc, g.W) * 256 + sym[q]]++;
        }
      });
    for (auto &th : pool) th.join();
    uint64_t cnt[4][256] = {};
    for (auto &pp : part)
      for (int i = 0; i < 1024; ++i) cnt[i / 256][i % 256] += pp[i];
    for (int c = 0; c < 4; ++c) {
      normalize_counts(cnt[c], t.f[c]);
      t.c[c][0] = 0;
      for (int s = 0; s < 256; ++s) t.c[c][s + 1] = t.c[c][s] + t.f[c][s];
    }
  }

  // ---- rANS per segment
  std::vector<Coded> coded(g.n_seg);
  {
    std::atomic<uint64_t> next{0};
    std::vector<std::thread> pool;
    for (int th = 0; th < threads; ++th)
      pool.emplace_back([&] {
        std::vector<uint8_t> sym(kMaxSym);
        for (;;) {
          uint64_t s = next.fetch_add(1);
          if (s >= g.n_seg) break;
          uint64_t nc = cmds[s].size(), ns = segment_symbols(in, g, s, cmds[s], sym.data());
          coded[s].n_lit = (uint32_t)(ns - nc * (4 + g.W));
          rans_encode(sym.data(), ns, nc, g.W, t, coded[s]);
        }
      });
    for (auto &th : pool) th.join();
  }

  // ---- layout (the format's section layout)
  std::vector<uint64_t> poff(g.n_seg + 1, 0);
  for (uint64_t s = 0; s < g.n_seg; ++s) poff[s + 1] = round16(poff[s] + 128 + 2 * coded[s].words.size());
  uint64_t payload = poff[g.n_seg];
  uint64_t off_dir = kHeaderBytes + kTablesBytes;
  uint64_t off_dep_ptr = round16(off_dir + 24 * g.n_seg);
  uint64_t off_deps = round16(off_dep_ptr + 8 * (g.n_seg + 1));
  uint64_t off_reads = round16(off_deps + 4 * deps.size());
  uint64_t off_payload = round16(off_reads + 8 * n_reads);
  uint64_t total = off_payload + payload;
  uint8_t *a = (uint8_t *)std::calloc(total, 1);
  if (!a) return 3;
  std::memcpy(a, "ACEAPEX1", 8);
  put32(a + 8, 1);
  put32(a + 12, 128);
  put64(a + 16, n);
  a[24] = (uint8_t)g.log2_B;
  a[25] = (uint8_t)g.log2_S;
  a[26] = (uint8_t)g.W;
  a[27] = (uint8_t)g.min_match;
  a[28] = (uint8_t)kScaleBits;
  a[29] = (uint8_t)kLanes;
  a[30] = (uint8_t)cap;
  a[31] = n_reads ? 1 : 0;
  put64(a + 32, D);
  put64(a + 40, g.n_seg);
  put64(a + 48, deps.size());
  put64(a + 56, n_reads);
  put64(a + 64, kHeaderBytes);
  put64(a + 72, off_dir);
  put64(a + 80, off_dep_ptr);
  put64(a + 88, off_deps);
  put64(a + 96, off_reads);
  put64(a + 104, off_payload);
  put64(a + 112, payload);
  put64(a + 120, total);
  for (int c = 0; c < 4; ++c)
    for (int s = 0; s < 256; ++s) put16(a + kHeaderBytes + 512 * c + 2 * s, t.f[c][s]);
  parallel_for(g.n_seg, threads, [&](uint64_t s) {
    SegRec r{poff[s], (uint32_t)coded[s].words.size(), (uint32_t)cmds[s].size(), coded[s].n_lit, level[s], 0};
    std::memcpy(a + off_dir + 24 * s, &r, 24);
    uint8_t *pl = a + off_payload + poff[s];
    std::memcpy(pl, coded[s].states, 128);
    std::memcpy(pl + 128, coded[s].words.data(), 2 * coded[s].words.size());
  });
  std::memcpy(a + off_dep_ptr, dep_ptr.data(), 8 * (g.n_seg + 1));
  if (!deps.empty()) std::memcpy(a + off_deps, deps.data(), 4 * deps.size());
  if (n_reads) std::memcpy(a + off_reads, reads, 8 * n_reads);
  *out = a;
  *out_len = total;
  return 0;
}

uint64_t fastq_index(const uint8_t *in, uint64_t n, uint64_t *out, uint64_t cap) {
  uint64_t k = 0, line = 0;
  bool start = true;
  for (uint64_t p = 0; p < n; ++p) {
    if (start) {
      if ((line & 3) == 0) {
        if (k < cap) out[k] = p;
        ++k;
      }
      start = false;
    }
    if (in[p] == '\n') {
      ++line;
      start = true;
    }
  }
  return k;
}

// FASTA coordinate index: for every record, the offset of its '>' and the
// offset of its first sequence byte (the byte after the header line). The
// line width is the longest first sequence line of any record (every line
// of a record but its last has that length in a well-formed file). '>' only
// starts headers, so the scan jumps from one '>' to the next with memchr.
uint64_t fasta_index(const uint8_t *in, uint64_t n, uint64_t *out, uint64_t cap, uint32_t *line_width) {
  uint64_t k = 0, width = 0;
  for (uint64_t p = 0; p < n;) {
    const void *g = std::memchr(in + p, '>', n - p);
    if (!g) break;
    const uint64_t q = static_cast<const uint8_t *>(g) - in;
    p = q + 1;
    if (q > 0 && in[q - 1] != '\n') continue;  // not at a line start
    const void *e = std::memchr(in + q, '\n', n - q);
    if (!e) break;  // a header without a sequence line
    const uint64_t seq = static_cast<const uint8_t *>(e) - in + 1;
    if (k < cap) out[k] = q;
    if (k + 1 < cap) out[k + 1] = seq;
    k += 2;
    const void *l = seq < n ? std::memchr(in + seq, '\n', n - seq) : nullptr;
    if (l) width = std::max<uint64_t>(width, static_cast<const uint8_t *>(l) - in - seq);
    p = seq;
  }
  // a file whose last line has no newline gets one more entry, the offset of
  // its last byte, so that lookups know the last line is not terminated
  if (k >= 2 && n > 0 && in[n - 1] != '\n' && (k > cap || n - 1 > out[k - 1])) {
    if (k < cap) out[k] = n - 1;
    ++k;
  }
  if (line_width) *line_width = (uint32_t)width;
  return k;
}

// FASTQ stream separation: line k of the input goes to stream k mod 4
// (headers, sequences, '+' lines, qualities), each line with its newline; the
// streams are written back to back to out (n bytes) and their lengths to
// len[0..3]. Returns the number of records (lines of stream 0).
uint64_t fastq_split(const uint8_t *in, uint64_t n, uint8_t *out, uint64_t len[4]) {
  for (int k = 0; k < 4; ++k) len[k] = 0;
  uint64_t line = 0;
  for (uint64_t p = 0; p < n;) {  // pass 1: stream lengths
    const void *e = std::memchr(in + p, '\n', n - p);
    const uint64_t q = e ? static_cast<const uint8_t *>(e) - in + 1 : n;
    len[line & 3] += q - p;
    ++line;
    p = q;
  }
  uint64_t at[4] = {0, len[0], len[0] + len[1], len[0] + len[1] + len[2]};
  line = 0;
  for (uint64_t p = 0; p < n;) {  // pass 2: copy
    const void *e = std::memchr(in + p, '\n', n - p);
    const uint64_t q = e ? static_cast<const uint8_t *>(e) - in + 1 : n;
    std::memcpy(out + at[line & 3], in + p, q - p);
    at[line & 3] += q - p;
    ++line;
    p = q;
  }
  return (line + 3) / 4;
}

}  // namespace aceapex
