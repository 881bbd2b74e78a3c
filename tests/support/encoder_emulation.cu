// Test helper (built by tests/test_library_host.py): runs the GPU encoder's
// per-thread device functions (match_at_slot, TableFinder, parse_segment,
// flatten, collect_deps, compiled for the host from gpu_encoder.cu) over a
// host-side stable sort, completes the archive on the host (levels, symbols,
// tables, rANS, layout as the archive format defines them) and compares it with the
// library's CPU encoder, byte for byte.
//
// usage: encoder_emulation <input file> <log2_B,min_match,max_level,D> ...
// prints one line per case and exits 1 if any archive differs.
#include "gpu_encoder.cu"

#include <algorithm>
#include <array>
#include <cstdio>

namespace aceapex {
int encode_archive(const uint8_t *in, uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t cap, uint64_t D,
                   const uint64_t *reads, uint64_t n_reads, int threads, uint8_t **out, uint64_t *out_len);
}
using namespace aceapex;

static void put(std::vector<uint8_t> &a, uint64_t off, const void *p, size_t len) { std::memcpy(&a[off], p, len); }

static std::vector<uint8_t> emulate(const std::vector<uint8_t> &src, uint32_t log2_B, uint32_t min_match, uint32_t cap,
                                    uint64_t D) {
  const uint64_t n = src.size();
  std::vector<uint8_t> in(src);
  in.resize(n + 64, 0);
  const uint32_t log2_S = std::min<uint32_t>(log2_B, kMaxLog2S);
  const uint64_t S = uint64_t(1) << log2_S, n_seg = (n + S - 1) >> log2_S;
  const uint32_t W = offset_width(n), mm = min_match ? min_match : 4 + W;
  const uint32_t hlen = hash_len_for(mm), smask = sample_mask_for(mm);
  const uint32_t cap_cmd = (uint32_t)std::min<uint64_t>(kMaxSym / (4 + W) + 1, S);
  std::vector<std::vector<uint32_t>> LM(n_seg), DP(n_seg);
  std::vector<std::vector<uint64_t>> SR(n_seg);
  const uint64_t chunk = D ? std::max<uint64_t>(kDistWindow, S) : std::max<uint64_t>(n, 1);
  for (uint64_t a = 0; a < n; a += chunk) {
    const uint64_t b = std::min(n, a + chunk), base = D ? (a > D ? a - D : 0) : 0, len = b - base;
    const int bits = hash_bits_for(len);
    const uint64_t lim = (base + hlen <= n) ? std::min<uint64_t>(len, n - hlen + 1 - base) : 0;
    const uint64_t ma = hlen >= 8 ? ~0ull : (1ull << (8 * hlen)) - 1;
    const uint64_t mb = hlen <= 8 ? 0 : hlen >= 16 ? ~0ull : (1ull << (8 * (hlen - 8))) - 1;
    std::vector<uint32_t> keys(lim), order(lim);
    for (uint64_t i = 0; i < lim; ++i) {
      const uint8_t *p = in.data() + base + i;
      const uint32_t h = hash_words(load_le64(p) & ma, mb ? load_le64(p + 8) & mb : 0, bits);
      keys[i] = (smask && (h & smask) != 0) ? (1u << bits) : h;
      order[i] = (uint32_t)i;
    }
    std::stable_sort(order.begin(), order.end(), [&](uint32_t u, uint32_t v) { return keys[u] < keys[v]; });
    std::vector<uint32_t> K(lim + 1), V(lim + 1);
    for (uint64_t j = 0; j < lim; ++j) K[j] = keys[order[j]], V[j] = order[j];
    const uint32_t sentinel = smask ? (1u << bits) : 0xffffffffu;
    const ParseCtx g{in.data(), n, base, S, D, log2_S, W, mm, cap, smask};
    std::vector<uint64_t> table(b - a, 0), mask((b - a + 63) / 64 + 1, 0);
    for (uint64_t j = 0; j < lim; ++j) {
      const uint64_t p = base + V[j];
      if (p < a || p >= b || K[j] == sentinel) continue;
      uint64_t s;
      const uint64_t l = match_at_slot(g, K.data(), V.data(), j, p, &s);
      if (l) table[p - a] = (l << 32) | (p - s);
    }
    const uint64_t min_len = smask ? 1 : mm;
    for (uint64_t q = 0; q < b - a; ++q)
      if ((table[q] >> 32) >= min_len) mask[q >> 6] |= 1ull << (q & 63);
    const TableFinder find{table.data(), mask.data(), a};
    for (uint64_t s = a >> log2_S; s < ((b + S - 1) >> log2_S); ++s) {
      std::vector<uint32_t> lm(cap_cmd), tmp(2 * cap_cmd);
      std::vector<uint64_t> sr(cap_cmd);
      std::vector<uint16_t> dst(cap_cmd);
      bool overflow = false;
      const uint32_t nc = parse_segment(g, s, find, lm.data(), sr.data(), dst.data(), cap_cmd, &overflow);
      if (overflow) return {};
      flatten(g, s << log2_S, nc, lm.data(), sr.data(), dst.data());
      const uint32_t nd = collect_deps(s, log2_S, nc, lm.data(), sr.data(), tmp.data());
      LM[s].assign(lm.begin(), lm.begin() + nc);
      SR[s].assign(sr.begin(), sr.begin() + nc);
      DP[s].assign(tmp.begin(), tmp.begin() + nd);
    }
  }
  // levels, symbol messages (the format's symbol message) and class counts
  std::vector<uint16_t> level(n_seg);
  std::vector<std::vector<uint8_t>> sym(n_seg);
  std::vector<uint32_t> nlit(n_seg);
  uint64_t cnt[1024] = {};
  auto cls = [&](uint64_t q, uint64_t nc) { return q < 2 * nc ? 0 : q < 4 * nc ? 1 : q < (4 + W) * nc ? 2 : 3; };
  for (uint64_t s = 0; s < n_seg; ++s) {
    uint32_t lv = 0;
    for (uint32_t d : DP[s]) lv = std::max<uint32_t>(lv, level[d] + 1u);
    if (lv > cap) return {};
    level[s] = (uint16_t)lv;
    const uint64_t nc = LM[s].size();
    auto &m = sym[s];
    for (uint32_t v : LM[s]) m.push_back(v & 255), m.push_back((v >> 8) & 255);
    for (uint32_t v : LM[s]) m.push_back(((v >> 16) - mm) & 255), m.push_back(((v >> 16) - mm) >> 8);
    for (uint64_t x : SR[s])
      for (uint32_t k = 0; k < W; ++k) m.push_back((x >> (8 * k)) & 255);
    uint64_t p = s << log2_S;
    const uint64_t end = std::min(n, p + S);
    for (uint32_t v : LM[s]) {
      for (uint32_t t = 0; t < (v & 0xffffu); ++t) m.push_back(in[p + t]);
      p += (v & 0xffffu) + (v >> 16);
    }
    while (p < end) m.push_back(in[p++]);
    nlit[s] = (uint32_t)(m.size() - nc * (4 + W));
    for (uint64_t q = 0; q < m.size(); ++q) cnt[256 * cls(q, nc) + m[q]]++;
  }
  uint16_t f[4][256];
  uint32_t cum[4][256];
  for (int c = 0; c < 4; ++c) {
    normalize_counts(cnt + 256 * c, f[c]);
    uint32_t acc = 0;
    for (int x = 0; x < 256; ++x) cum[c][x] = acc, acc += f[c][x];
  }
  // rANS (the format's rANS encoder, run backwards over the symbols) and layout (§5)
  std::vector<std::vector<uint16_t>> words(n_seg);
  std::vector<std::array<uint32_t, 32>> states(n_seg);
  for (uint64_t s = 0; s < n_seg; ++s) {
    const auto &m = sym[s];
    const uint64_t nc = LM[s].size();
    uint32_t x[32];
    for (auto &v : x) v = kRansL;
    for (uint64_t q = m.size(); q-- > 0;) {
      const int c = cls(q, nc);
      const uint32_t j = q & 31, fv = f[c][m[q]];
      if ((uint64_t)x[j] >= ((uint64_t)fv << 20)) words[s].push_back(x[j] & 0xffffu), x[j] >>= 16;
      x[j] = (x[j] / fv) * kScale + x[j] % fv + cum[c][m[q]];
    }
    std::reverse(words[s].begin(), words[s].end());
    for (int j = 0; j < 32; ++j) states[s][j] = x[j];
  }
  std::vector<uint64_t> poff(n_seg + 1, 0), dep_ptr(n_seg + 1, 0);
  for (uint64_t s = 0; s < n_seg; ++s) {
    poff[s + 1] = round16(poff[s] + 128 + 2 * words[s].size());
    dep_ptr[s + 1] = dep_ptr[s] + DP[s].size();
  }
  const uint64_t n_deps = dep_ptr[n_seg], off_dir = kHeaderBytes + kTablesBytes;
  const uint64_t off_dep_ptr = round16(off_dir + 24 * n_seg), off_deps = round16(off_dep_ptr + 8 * (n_seg + 1));
  const uint64_t off_reads = round16(off_deps + 4 * n_deps), off_payload = off_reads;
  const uint64_t total = off_payload + poff[n_seg];
  std::vector<uint8_t> A(total, 0);
  put(A, 0, "ACEAPEX1", 8);
  const uint32_t h32[2] = {1, kHeaderBytes};
  put(A, 8, h32, 8);
  put(A, 16, &n, 8);
  const uint8_t h8[8] = {(uint8_t)log2_B, (uint8_t)log2_S, (uint8_t)W, (uint8_t)mm, (uint8_t)kScaleBits,
                         (uint8_t)kLanes, (uint8_t)cap, 0};
  put(A, 24, h8, 8);
  const uint64_t h64[12] = {D, n_seg, n_deps, 0, kHeaderBytes, off_dir, off_dep_ptr, off_deps, off_reads,
                            off_payload, poff[n_seg], total};
  put(A, 32, h64, sizeof(h64));
  put(A, kHeaderBytes, f, sizeof(f));
  for (uint64_t s = 0; s < n_seg; ++s) {
    const SegRec r{poff[s], (uint32_t)words[s].size(), (uint32_t)LM[s].size(), nlit[s], level[s], 0};
    put(A, off_dir + 24 * s, &r, 24);
    put(A, off_payload + poff[s], states[s].data(), 128);
    if (!words[s].empty()) put(A, off_payload + poff[s] + 128, words[s].data(), 2 * words[s].size());
  }
  put(A, off_dep_ptr, dep_ptr.data(), 8 * (n_seg + 1));
  for (uint64_t s = 0, k = 0; s < n_seg; ++s)
    for (uint32_t d : DP[s]) put(A, off_deps + 4 * k++, &d, 4);
  return A;
}

int main(int argc, char **argv) {
  if (argc < 3) return 2;
  FILE *fp = std::fopen(argv[1], "rb");
  if (!fp) return 2;
  std::vector<uint8_t> data;
  for (int c; (c = std::fgetc(fp)) != EOF;) data.push_back((uint8_t)c);
  std::fclose(fp);
  int bad = 0;
  for (int i = 2; i < argc; ++i) {
    unsigned log2_B = 14, mm = 0, cap = 8;
    unsigned long long D = 0;
    if (std::sscanf(argv[i], "%u,%u,%u,%llu", &log2_B, &mm, &cap, &D) != 4) return 2;
    const auto A = emulate(data, log2_B, mm, cap, D);
    uint8_t *o = nullptr;
    uint64_t ol = 0;
    const int rc = encode_archive(data.data(), data.size(), log2_B, mm, cap, D, nullptr, 0, 4, &o, &ol);
    const bool same = rc == 0 && !A.empty() && ol == A.size() && std::memcmp(o, A.data(), ol) == 0;
    std::printf("%s %s n=%zu bytes=%llu\n", same ? "same" : "DIFF", argv[i], data.size(), (unsigned long long)ol);
    bad += !same;
    std::free(o);
  }
  return bad ? 1 : 0;
}
