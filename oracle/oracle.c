/*
 * ACEAPEX CPU oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential implementation of the absolute-offset LZ77 block
 * codec of the paper (§2: absolute back-references into the decompressed
 * output, global match search, fixed-size blocks, four streams per block; §5:
 * 64-bit size and offset fields) in the byte format of version 1 of the archive format.
 * It exists to produce archives for the tests and to define the expected
 * decoded bytes. Only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg may load it; the GPU library never links or calls it, and
 * the two share no code.
 *
 * Contents:
 *   orc_crc32            CRC-32/IEEE (reflected 0xEDB88320): the bitwise
 *                        definition and its byte-table form.
 *   orc_geometry         segment/block counts and offset width (segment geometry of the format).
 *   orc_normalize        rANS frequency normalisation (the format's frequency
 *                        tables: 256 u16 per class summing to 4096).
 *   orc_parse            encoder, match search (paper §2: global search over
 *                        the whole history, absolute offsets, fixed blocks),
 *                        greedy with one-step lazy evaluation, under the
 *                        level cap and distance bound readings.
 *   orc_serialize        streams + rANS + archive layout (the format's symbol message, rANS coding and layout).
 *   orc_decode           sequential decoder + validator (every rule of the format).
 *   orc_decode_stream    the same decoder writing into a ring with one CRC
 *                        per window (paper §5 range decode; CRC replaces the
 *                        paper's FNV/XXH3 check).
 *   orc_segment_info     per-segment commands, symbols and final states for
 *                        the invariant tests.
 *   orc_fastq_record_starts  the read-to-block index of paper §4.1.
 *   orc_decode_wavefront the same segment decoder run level by level on
 *                        several host threads (all segments of a level at
 *                        once, a barrier between levels): the all-core CPU
 *                        baseline, the analog of the paper's CPU-T8 runs.
 *
 * Everything is integer arithmetic; there is no precision axis (the paper
 * requires bit-perfect output, §2.2).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ECORRUPT = 2, ORC_ENOMEM = 3, ORC_ERANGE = 6 };

#define SYM_MAX 16384u
#define LANES 32u
#define SCALE_BITS 12u
#define M_SCALE 4096u
#define RANS_L 65536u

typedef struct {
  uint32_t lit_len;
  uint32_t mlen;
  uint64_t src;
} orc_cmd;

/* ------------------------------------------------------------------ CRC-32 */

/* bitwise definition: shift out one bit at a time, reflected polynomial */
uint32_t orc_crc32_bitwise(uint32_t crc, const uint8_t *p, uint64_t n) {
  crc = ~crc;
  for (uint64_t i = 0; i < n; ++i) {
    crc ^= p[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

/* byte-table form (Sarwate): the table entry of a byte is its bitwise CRC step */
static uint32_t crc_table[256];
static int crc_table_ready = 0;

uint32_t orc_crc32(uint32_t crc, const uint8_t *p, uint64_t n) {
  if (!crc_table_ready) {
    for (uint32_t b = 0; b < 256; ++b) {
      uint32_t c = b;
      for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
      crc_table[b] = c;
    }
    crc_table_ready = 1;
  }
  crc = ~crc;
  for (uint64_t i = 0; i < n; ++i) crc = (crc >> 8) ^ crc_table[(crc ^ p[i]) & 0xFFu];
  return ~crc;
}

/* ---------------------------------------------------------------- helpers */

static uint64_t round16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }

static void put_u16(uint8_t *p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put_u32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static void put_u64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t get_u16(const uint8_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t get_u32(const uint8_t *p) {
  uint32_t v = 0;
  for (int i = 3; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
static uint64_t get_u64(const uint8_t *p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}

/* smallest w >= 1 with 256^w >= n (segment geometry of the format) */
static uint32_t offset_width(uint64_t n) {
  uint32_t w = 1;
  while (w < 8 && (n > (((uint64_t)1) << (8 * w)))) ++w;
  return w;
}

/* ------------------------------------------------------- rANS tables (§4) */

/*
 * counts -> frequencies summing to 4096, each present symbol >= 1. Any rule
 * is valid because tables are stored; this one: proportional floor, then the
 * rounding deficit goes to the most frequent symbol (lowest on ties), or an
 * excess is taken one unit at a time from the largest frequency > 1.
 */
void orc_normalize(const uint64_t counts[256], uint16_t freqs[256]) {
  uint64_t total = 0;
  for (int s = 0; s < 256; ++s) total += counts[s];
  for (int s = 0; s < 256; ++s) freqs[s] = 0;
  if (total == 0) return;
  int64_t sum = 0;
  for (int s = 0; s < 256; ++s) {
    if (counts[s] == 0) continue;
    uint64_t f = (uint64_t)(((unsigned __int128)counts[s] * M_SCALE) / total);
    if (f < 1) f = 1;
    freqs[s] = (uint16_t)f;
    sum += (int64_t)f;
  }
  int64_t diff = (int64_t)M_SCALE - sum;
  if (diff > 0) {
    int best = -1;
    for (int s = 0; s < 256; ++s)
      if (counts[s] && (best < 0 || counts[s] > counts[best])) best = s;
    freqs[best] = (uint16_t)(freqs[best] + diff);
  }
  while (diff < 0) {
    int best = -1;
    for (int s = 0; s < 256; ++s)
      if (freqs[s] > 1 && (best < 0 || freqs[s] > freqs[best])) best = s;
    freqs[best]--;
    diff++;
  }
}

/* ---------------------------------------------------------- parsing (§2) */

typedef struct {
  uint32_t log2_B, log2_S, W, min_match, max_level;
  uint64_t D, n, S, n_seg;
} geom_t;

static int make_geom(uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t max_level, uint64_t D,
                     geom_t *g) {
  if (log2_B < 2 || log2_B > 30 || min_match < 1 || min_match > 255 || max_level > 255) return ORC_EINVAL;
  g->log2_B = log2_B;
  g->log2_S = log2_B < 14 ? log2_B : 14;
  g->S = (uint64_t)1 << g->log2_S;
  g->W = offset_width(n);
  g->min_match = min_match;
  g->max_level = max_level;
  g->D = D;
  g->n = n;
  g->n_seg = (n + g->S - 1) / g->S;
  return ORC_OK;
}

/* n_segments, n_blocks and W of an archive of n bytes (segment geometry of the format) */
int orc_geometry(uint64_t n, uint32_t log2_B, uint64_t *n_segments, uint64_t *n_blocks, uint32_t *W,
                 uint32_t *log2_S) {
  geom_t g;
  if (make_geom(n, log2_B, 1, 0, 0, &g)) return ORC_EINVAL;
  *n_segments = g.n_seg;
  *n_blocks = (n + ((uint64_t)1 << log2_B) - 1) >> log2_B;
  *W = g.W;
  *log2_S = g.log2_S;
  return ORC_OK;
}

#define HASH_BITS 20

static uint32_t hash_at(const uint8_t *in, uint64_t p, uint32_t hlen) {
  uint64_t v = 0;
  for (uint32_t i = 0; i < hlen; ++i) v = (v << 8) | in[p + i];
  return (uint32_t)((v * 0x9E3779B97F4A7C15ull) >> (64 - HASH_BITS));
}

typedef struct {
  const uint8_t *in;
  const geom_t *g;
  uint64_t *head, *prev;     /* hash chains over every earlier position */
  uint16_t *level;           /* levels of finished segments */
  uint32_t hlen, chain;
} parser_t;

/*
 * Longest legal match at position p of segment s (p < seg_end). Walks at most
 * `chain` earlier positions with the same hash, newest first. A candidate c is
 * legal for length L if c + L <= p (R-order), p + L <= seg_end (a match stays
 * in its segment), p - c <= D when D > 0 (R-dist), and every source segment
 * other than s has level < max_level (R-level reading: sources of a level
 * at the cap are skipped). Returns the length (0 if none), source in *src.
 */
static uint64_t find_match(const parser_t *P, uint64_t s, uint64_t p, uint64_t seg_end, uint64_t *src) {
  const geom_t *g = P->g;
  const uint8_t *in = P->in;
  if (p + P->hlen > g->n) return 0;
  uint64_t best = 0, best_src = 0;
  uint64_t c = P->head[hash_at(in, p, P->hlen)];
  for (uint32_t k = 0; k < P->chain && c != UINT64_MAX; ++k, c = P->prev[c]) {
    if (g->D && p - c > g->D) break;
    uint64_t lim = p - c;
    if (seg_end - p < lim) lim = seg_end - p;
    /* stop before the first source segment that may not be referenced */
    uint64_t L = 0;
    while (L < lim && in[c + L] == in[p + L]) {
      uint64_t sseg = (c + L) >> g->log2_S;
      if (sseg != s && P->level[sseg] >= g->max_level) break;
      ++L;
    }
    if (L > best) { best = L; best_src = c; }
  }
  *src = best_src;
  return best;
}

static void insert_pos(parser_t *P, uint64_t p) {
  if (p + P->hlen > P->g->n) return;
  uint32_t h = hash_at(P->in, p, P->hlen);
  P->prev[p] = P->head[h];
  P->head[h] = p;
}

/*
 * Encoder parse. Returns the number of commands (>= 0) or a negative error.
 * *cmds_out (n_cmd entries) and *cmd_ptr_out (n_seg + 1 entries, commands of
 * segment s are [cmd_ptr[s], cmd_ptr[s+1])) are malloc'd; free with orc_free.
 */
int64_t orc_parse(const uint8_t *in, uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t max_level,
                  uint64_t D, uint32_t chain, orc_cmd **cmds_out, uint64_t **cmd_ptr_out) {
  geom_t g;
  if (make_geom(n, log2_B, min_match, max_level, D, &g)) return -ORC_EINVAL;
  parser_t P;
  P.in = in;
  P.g = &g;
  P.hlen = min_match < 6 ? min_match : 6;
  P.chain = chain ? chain : 16;
  P.head = (uint64_t *)malloc(sizeof(uint64_t) << HASH_BITS);
  P.prev = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
  P.level = (uint16_t *)calloc(g.n_seg + 1, sizeof(uint16_t));
  uint8_t *mark = (uint8_t *)calloc(g.n_seg + 1, 1);
  uint64_t *touched = (uint64_t *)malloc(sizeof(uint64_t) * (g.n_seg + 1));
  uint64_t cap = 1024, n_cmd = 0;
  orc_cmd *cmds = (orc_cmd *)malloc(sizeof(orc_cmd) * cap);
  uint64_t *cmd_ptr = (uint64_t *)malloc(sizeof(uint64_t) * (g.n_seg + 1));
  if (!P.head || !P.prev || !P.level || !mark || !touched || !cmds || !cmd_ptr) {
    free(P.head); free(P.prev); free(P.level); free(mark); free(touched); free(cmds); free(cmd_ptr);
    return -ORC_ENOMEM;
  }
  for (uint64_t i = 0; i < ((uint64_t)1 << HASH_BITS); ++i) P.head[i] = UINT64_MAX;
  const uint64_t cmd_syms = 4 + g.W;

  for (uint64_t s = 0; s < g.n_seg; ++s) {
    cmd_ptr[s] = n_cmd;
    uint64_t seg_start = s * g.S, seg_end = seg_start + g.S < n ? seg_start + g.S : n;
    uint64_t p = seg_start, lit_start = seg_start, seg_cmds = 0, n_touched = 0, seg_mlen = 0;
    uint16_t lvl = 0;
    while (p < seg_end) {
      uint64_t src = 0, len = find_match(&P, s, p, seg_end, &src);
      /* one-step lazy evaluation: prefer a literal if p + 1 starts a longer match */
      if (len >= min_match && p + 1 < seg_end) {
        insert_pos(&P, p);
        uint64_t src2 = 0, len2 = find_match(&P, s, p + 1, seg_end, &src2);
        P.head[hash_at(in, p, P.hlen)] = P.prev[p]; /* undo the insert; redone below */
        if (len2 > len) len = 0;
      }
      /* R-sym: n_cmd(4+W) + literals + bytes still to produce never exceeds SYM_MAX */
      uint64_t lits = p - seg_start - seg_mlen;
      uint64_t v_now = seg_cmds * cmd_syms + lits + (seg_end - p);
      if (len >= min_match && v_now + cmd_syms > SYM_MAX + len) len = 0;
      if (len >= min_match) {
        if (n_cmd == cap) {
          cap *= 2;
          orc_cmd *nc = (orc_cmd *)realloc(cmds, sizeof(orc_cmd) * cap);
          if (!nc) { free(P.head); free(P.prev); free(P.level); free(mark); free(touched); free(cmds); free(cmd_ptr); return -ORC_ENOMEM; }
          cmds = nc;
        }
        cmds[n_cmd].lit_len = (uint32_t)(p - lit_start);
        cmds[n_cmd].mlen = (uint32_t)len;
        cmds[n_cmd].src = src;
        ++n_cmd;
        ++seg_cmds;
        seg_mlen += len;
        for (uint64_t q = src >> g.log2_S; q <= (src + len - 1) >> g.log2_S; ++q) {
          if (q == s || mark[q]) continue;
          mark[q] = 1;
          touched[n_touched++] = q;
          if (P.level[q] + 1 > lvl) lvl = (uint16_t)(P.level[q] + 1);
        }
        for (uint64_t q = p; q < p + len; ++q) insert_pos(&P, q);
        p += len;
        lit_start = p;
      } else {
        insert_pos(&P, p);
        ++p;
      }
    }
    for (uint64_t i = 0; i < n_touched; ++i) mark[touched[i]] = 0;
    P.level[s] = lvl;
  }
  cmd_ptr[g.n_seg] = n_cmd;
  free(P.head); free(P.prev); free(P.level); free(mark); free(touched);
  *cmds_out = cmds;
  *cmd_ptr_out = cmd_ptr;
  return (int64_t)n_cmd;
}

void orc_free(void *p) { free(p); }

/* ----------------------------------------------------- serialization (§3-5) */

/* class of symbol q in a segment with n commands (the format's symbol message) */
static int sym_class(uint64_t q, uint64_t n, uint32_t W) {
  if (q < 2 * n) return 0;
  if (q < 4 * n) return 1;
  if (q < (4 + (uint64_t)W) * n) return 2;
  return 3;
}

/* the n_sym symbols of segment s (the format's symbol message) */
static uint64_t segment_symbols(const uint8_t *in, const geom_t *g, uint64_t s, const orc_cmd *c, uint64_t nc,
                                uint8_t *sym) {
  uint64_t q = 0;
  for (uint64_t i = 0; i < nc; ++i) { put_u16(sym + q, c[i].lit_len); q += 2; }
  for (uint64_t i = 0; i < nc; ++i) { put_u16(sym + q, c[i].mlen - g->min_match); q += 2; }
  for (uint64_t i = 0; i < nc; ++i)
    for (uint32_t b = 0; b < g->W; ++b) sym[q++] = (uint8_t)(c[i].src >> (8 * b));
  uint64_t p = s * g->S, seg_end = p + g->S < g->n ? p + g->S : g->n;
  for (uint64_t i = 0; i < nc; ++i) {
    for (uint32_t k = 0; k < c[i].lit_len; ++k) sym[q++] = in[p++];
    p += c[i].mlen;
  }
  while (p < seg_end) sym[q++] = in[p++];
  return q;
}

/* check one segment's commands against R-len / R-order / R-dist / R-sym */
static int check_commands(const geom_t *g, uint64_t s, const orc_cmd *c, uint64_t nc, uint64_t *n_lit_out) {
  uint64_t seg_start = s * g->S, seg_end = seg_start + g->S < g->n ? seg_start + g->S : g->n;
  uint64_t p = seg_start, n_lit = 0;
  for (uint64_t i = 0; i < nc; ++i) {
    if (c[i].mlen < g->min_match || c[i].lit_len >= 65536u || c[i].mlen - g->min_match >= 65536u) return ORC_ECORRUPT;
    p += c[i].lit_len;
    n_lit += c[i].lit_len;
    if (p > seg_end) return ORC_ECORRUPT;
    uint64_t dst = p;
    if (c[i].src + c[i].mlen > dst || c[i].src + c[i].mlen < c[i].src) return ORC_ECORRUPT;  /* R-order */
    if (g->D && dst - c[i].src > g->D) return ORC_ECORRUPT;                                 /* R-dist */
    p += c[i].mlen;
    if (p > seg_end) return ORC_ECORRUPT;                                                    /* R-len */
  }
  n_lit += seg_end - p;
  if (nc * (4 + (uint64_t)g->W) + n_lit > SYM_MAX) return ORC_ECORRUPT;                    /* R-sym */
  *n_lit_out = n_lit;
  return ORC_OK;
}

/* deps(s) (ascending, distinct, != s) into out; returns the count */
static uint64_t segment_deps(const geom_t *g, uint64_t s, const orc_cmd *c, uint64_t nc, uint8_t *mark,
                             uint64_t *out) {
  uint64_t k = 0;
  for (uint64_t i = 0; i < nc; ++i)
    for (uint64_t q = c[i].src >> g->log2_S; q <= (c[i].src + c[i].mlen - 1) >> g->log2_S; ++q)
      if (q != s && !mark[q]) { mark[q] = 1; out[k++] = q; }
  for (uint64_t i = 0; i < k; ++i) mark[out[i]] = 0;
  /* insertion sort: lists are short */
  for (uint64_t i = 1; i < k; ++i) {
    uint64_t v = out[i], j = i;
    while (j > 0 && out[j - 1] > v) { out[j] = out[j - 1]; --j; }
    out[j] = v;
  }
  return k;
}

/* rANS-encode one segment (the format's rANS encoder, run backwards over the
 * symbols); words land reversed in words[] */
static uint64_t rans_encode_segment(const uint8_t *sym, uint64_t n_sym, uint64_t nc, uint32_t W,
                                    const uint16_t freq[4][256], const uint32_t cum[4][257], uint32_t states[LANES],
                                    uint16_t *words) {
  uint32_t x[LANES];
  for (uint32_t j = 0; j < LANES; ++j) x[j] = RANS_L;
  uint64_t nw = 0;
  for (uint64_t q = n_sym; q-- > 0;) {
    uint32_t j = (uint32_t)(q % LANES);
    int c = sym_class(q, nc, W);
    uint32_t s = sym[q];
    uint32_t f = freq[c][s];
    if ((uint64_t)x[j] >= ((uint64_t)1 << 20) * f) {
      words[nw++] = (uint16_t)(x[j] & 0xFFFFu);
      x[j] >>= 16;
    }
    x[j] = (x[j] / f) * M_SCALE + (x[j] % f) + cum[c][s];
  }
  for (uint32_t j = 0; j < LANES; ++j) states[j] = x[j];
  /* reverse so the decoder reads forward */
  for (uint64_t i = 0; i < nw / 2; ++i) {
    uint16_t t = words[i];
    words[i] = words[nw - 1 - i];
    words[nw - 1 - i] = t;
  }
  return nw;
}

/*
 * Build an archive from explicit commands (the second half of the encoder;
 * the tests also feed it hand-made command lists). reads: optional record
 * offsets for the read index. The archive is malloc'd into *out; returns its
 * size or a negative error (-ORC_ECORRUPT for commands that break a rule).
 */
int64_t orc_serialize(const uint8_t *in, uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t max_level,
                      uint64_t D, const orc_cmd *cmds, const uint64_t *cmd_ptr, const uint64_t *reads,
                      uint64_t n_reads, uint8_t **out) {
  geom_t g;
  if (make_geom(n, log2_B, min_match, max_level, D, &g)) return -ORC_EINVAL;
  for (uint64_t r = 0; r < n_reads; ++r)
    if (reads[r] >= n || (r && reads[r] <= reads[r - 1])) return -ORC_EINVAL;
  uint64_t n_seg = g.n_seg;
  uint64_t *n_lit = (uint64_t *)malloc(sizeof(uint64_t) * (n_seg + 1));
  uint64_t *dep_ptr = (uint64_t *)malloc(sizeof(uint64_t) * (n_seg + 1));
  uint16_t *level = (uint16_t *)malloc(sizeof(uint16_t) * (n_seg + 1));
  uint8_t *mark = (uint8_t *)calloc(n_seg + 1, 1);
  uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (n_seg + 1));
  uint8_t *sym = (uint8_t *)malloc(SYM_MAX);
  uint16_t *words = (uint16_t *)malloc(sizeof(uint16_t) * SYM_MAX);
  uint32_t *states = (uint32_t *)malloc(sizeof(uint32_t) * LANES * (n_seg + 1));
  uint64_t *n_words = (uint64_t *)malloc(sizeof(uint64_t) * (n_seg + 1));
  uint64_t dep_cap = 1024, n_deps = 0;
  uint32_t *deps = (uint32_t *)malloc(sizeof(uint32_t) * dep_cap);
  uint8_t *arc = NULL;
  int64_t rc = 0;
  uint16_t **seg_words = (uint16_t **)calloc(n_seg + 1, sizeof(uint16_t *));
  if (!n_lit || !dep_ptr || !level || !mark || !tmp || !sym || !words || !states || !n_words || !deps || !seg_words) {
    rc = -ORC_ENOMEM;
    goto done;
  }
  /* pass 1: rules, deps, levels, symbol counts */
  uint64_t counts[4][256];
  memset(counts, 0, sizeof(counts));
  for (uint64_t s = 0; s < n_seg; ++s) {
    const orc_cmd *c = cmds + cmd_ptr[s];
    uint64_t nc = cmd_ptr[s + 1] - cmd_ptr[s];
    if (check_commands(&g, s, c, nc, &n_lit[s])) { rc = -ORC_ECORRUPT; goto done; }
    uint64_t k = segment_deps(&g, s, c, nc, mark, tmp);
    dep_ptr[s] = n_deps;
    uint32_t lv = 0;
    for (uint64_t i = 0; i < k; ++i) {
      if (n_deps == dep_cap) {
        dep_cap *= 2;
        uint32_t *nd = (uint32_t *)realloc(deps, sizeof(uint32_t) * dep_cap);
        if (!nd) { rc = -ORC_ENOMEM; goto done; }
        deps = nd;
      }
      deps[n_deps++] = (uint32_t)tmp[i];
      if (level[tmp[i]] + 1u > lv) lv = level[tmp[i]] + 1u;
    }
    if (lv > max_level) { rc = -ORC_ECORRUPT; goto done; }
    level[s] = (uint16_t)lv;
    uint64_t ns = segment_symbols(in, &g, s, c, nc, sym);
    for (uint64_t q = 0; q < ns; ++q) counts[sym_class(q, nc, g.W)][sym[q]]++;
  }
  dep_ptr[n_seg] = n_deps;
  uint16_t freq[4][256];
  uint32_t cum[4][257];
  for (int c = 0; c < 4; ++c) {
    orc_normalize(counts[c], freq[c]);
    cum[c][0] = 0;
    for (int s = 0; s < 256; ++s) cum[c][s + 1] = cum[c][s] + freq[c][s];
  }
  /* pass 2: rANS */
  uint64_t payload = 0;
  for (uint64_t s = 0; s < n_seg; ++s) {
    const orc_cmd *c = cmds + cmd_ptr[s];
    uint64_t nc = cmd_ptr[s + 1] - cmd_ptr[s];
    uint64_t ns = segment_symbols(in, &g, s, c, nc, sym);
    n_words[s] = rans_encode_segment(sym, ns, nc, g.W, (const uint16_t(*)[256])freq,
                                     (const uint32_t(*)[257])cum, states + LANES * s, words);
    seg_words[s] = (uint16_t *)malloc(sizeof(uint16_t) * (n_words[s] ? n_words[s] : 1));
    if (!seg_words[s]) { rc = -ORC_ENOMEM; goto done; }
    memcpy(seg_words[s], words, sizeof(uint16_t) * n_words[s]);
    payload = round16(payload + 128 + 2 * n_words[s]);
  }
  /* layout (the format's section layout) */
  uint64_t off_tables = 128, off_dir = off_tables + 2048;
  uint64_t off_dep_ptr = round16(off_dir + 24 * n_seg);
  uint64_t off_deps = round16(off_dep_ptr + 8 * (n_seg + 1));
  uint64_t off_reads = round16(off_deps + 4 * n_deps);
  uint64_t off_payload = round16(off_reads + 8 * n_reads);
  uint64_t total = off_payload + payload;
  arc = (uint8_t *)calloc(total, 1);
  if (!arc) { rc = -ORC_ENOMEM; goto done; }
  memcpy(arc, "ACEAPEX1", 8);
  put_u32(arc + 8, 1);
  put_u32(arc + 12, 128);
  put_u64(arc + 16, n);
  arc[24] = (uint8_t)g.log2_B;
  arc[25] = (uint8_t)g.log2_S;
  arc[26] = (uint8_t)g.W;
  arc[27] = (uint8_t)min_match;
  arc[28] = SCALE_BITS;
  arc[29] = LANES;
  arc[30] = (uint8_t)max_level;
  arc[31] = n_reads ? 1 : 0;
  put_u64(arc + 32, D);
  put_u64(arc + 40, n_seg);
  put_u64(arc + 48, n_deps);
  put_u64(arc + 56, n_reads);
  put_u64(arc + 64, off_tables);
  put_u64(arc + 72, off_dir);
  put_u64(arc + 80, off_dep_ptr);
  put_u64(arc + 88, off_deps);
  put_u64(arc + 96, off_reads);
  put_u64(arc + 104, off_payload);
  put_u64(arc + 112, payload);
  put_u64(arc + 120, total);
  for (int c = 0; c < 4; ++c)
    for (int s = 0; s < 256; ++s) put_u16(arc + off_tables + 512 * c + 2 * s, freq[c][s]);
  uint64_t po = 0;
  for (uint64_t s = 0; s < n_seg; ++s) {
    uint8_t *d = arc + off_dir + 24 * s;
    uint64_t nc = cmd_ptr[s + 1] - cmd_ptr[s];
    put_u64(d, po);
    put_u32(d + 8, (uint32_t)n_words[s]);
    put_u32(d + 12, (uint32_t)nc);
    put_u32(d + 16, (uint32_t)n_lit[s]);
    put_u16(d + 20, level[s]);
    uint8_t *pl = arc + off_payload + po;
    for (uint32_t j = 0; j < LANES; ++j) put_u32(pl + 4 * j, states[LANES * s + j]);
    for (uint64_t w = 0; w < n_words[s]; ++w) put_u16(pl + 128 + 2 * w, seg_words[s][w]);
    po = round16(po + 128 + 2 * n_words[s]);
  }
  for (uint64_t s = 0; s <= n_seg; ++s) put_u64(arc + off_dep_ptr + 8 * s, dep_ptr[s]);
  for (uint64_t i = 0; i < n_deps; ++i) put_u32(arc + off_deps + 4 * i, deps[i]);
  for (uint64_t r = 0; r < n_reads; ++r) put_u64(arc + off_reads + 8 * r, reads[r]);
  *out = arc;
  rc = (int64_t)total;
done:
  if (seg_words)
    for (uint64_t s = 0; s < n_seg; ++s) free(seg_words[s]);
  free(seg_words);
  free(n_lit); free(dep_ptr); free(level); free(mark); free(tmp); free(sym); free(words);
  free(states); free(n_words); free(deps);
  return rc;
}

/* parse + serialize */
int64_t orc_encode(const uint8_t *in, uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t max_level,
                   uint64_t D, uint32_t chain, const uint64_t *reads, uint64_t n_reads, uint8_t **out) {
  orc_cmd *cmds = NULL;
  uint64_t *cmd_ptr = NULL;
  int64_t k = orc_parse(in, n, log2_B, min_match, max_level, D, chain, &cmds, &cmd_ptr);
  if (k < 0) return k;
  int64_t rc = orc_serialize(in, n, log2_B, min_match, max_level, D, cmds, cmd_ptr, reads, n_reads, out);
  free(cmds);
  free(cmd_ptr);
  return rc;
}

/* ------------------------------------------------------- archive reading */

typedef struct {
  const uint8_t *a;
  uint64_t len;
  geom_t g;
  uint64_t n_deps, n_reads;
  uint64_t off_tables, off_dir, off_dep_ptr, off_deps, off_reads, off_payload, payload_bytes;
  uint16_t freq[4][256];
  uint32_t cum[4][257];
  uint8_t *lut[4];            /* slot -> symbol, 4096 entries per class */
} arc_t;

static void arc_release(arc_t *A) {
  for (int c = 0; c < 4; ++c) free(A->lut[c]);
}

/* header, tables, directory and dependency checks of the format (header, tables, directory, dependency lists) */
static int arc_open(const uint8_t *a, uint64_t len, arc_t *A) {
  memset(A, 0, sizeof(*A));
  A->a = a;
  A->len = len;
  if (len < 128 + 2048 || memcmp(a, "ACEAPEX1", 8) != 0) return ORC_ECORRUPT;
  if (get_u32(a + 8) != 1 || get_u32(a + 12) != 128) return ORC_ECORRUPT;
  uint64_t n = get_u64(a + 16);
  uint32_t log2_B = a[24], log2_S = a[25], W = a[26], min_match = a[27];
  if (a[28] != SCALE_BITS || a[29] != LANES || (a[31] & ~1u)) return ORC_ECORRUPT;
  if (make_geom(n, log2_B, min_match, a[30], get_u64(a + 32), &A->g)) return ORC_ECORRUPT;
  if (log2_S != A->g.log2_S || W != A->g.W) return ORC_ECORRUPT;
  if (get_u64(a + 40) != A->g.n_seg) return ORC_ECORRUPT;
  A->n_deps = get_u64(a + 48);
  A->n_reads = get_u64(a + 56);
  if (!(a[31] & 1u) && A->n_reads) return ORC_ECORRUPT;
  uint64_t n_seg = A->g.n_seg;
  if (n_seg > (len / 24) || A->n_deps > len / 4 || A->n_reads > len / 8) return ORC_ECORRUPT;
  A->off_tables = get_u64(a + 64);
  A->off_dir = get_u64(a + 72);
  A->off_dep_ptr = get_u64(a + 80);
  A->off_deps = get_u64(a + 88);
  A->off_reads = get_u64(a + 96);
  A->off_payload = get_u64(a + 104);
  A->payload_bytes = get_u64(a + 112);
  if (A->off_tables != 128 || A->off_dir != 128 + 2048 ||
      A->off_dep_ptr != round16(A->off_dir + 24 * n_seg) ||
      A->off_deps != round16(A->off_dep_ptr + 8 * (n_seg + 1)) ||
      A->off_reads != round16(A->off_deps + 4 * A->n_deps) ||
      A->off_payload != round16(A->off_reads + 8 * A->n_reads) ||
      get_u64(a + 120) != A->off_payload + A->payload_bytes || get_u64(a + 120) != len)
    return ORC_ECORRUPT;
  /* tables */
  for (int c = 0; c < 4; ++c) {
    uint32_t sum = 0;
    A->cum[c][0] = 0;
    for (int s = 0; s < 256; ++s) {
      A->freq[c][s] = (uint16_t)get_u16(a + A->off_tables + 512 * c + 2 * s);
      sum += A->freq[c][s];
      A->cum[c][s + 1] = sum;
    }
    if (sum != 0 && sum != M_SCALE) return ORC_ECORRUPT;
    A->lut[c] = (uint8_t *)calloc(M_SCALE, 1);
    if (!A->lut[c]) return ORC_ENOMEM;
    for (int s = 0; s < 256; ++s)
      for (uint32_t k = A->cum[c][s]; k < A->cum[c][s + 1]; ++k) A->lut[c][k] = (uint8_t)s;
  }
  /* directory: packed payloads, R-sym, levels */
  uint64_t po = 0;
  for (uint64_t s = 0; s < n_seg; ++s) {
    const uint8_t *d = a + A->off_dir + 24 * s;
    uint64_t nw = get_u32(d + 8), nc = get_u32(d + 12), nl = get_u32(d + 16);
    if (get_u64(d) != po || get_u16(d + 22) != 0) return ORC_ECORRUPT;
    if (nc * (4 + (uint64_t)W) + nl > SYM_MAX) return ORC_ECORRUPT;
    if (get_u16(d + 20) > A->g.max_level) return ORC_ECORRUPT;
    po = round16(po + 128 + 2 * nw);
  }
  if (po != A->payload_bytes) return ORC_ECORRUPT;
  /* dep_ptr / deps */
  if (get_u64(a + A->off_dep_ptr) != 0 || get_u64(a + A->off_dep_ptr + 8 * n_seg) != A->n_deps) return ORC_ECORRUPT;
  for (uint64_t s = 0; s < n_seg; ++s) {
    uint64_t b = get_u64(a + A->off_dep_ptr + 8 * s), e = get_u64(a + A->off_dep_ptr + 8 * (s + 1));
    if (e < b || e > A->n_deps) return ORC_ECORRUPT;
    for (uint64_t i = b; i < e; ++i) {
      uint32_t d = get_u32(a + A->off_deps + 4 * i);
      if (d >= s || (i > b && d <= get_u32(a + A->off_deps + 4 * (i - 1)))) return ORC_ECORRUPT;
    }
  }
  /* read index */
  for (uint64_t r = 0; r < A->n_reads; ++r) {
    uint64_t o = get_u64(a + A->off_reads + 8 * r);
    if (o >= n || (r && o <= get_u64(a + A->off_reads + 8 * (r - 1)))) return ORC_ECORRUPT;
  }
  return ORC_OK;
}

/*
 * rANS-decode the n_sym symbols of segment s (the format's rANS decoding rule),
 * checking the final-state invariant. final_states (optional) receives the
 * 32 lane states after the last symbol.
 */
static int decode_symbols(const arc_t *A, uint64_t s, uint8_t *sym, uint64_t *n_sym_out, orc_cmd *cmds,
                          uint64_t *nc_out, uint32_t *final_states) {
  const uint8_t *d = A->a + A->off_dir + 24 * s;
  uint64_t po = get_u64(d), nw = get_u32(d + 8), nc = get_u32(d + 12), nl = get_u32(d + 16);
  uint32_t W = A->g.W;
  uint64_t n_sym = nc * (4 + W) + nl;
  const uint8_t *pl = A->a + A->off_payload + po;
  uint32_t x[LANES];
  for (uint32_t j = 0; j < LANES; ++j) {
    x[j] = get_u32(pl + 4 * j);
    if (x[j] < RANS_L) return ORC_ECORRUPT;
  }
  const uint8_t *wp = pl + 128;
  uint64_t p = 0;
  for (uint64_t q = 0; q < n_sym; ++q) {
    uint32_t j = (uint32_t)(q % LANES);
    int c = sym_class(q, nc, W);
    if (A->cum[c][256] == 0) return ORC_ECORRUPT;   /* symbol of an unused class */
    uint32_t slot = x[j] % M_SCALE;
    uint32_t sy = A->lut[c][slot];
    x[j] = A->freq[c][sy] * (x[j] / M_SCALE) + slot - A->cum[c][sy];
    if (x[j] < RANS_L) {
      if (p >= nw) return ORC_ECORRUPT;
      x[j] = (x[j] << 16) | get_u16(wp + 2 * p);
      ++p;
    }
    sym[q] = (uint8_t)sy;
  }
  if (final_states)
    for (uint32_t j = 0; j < LANES; ++j) final_states[j] = x[j];
  for (uint32_t j = 0; j < LANES; ++j)
    if (x[j] != RANS_L) return ORC_ECORRUPT;
  if (p != nw) return ORC_ECORRUPT;
  /* commands from the first three classes */
  for (uint64_t i = 0; i < nc; ++i) {
    cmds[i].lit_len = get_u16(sym + 2 * i);
    cmds[i].mlen = get_u16(sym + 2 * nc + 2 * i) + A->g.min_match;
    uint64_t src = 0;
    for (uint32_t b = 0; b < W; ++b) src |= (uint64_t)sym[4 * nc + W * i + b] << (8 * b);
    cmds[i].src = src;
  }
  *n_sym_out = n_sym;
  *nc_out = nc;
  return ORC_OK;
}

/*
 * Decode segment s into the output view (buf indexed by absolute position &
 * mask): literals and matches in command order, byte by byte, after checking
 * the command rules and recomputing deps(s) and level(s) against the stored
 * ones. levels[] holds the stored levels of all segments.
 */
static int decode_segment(const arc_t *A, uint64_t s, uint8_t *buf, uint64_t mask, uint8_t *sym, orc_cmd *cmds,
                          uint8_t *mark, uint64_t *tmp) {
  uint64_t n_sym, nc;
  int rc = decode_symbols(A, s, sym, &n_sym, cmds, &nc, NULL);
  if (rc) return rc;
  uint64_t nl;
  if (check_commands(&A->g, s, cmds, nc, &nl)) return ORC_ECORRUPT;
  const uint8_t *d = A->a + A->off_dir + 24 * s;
  if (nl != get_u32(d + 16)) return ORC_ECORRUPT;
  /* recompute deps and level */
  uint64_t k = segment_deps(&A->g, s, cmds, nc, mark, tmp);
  uint64_t b = get_u64(A->a + A->off_dep_ptr + 8 * s), e = get_u64(A->a + A->off_dep_ptr + 8 * (s + 1));
  if (e - b != k) return ORC_ECORRUPT;
  uint32_t lv = 0;
  for (uint64_t i = 0; i < k; ++i) {
    if (get_u32(A->a + A->off_deps + 4 * (b + i)) != tmp[i]) return ORC_ECORRUPT;
    uint32_t l = get_u16(A->a + A->off_dir + 24 * tmp[i] + 20);
    if (l + 1 > lv) lv = l + 1;
  }
  if (lv != get_u16(d + 20)) return ORC_ECORRUPT;
  /* execute */
  uint64_t p = s * A->g.S, seg_end = p + A->g.S < A->g.n ? p + A->g.S : A->g.n;
  const uint8_t *lit = sym + nc * (4 + A->g.W);
  for (uint64_t i = 0; i < nc; ++i) {
    for (uint32_t t = 0; t < cmds[i].lit_len; ++t) buf[(p++) & mask] = *lit++;
    for (uint32_t t = 0; t < cmds[i].mlen; ++t, ++p) buf[p & mask] = buf[(cmds[i].src + t) & mask];
  }
  while (p < seg_end) buf[(p++) & mask] = *lit++;
  return ORC_OK;
}

typedef struct {
  uint8_t *sym;
  orc_cmd *cmds;
  uint8_t *mark;
  uint64_t *tmp;
} scratch_t;

static int scratch_new(scratch_t *w, uint64_t n_seg) {
  w->sym = (uint8_t *)malloc(SYM_MAX);
  w->cmds = (orc_cmd *)malloc(sizeof(orc_cmd) * SYM_MAX);
  w->mark = (uint8_t *)calloc(n_seg + 1, 1);
  w->tmp = (uint64_t *)malloc(sizeof(uint64_t) * (n_seg + 1));
  return (w->sym && w->cmds && w->mark && w->tmp) ? ORC_OK : ORC_ENOMEM;
}

static void scratch_free(scratch_t *w) { free(w->sym); free(w->cmds); free(w->mark); free(w->tmp); }

/* Full sequential decode into out[0..N); returns an ORC_* status. */
int orc_decode(const uint8_t *a, uint64_t len, uint8_t *out, uint64_t cap) {
  arc_t A;
  int rc = arc_open(a, len, &A);
  if (rc) { arc_release(&A); return rc; }
  if (cap < A.g.n) { arc_release(&A); return ORC_ERANGE; }
  scratch_t w;
  rc = scratch_new(&w, A.g.n_seg);
  for (uint64_t s = 0; rc == ORC_OK && s < A.g.n_seg; ++s) rc = decode_segment(&A, s, out, ~(uint64_t)0, w.sym, w.cmds, w.mark, w.tmp);
  scratch_free(&w);
  arc_release(&A);
  return rc;
}

/*
 * Streaming decode of [lo, hi) with one CRC-32 per window of `window` bytes
 * (window k = [lo + k*window, min(hi, lo + (k+1)*window))). Segments are
 * decoded in order from segment 0 into a ring of 2^k >= D + S bytes when the
 * archive has a distance bound D, else into a buffer of N bytes.
 */
int orc_decode_stream(const uint8_t *a, uint64_t len, uint64_t lo, uint64_t hi, uint64_t window, uint32_t *crcs,
                      uint64_t n_windows) {
  arc_t A;
  int rc = arc_open(a, len, &A);
  if (rc) { arc_release(&A); return rc; }
  if (lo > hi || hi > A.g.n || window == 0 || n_windows < (hi - lo + window - 1) / window) {
    arc_release(&A);
    return ORC_EINVAL;
  }
  uint64_t ring = A.g.n ? A.g.n : 1, mask = ~(uint64_t)0;
  if (A.g.D) {
    ring = 1;
    while (ring < A.g.D + A.g.S) ring <<= 1;
    mask = ring - 1;
  }
  uint8_t *buf = (uint8_t *)malloc(ring);
  scratch_t w;
  rc = buf ? scratch_new(&w, A.g.n_seg) : ORC_ENOMEM;
  for (uint64_t k = 0; k * window < hi - lo; ++k) crcs[k] = 0;
  uint64_t s_end = hi ? ((hi - 1) >> A.g.log2_S) + 1 : 0;
  for (uint64_t s = 0; rc == ORC_OK && s < s_end; ++s) {
    rc = decode_segment(&A, s, buf, mask, w.sym, w.cmds, w.mark, w.tmp);
    if (rc) break;
    uint64_t b = s * A.g.S, e = b + A.g.S < A.g.n ? b + A.g.S : A.g.n;
    if (b < lo) b = lo;
    if (e > hi) e = hi;
    /* a segment is contiguous in the ring (the ring is a multiple of S) */
    while (b < e) {
      uint64_t k = (b - lo) / window, we = lo + (k + 1) * window;
      if (we > e) we = e;
      crcs[k] = orc_crc32(crcs[k], buf + (b & mask), we - b);
      b = we;
    }
  }
  if (buf) scratch_free(&w);
  free(buf);
  arc_release(&A);
  return rc;
}

/* ---------------------------------------------------------- inspection */

typedef struct {
  uint64_t n, n_segments, n_blocks, n_deps, n_reads, D, payload_bytes, total_bytes;
  uint32_t log2_B, log2_S, W, min_match, max_level;
} orc_info_t;

int orc_info(const uint8_t *a, uint64_t len, orc_info_t *info) {
  arc_t A;
  int rc = arc_open(a, len, &A);
  if (rc == ORC_OK) {
    info->n = A.g.n;
    info->n_segments = A.g.n_seg;
    info->n_blocks = (A.g.n + ((uint64_t)1 << A.g.log2_B) - 1) >> A.g.log2_B;
    info->n_deps = A.n_deps;
    info->n_reads = A.n_reads;
    info->D = A.g.D;
    info->payload_bytes = A.payload_bytes;
    info->total_bytes = len;
    info->log2_B = A.g.log2_B;
    info->log2_S = A.g.log2_S;
    info->W = A.g.W;
    info->min_match = A.g.min_match;
    info->max_level = A.g.max_level;
  }
  arc_release(&A);
  return rc;
}

/*
 * Commands, symbols and final lane states of one segment, for the invariant
 * tests. cmds needs room for SYM_MAX entries, sym for SYM_MAX bytes. The
 * final-state check is not applied here: the states are returned as found.
 */
int orc_segment_info(const uint8_t *a, uint64_t len, uint64_t s, orc_cmd *cmds, uint64_t *n_cmd, uint8_t *sym,
                     uint64_t *n_sym, uint32_t *final_states) {
  arc_t A;
  int rc = arc_open(a, len, &A);
  if (rc == ORC_OK && s >= A.g.n_seg) rc = ORC_EINVAL;
  if (rc == ORC_OK) {
    rc = decode_symbols(&A, s, sym, n_sym, cmds, n_cmd, final_states);
    if (rc == ORC_ECORRUPT) {
      /* report what was decoded even when the final state is off */
      const uint8_t *d = a + A.off_dir + 24 * s;
      *n_cmd = get_u32(d + 12);
      *n_sym = *n_cmd * (4 + A.g.W) + get_u32(d + 16);
    }
  }
  arc_release(&A);
  return rc;
}

/*
 * Offsets of the FASTQ records of in[0..n): a record is four lines, so every
 * line whose index is a multiple of four starts one (paper §4.1 read index).
 */
uint64_t orc_fastq_record_starts(const uint8_t *in, uint64_t n, uint64_t *out, uint64_t cap) {
  uint64_t line = 0, k = 0;
  int at_line_start = 1;
  for (uint64_t p = 0; p < n; ++p) {
    if (at_line_start) {
      if (line % 4 == 0) {
        if (k < cap) out[k] = p;
        ++k;
      }
      at_line_start = 0;
    }
    if (in[p] == '\n') { ++line; at_line_start = 1; }
  }
  return k;
}

/* ---------------------------------------------- all-core CPU baseline */

typedef struct {
  const arc_t *A;
  uint8_t *out;
  const uint64_t *segs; /* the segments of the current level */
  uint64_t n;
  uint64_t next;        /* next index into segs (taken under mu) */
  int rc;
  pthread_mutex_t mu;
} wave_t;

static void *wave_worker(void *arg) {
  wave_t *W = (wave_t *)arg;
  scratch_t w;
  int rc = scratch_new(&w, W->A->g.n_seg);
  for (;;) {
    pthread_mutex_lock(&W->mu);
    if (rc && !W->rc) W->rc = rc;
    const uint64_t i = W->rc ? W->n : W->next++;
    pthread_mutex_unlock(&W->mu);
    if (i >= W->n) break;
    rc = decode_segment(W->A, W->segs[i], W->out, ~(uint64_t)0, w.sym, w.cmds, w.mark, w.tmp);
  }
  scratch_free(&w);
  return NULL;
}

/*
 * Decode into out[0..N) on `threads` host threads: every segment of level L
 * reads only segments of lower levels, so the segments of one level decode
 * in any order once the lower levels are done. Returns an ORC_* status.
 */
int orc_decode_wavefront(const uint8_t *a, uint64_t len, uint8_t *out, uint64_t cap, int threads) {
  arc_t A;
  int rc = arc_open(a, len, &A);
  if (rc) { arc_release(&A); return rc; }
  if (cap < A.g.n) { arc_release(&A); return ORC_ERANGE; }
  if (threads < 1) threads = 1;
  uint64_t *segs = (uint64_t *)malloc(sizeof(uint64_t) * (A.g.n_seg + 1));
  pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
  if (!segs || !tid) { free(segs); free(tid); arc_release(&A); return ORC_ENOMEM; }
  uint32_t max_level = 0;
  for (uint64_t s = 0; s < A.g.n_seg; ++s) {
    uint32_t l = get_u16(A.a + A.off_dir + 24 * s + 20);
    if (l > max_level) max_level = l;
  }
  wave_t W;
  W.A = &A;
  W.out = out;
  W.segs = segs;
  W.rc = ORC_OK;
  pthread_mutex_init(&W.mu, NULL);
  for (uint32_t L = 0; L <= max_level && W.rc == ORC_OK; ++L) {
    uint64_t n = 0;
    for (uint64_t s = 0; s < A.g.n_seg; ++s)
      if (get_u16(A.a + A.off_dir + 24 * s + 20) == L) segs[n++] = s;
    W.n = n;
    W.next = 0;
    for (int t = 0; t < threads; ++t) pthread_create(&tid[t], NULL, wave_worker, &W);
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  }
  rc = W.rc;
  pthread_mutex_destroy(&W.mu);
  free(segs);
  free(tid);
  arc_release(&A);
  return rc;
}
