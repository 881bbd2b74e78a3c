/*
 * Seeded synthetic genomic inputs (FASTQ reads, FASTA genomes).
 *
 * This module holds no codec arithmetic: it only produces the decompressed
 * bytes that the encoders take as input. Both the CPU oracle's tests and the
 * GPU library's tests and benchmark draw their inputs from it, so it is kept
 * in a module of its own. Each generator states its recipe where it is defined.
 *
 * Randomness: SplitMix64 expands a (seed_a, seed_b) pair into the 256-bit
 * state of xoshiro256** (Blackman & Vigna, "Scrambled linear pseudorandom
 * number generators", 2018). Normal variates use the Irwin-Hall sum of twelve
 * 16-bit uniforms in integer fixed point, so quality strings are bit-identical
 * on every host. Log-uniform draws use exp2() from the C library.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ PRNG */

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static void rng_seed(rng_t *r, uint64_t a, uint64_t b) {
  uint64_t x = (a << 32) ^ b ^ 0x5EEDC0DEull;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t *r) {
  uint64_t *s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl(s[3], 45);
  return result;
}

/* uniform integer in [0, n), n >= 1 (multiply-shift; bias < 2^-32 for n < 2^32) */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

/* true with probability ppm / 1e6 */
static inline int rng_ppm(rng_t *r, uint32_t ppm) { return rng_below(r, 1000000) < ppm; }

/* uniform double in [0,1) with 53 bits */
static inline double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* floor(lo * (hi/lo)^u), u uniform in [0,1) */
static uint64_t rng_loguniform(rng_t *r, double lo, double hi) {
  double u = rng_unit(r);
  double v = lo * exp2(u * log2(hi / lo));
  uint64_t o = (uint64_t)v;
  if (o < (uint64_t)lo) o = (uint64_t)lo;
  return o;
}

/* Irwin-Hall(12) - 6 in units of 2^-16: approx N(0,1) * 65536 */
static inline int64_t rng_normal16(rng_t *r) {
  int64_t s = 0;
  for (int k = 0; k < 3; ++k) {
    uint64_t v = rng_next(r);
    s += (int64_t)(v & 0xFFFF) + (int64_t)((v >> 16) & 0xFFFF) + (int64_t)((v >> 32) & 0xFFFF) +
         (int64_t)(v >> 48);
  }
  return s - 6 * 65536;
}

static inline int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

static inline int base_idx(uint8_t b) { return b == 'A' ? 0 : b == 'C' ? 1 : b == 'G' ? 2 : 3; }

/* ------------------------------------------------------- reference + repeats */

/*
 * Random ACGT reference of ref_len bases. When repeat_ppm > 0, n_fam repeat
 * families (lengths log-uniform in [300, 6000]) are pasted as copies diverged
 * 5-20% (substitutions) at uniform positions until repeat_ppm/1e6 of the
 * reference is covered.
 */
int synth_reference(uint64_t seed_a, uint64_t seed_b, uint64_t ref_len, uint32_t repeat_ppm,
                    uint32_t n_fam, uint8_t *out) {
  rng_t r;
  rng_seed(&r, seed_a, seed_b);
  for (uint64_t i = 0; i < ref_len; ++i) out[i] = (uint8_t)BASES[rng_next(&r) >> 62];
  if (repeat_ppm == 0 || n_fam == 0 || ref_len < 6000) return 0;
  uint64_t *flen = (uint64_t *)malloc(sizeof(uint64_t) * n_fam);
  uint8_t **fam = (uint8_t **)malloc(sizeof(uint8_t *) * n_fam);
  if (!flen || !fam) { free(flen); free(fam); return -1; }
  for (uint32_t f = 0; f < n_fam; ++f) {
    flen[f] = rng_loguniform(&r, 300.0, 6000.0);
    fam[f] = (uint8_t *)malloc(flen[f]);
    if (!fam[f]) return -1;
    for (uint64_t i = 0; i < flen[f]; ++i) fam[f][i] = (uint8_t)BASES[rng_next(&r) >> 62];
  }
  uint64_t target = (uint64_t)(((unsigned __int128)ref_len * repeat_ppm) / 1000000u), covered = 0;
  while (covered < target) {
    uint32_t f = (uint32_t)rng_below(&r, n_fam);
    uint64_t len = flen[f];
    if (len >= ref_len) break;
    uint64_t pos = rng_below(&r, ref_len - len);
    uint32_t div_ppm = 50000 + (uint32_t)rng_below(&r, 150001); /* 5% .. 20% */
    for (uint64_t i = 0; i < len; ++i) {
      uint8_t b = fam[f][i];
      if (rng_ppm(&r, div_ppm)) {
        int k = (int)(base_idx(b) + 1 + rng_below(&r, 3)) & 3;
        b = (uint8_t)BASES[k];
      }
      out[pos + i] = b;
    }
    covered += len;
  }
  for (uint32_t f = 0; f < n_fam; ++f) free(fam[f]);
  free(fam);
  free(flen);
  return 0;
}

/* ------------------------------------------------------------------ FASTQ */

static inline uint8_t comp(uint8_t b) {
  switch (b) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    default: return 'A';
  }
}

/* copy n bases of src (reverse-complemented if rc) with 1% substitutions */
static void read_seq(rng_t *sub, const uint8_t *src, uint64_t n, int rc, uint8_t *dst) {
  for (uint64_t i = 0; i < n; ++i) {
    uint8_t b = rc ? comp(src[n - 1 - i]) : src[i];
    if (rng_ppm(sub, 10000)) {
      int k = (int)(base_idx(b) + 1 + rng_below(sub, 3)) & 3;
      b = (uint8_t)BASES[k];
    }
    dst[i] = b;
  }
}

/* Phred+33 string: mean 38 - 6p/len, sd 2.5, clamp [2,41]; 3% tail U{2..20} */
static void read_qual(rng_t *r, uint64_t n, uint8_t *dst) {
  for (uint64_t p = 0; p < n; ++p) {
    int64_t q;
    if (rng_ppm(r, 30000)) {
      q = 2 + (int64_t)rng_below(r, 19);
    } else {
      int64_t z = rng_normal16(r);                          /* N(0,1) * 2^16 */
      int64_t v = 38 * 65536 - floor_div(6 * (int64_t)p * 65536, (int64_t)n) + floor_div(5 * z, 2);
      q = floor_div(v + 32768, 65536);
      if (q < 2) q = 2;
      if (q > 41) q = 41;
    }
    dst[p] = (uint8_t)(q + 33);
  }
}

static uint64_t put_record(uint8_t *out, uint64_t cap, uint64_t at, uint64_t ordinal, int mate,
                           const uint8_t *seq, const uint8_t *qual, uint64_t rl) {
  char hdr[96];
  uint64_t tile = 1 + ordinal / 1000000, x = 1 + (ordinal / 1000) % 1000, y = 1 + ordinal % 1000;
  /* manual formatting: "@SIM:1:FC1:1:<tile>:<x>:<y> <mate>:N:0:ACGTAC\n" */
  char num[3][24];
  uint64_t v[3] = {tile, x, y};
  for (int k = 0; k < 3; ++k) {
    char t[24];
    int n = 0;
    uint64_t u = v[k];
    do { t[n++] = (char)('0' + u % 10); u /= 10; } while (u);
    for (int i = 0; i < n; ++i) num[k][i] = t[n - 1 - i];
    num[k][n] = 0;
  }
  size_t h = 0;
  const char *pre = "@SIM:1:FC1:1:";
  memcpy(hdr + h, pre, 13); h += 13;
  for (int k = 0; k < 3; ++k) {
    size_t l = strlen(num[k]);
    memcpy(hdr + h, num[k], l); h += l;
    hdr[h++] = (k < 2) ? ':' : ' ';
  }
  hdr[h++] = (char)('0' + mate);
  memcpy(hdr + h, ":N:0:ACGTAC\n", 12); h += 12;
  uint64_t need = h + rl + 1 + 2 + rl + 1;
  if (at + need > cap) return 0;
  uint8_t *o = out + at;
  memcpy(o, hdr, h); o += h;
  memcpy(o, seq, rl); o += rl; *o++ = '\n';
  *o++ = '+'; *o++ = '\n';
  memcpy(o, qual, rl); o += rl; *o++ = '\n';
  return need;
}

typedef struct { uint64_t start, frag; uint64_t sub_seed; } read_src;

/*
 * FASTQ reads sampled from ref. Single-end (paired = 0) or interleaved
 * paired-end (paired = 1; R2 is the reverse complement of the fragment end,
 * fragment length ~ N(350, 50) clamped to >= 150). Records are added while
 * they fit in max_bytes and fewer than max_units reads (SE) or pairs (PE)
 * were written. With truncate = 1 the output is filled to exactly max_bytes,
 * cutting the last record. 10% of reads (pairs) repeat the sequence of a
 * uniformly chosen earlier read (pair) with fresh qualities. Returns the byte
 * count, or -1 on allocation failure. *n_units gets the number of reads
 * (SE) or pairs (PE) started.
 */
int64_t synth_fastq(const uint8_t *ref, uint64_t ref_len, uint64_t seed_a, uint64_t seed_b,
                    int paired, int read_len, uint64_t max_bytes, uint64_t max_units, int truncate,
                    uint8_t *out, uint64_t *n_units) {
  rng_t r;
  rng_seed(&r, seed_a ^ 0xFA57Full, seed_b);
  uint64_t rl = (uint64_t)read_len;
  uint64_t cap_units = max_units ? max_units : (max_bytes / (2 * rl) + 2);
  read_src *hist = (read_src *)malloc(sizeof(read_src) * (cap_units + 1));
  uint8_t *seq = (uint8_t *)malloc(rl), *qual = (uint8_t *)malloc(rl);
  uint8_t *tmp = (uint8_t *)malloc(4 * rl + 256);
  if (!hist || !seq || !qual || !tmp) { free(hist); free(seq); free(qual); free(tmp); return -1; }
  uint64_t at = 0, i = 0;
  for (; i < cap_units; ++i) {
    read_src rs;
    if (i > 0 && rng_ppm(&r, 100000)) {
      rs = hist[rng_below(&r, i)];
    } else {
      uint64_t frag = rl;
      if (paired) {
        int64_t f = 350 + floor_div(50 * rng_normal16(&r), 65536);
        if (f < (int64_t)rl) f = (int64_t)rl;
        if ((uint64_t)f > ref_len) f = (int64_t)ref_len;
        frag = (uint64_t)f;
      }
      rs.frag = frag;
      rs.start = rng_below(&r, ref_len - frag + 1);
      rs.sub_seed = rng_next(&r);
    }
    hist[i] = rs;
    rng_t sub;
    rng_seed(&sub, rs.sub_seed, 0x5B5);
    int mates = paired ? 2 : 1;
    uint64_t at0 = at;
    int full = 1;
    for (int m = 0; m < mates; ++m) {
      if (m == 0) read_seq(&sub, ref + rs.start, rl, 0, seq);
      else read_seq(&sub, ref + rs.start + rs.frag - rl, rl, 1, seq);
      read_qual(&r, rl, qual);
      uint64_t w = put_record(out, max_bytes, at, i, paired ? m + 1 : 1, seq, qual, rl);
      if (w == 0) {
        full = 0;
        if (truncate) {
          /* write the partial record into tmp, then cut at max_bytes */
          uint64_t w2 = put_record(tmp, 4 * rl + 256, 0, i, paired ? m + 1 : 1, seq, qual, rl);
          uint64_t room = max_bytes - at;
          memcpy(out + at, tmp, room < w2 ? room : w2);
          at = max_bytes;
        }
        break;
      }
      at += w;
    }
    if (!full) {
      if (!truncate) at = at0; /* drop a partial pair */
      else ++i;
      break;
    }
  }
  if (n_units) *n_units = i;
  free(hist); free(seq); free(qual); free(tmp);
  return (int64_t)at;
}

/* ------------------------------------------------------------------ FASTA */

/*
 * FASTA genome of exactly total_bytes bytes: n_chrom records ">chrK\n" +
 * 60-column lines (a newline after every full line and after the last bases
 * of a chromosome). Chromosome lengths are 2.5e9 - s(2.5e9 - u_k), u_k ~
 * U[0.5e9, 2.5e9], with s fitted so the file totals total_bytes (u_k scaled
 * proportionally when the fit leaves [0, 1]); the last chromosome runs until
 * the file reaches total_bytes. Sequence: uppercase unique stretches
 * alternate with lowercase copies of 500 repeat families (diverged 5-20%,
 * 1% indels), about 45% of bases in repeats; each chromosome holds Poisson(4)
 * runs of 'N' of log-uniform length in [1e4, 3e6].
 *
 * Randomness: one stream draws the families and lengths; chromosome k has a
 * stream of its own (seed_b + 1 + k), so chromosomes can be generated in
 * parallel and the streaming reader yields the same bytes.
 */
#define FA_MAX_CHROM 64
#define FA_NFAM 500
#define FA_MAX_NRUN 32

typedef struct {
  uint64_t total;
  int n_chrom;
  uint64_t clen[FA_MAX_CHROM];   /* bases per chromosome (last: unbounded) */
  uint64_t cbytes[FA_MAX_CHROM]; /* bytes per chromosome record (last: rest of the file) */
  uint64_t coff[FA_MAX_CHROM];   /* byte offset of each record */
  uint8_t *fam[FA_NFAM];
  uint32_t flen[FA_NFAM];
  uint64_t seed_a, seed_b;
} fa_spec_t;

typedef struct {
  const fa_spec_t *sp;
  rng_t r;
  int k;
  uint64_t pos, emitted, limit; /* bases emitted, bytes emitted, byte limit of this record */
  int col;
  char hdr[32];
  int hdr_len, hdr_at;
  uint64_t nrun_start[FA_MAX_NRUN], nrun_len[FA_MAX_NRUN];
  int n_nrun, nrun_at;
  int feat; /* 0 unique, 1 repeat copy, 2 N run */
  uint64_t feat_left;
  uint32_t rep_fam, rep_at, rep_div_ppm;
  int ended;
} fa_chrom_t;

static uint64_t fa_record_bytes(int k, uint64_t L) {
  uint64_t h = (k + 1 < 10) ? 6 : 7;
  return h + L + (L + 59) / 60;
}

static void fa_chrom_init(fa_chrom_t *c, const fa_spec_t *sp, int k) {
  memset(c, 0, sizeof(*c));
  c->sp = sp;
  c->k = k;
  rng_seed(&c->r, sp->seed_a ^ 0xFA5Aull, sp->seed_b + 1 + (uint64_t)k);
  c->limit = sp->cbytes[k];
  int n = 0;
  c->hdr[n++] = '>'; c->hdr[n++] = 'c'; c->hdr[n++] = 'h'; c->hdr[n++] = 'r';
  char t[16];
  int m = 0, v = k + 1;
  do { t[m++] = (char)('0' + v % 10); v /= 10; } while (v);
  while (m) c->hdr[n++] = t[--m];
  c->hdr[n++] = '\n';
  c->hdr_len = n;
  /* N runs: Poisson(4) count, uniform starts, log-uniform lengths */
  double lim = exp(-4.0), p = 1.0;
  int cnt = 0;
  for (;;) { p *= rng_unit(&c->r); if (p <= lim) break; ++cnt; }
  if (cnt > FA_MAX_NRUN) cnt = FA_MAX_NRUN;
  uint64_t L = sp->clen[k];
  uint64_t span = (k == sp->n_chrom - 1) ? (sp->cbytes[k] * 60 / 61) : L;
  for (int i = 0; i < cnt; ++i) {
    c->nrun_start[i] = span ? rng_below(&c->r, span) : 0;
    c->nrun_len[i] = rng_loguniform(&c->r, 1e4, 3e6);
  }
  for (int i = 1; i < cnt; ++i) {
    uint64_t s0 = c->nrun_start[i], l0 = c->nrun_len[i];
    int j = i - 1;
    while (j >= 0 && c->nrun_start[j] > s0) { c->nrun_start[j + 1] = c->nrun_start[j]; c->nrun_len[j + 1] = c->nrun_len[j]; --j; }
    c->nrun_start[j + 1] = s0; c->nrun_len[j + 1] = l0;
  }
  c->n_nrun = cnt;
  c->feat = 0;
  c->feat_left = 1 + rng_below(&c->r, 2 * 2326);
}

/* pick the next feature: a due N run, else a repeat copy after a unique
 * stretch and a unique stretch after anything else (mean unique length 2326
 * against a mean repeat length of ~1900 gives a ~45% repeat share) */
static void fa_next_feature(fa_chrom_t *c, int after_unique) {
  if (c->nrun_at < c->n_nrun && c->nrun_start[c->nrun_at] <= c->pos) {
    c->feat = 2;
    c->feat_left = c->nrun_len[c->nrun_at++];
    return;
  }
  if (after_unique) {
    c->feat = 1;
    c->rep_fam = (uint32_t)rng_below(&c->r, FA_NFAM);
    c->rep_at = 0;
    c->rep_div_ppm = 50000 + (uint32_t)rng_below(&c->r, 150001);
    return;
  }
  c->feat = 0;
  c->feat_left = 1 + rng_below(&c->r, 2 * 2326);
}

static uint8_t fa_base(fa_chrom_t *c) {
  const fa_spec_t *sp = c->sp;
  for (;;) {
    if (c->feat == 2) {
      if (c->feat_left) { --c->feat_left; return 'N'; }
      fa_next_feature(c, 0);
      continue;
    }
    if (c->feat == 1) {
      uint32_t f = c->rep_fam;
      if (c->rep_at >= sp->flen[f]) { fa_next_feature(c, 0); continue; }
      uint64_t u = rng_below(&c->r, 1000000);
      if (u < 5000) { ++c->rep_at; continue; }                            /* deletion */
      if (u < 10000) return (uint8_t)(BASES[rng_next(&c->r) >> 62] | 0x20); /* insertion */
      uint8_t b = sp->fam[f][c->rep_at++];
      if (u < 10000 + c->rep_div_ppm) {
        int k = (int)(base_idx(b) + 1 + rng_below(&c->r, 3)) & 3;
        b = (uint8_t)BASES[k];
      }
      return (uint8_t)(b | 0x20);
    }
    if (c->nrun_at < c->n_nrun && c->nrun_start[c->nrun_at] <= c->pos) { fa_next_feature(c, 0); continue; }
    if (c->feat_left == 0) { fa_next_feature(c, 1); continue; }
    --c->feat_left;
    return (uint8_t)BASES[rng_next(&c->r) >> 62];
  }
}

/* next n bytes of chromosome record c (fewer at its end) */
static uint64_t fa_chrom_read(fa_chrom_t *c, uint8_t *out, uint64_t n) {
  uint64_t w = 0;
  const uint64_t L = c->sp->clen[c->k];
  while (w < n && c->emitted < c->limit) {
    if (c->hdr_at < c->hdr_len) { out[w++] = (uint8_t)c->hdr[c->hdr_at++]; ++c->emitted; continue; }
    if (c->col == 60 || (c->pos == L && c->col > 0)) {
      out[w++] = '\n'; ++c->emitted; c->col = 0;
      continue;
    }
    out[w++] = fa_base(c); ++c->emitted;
    ++c->col; ++c->pos;
  }
  return w;
}

static fa_spec_t *fa_spec_new(uint64_t seed_a, uint64_t seed_b, uint64_t total_bytes, int n_chrom) {
  if (n_chrom < 1 || n_chrom > FA_MAX_CHROM) return NULL;
  fa_spec_t *sp = (fa_spec_t *)calloc(1, sizeof(fa_spec_t));
  if (!sp) return NULL;
  rng_t r;
  rng_seed(&r, seed_a ^ 0xFA5Aull, seed_b);
  sp->total = total_bytes;
  sp->n_chrom = n_chrom;
  sp->seed_a = seed_a;
  sp->seed_b = seed_b;
  for (int f = 0; f < FA_NFAM; ++f) {
    sp->flen[f] = (uint32_t)rng_loguniform(&r, 300.0, 6000.0);
    sp->fam[f] = (uint8_t *)malloc(sp->flen[f]);
    for (uint32_t i = 0; i < sp->flen[f]; ++i) sp->fam[f][i] = (uint8_t)BASES[rng_next(&r) >> 62];
  }
  double u[FA_MAX_CHROM], su = 0;
  for (int k = 0; k < n_chrom; ++k) { u[k] = 0.5e9 + 2.0e9 * rng_unit(&r); su += u[k]; }
  double hdr = 0;
  for (int k = 0; k < n_chrom; ++k) hdr += (k + 1 < 10) ? 6 : 7;
  double bases = ((double)total_bytes - hdr) * 60.0 / 61.0;
  if (bases < n_chrom) bases = n_chrom;
  double top = 2.5e9 * n_chrom, gap = top - su;
  double s = gap > 0 ? (top - bases) / gap : -1;
  uint64_t off = 0;
  for (int k = 0; k < n_chrom; ++k) {
    double L = (s >= 0 && s <= 1) ? 2.5e9 - s * (2.5e9 - u[k]) : u[k] * (bases / su);
    sp->clen[k] = L < 1 ? 1 : (uint64_t)L;
    sp->coff[k] = off;
    uint64_t b = fa_record_bytes(k, sp->clen[k]);
    if (k == n_chrom - 1 || off + b >= total_bytes) {
      /* this record runs to the end of the file */
      sp->cbytes[k] = total_bytes > off ? total_bytes - off : 0;
      sp->clen[k] = UINT64_MAX / 4;
      sp->n_chrom = k + 1;
      break;
    }
    sp->cbytes[k] = b;
    off += b;
  }
  return sp;
}

static void fa_spec_free(fa_spec_t *sp) {
  if (!sp) return;
  for (int f = 0; f < FA_NFAM; ++f) free(sp->fam[f]);
  free(sp);
}

typedef struct {
  fa_spec_t *sp;
  fa_chrom_t c;
  int k;
  uint64_t emitted;
} fasta_t;

void *synth_fasta_new(uint64_t seed_a, uint64_t seed_b, uint64_t total_bytes, int n_chrom) {
  fasta_t *g = (fasta_t *)calloc(1, sizeof(fasta_t));
  if (!g) return NULL;
  g->sp = fa_spec_new(seed_a, seed_b, total_bytes, n_chrom);
  if (!g->sp) { free(g); return NULL; }
  g->k = 0;
  fa_chrom_init(&g->c, g->sp, 0);
  return g;
}

void synth_fasta_free(void *p) {
  fasta_t *g = (fasta_t *)p;
  if (!g) return;
  fa_spec_free(g->sp);
  free(g);
}

/* write the next n bytes of the stream (fewer at the end); returns the count */
uint64_t synth_fasta_read(void *p, uint8_t *out, uint64_t n) {
  fasta_t *g = (fasta_t *)p;
  uint64_t w = 0;
  while (w < n && g->k < g->sp->n_chrom) {
    uint64_t got = fa_chrom_read(&g->c, out + w, n - w);
    w += got;
    g->emitted += got;
    if (g->c.emitted >= g->c.limit) {
      if (++g->k < g->sp->n_chrom) fa_chrom_init(&g->c, g->sp, g->k);
    }
  }
  return w;
}

uint64_t synth_fasta_emitted(void *p) { return ((fasta_t *)p)->emitted; }

typedef struct {
  const fa_spec_t *sp;
  uint8_t *out;
  int next;
  pthread_mutex_t mu;
} fa_fill_t;

static void *fa_fill_worker(void *arg) {
  fa_fill_t *F = (fa_fill_t *)arg;
  for (;;) {
    pthread_mutex_lock(&F->mu);
    int k = F->next++;
    pthread_mutex_unlock(&F->mu);
    if (k >= F->sp->n_chrom) break;
    fa_chrom_t c;
    fa_chrom_init(&c, F->sp, k);
    fa_chrom_read(&c, F->out + F->sp->coff[k], F->sp->cbytes[k]);
  }
  return NULL;
}

/* the whole file into out[0..total_bytes), chromosomes generated by up to
 * `threads` threads (same bytes as the streaming reader) */
int synth_fasta_fill(uint64_t seed_a, uint64_t seed_b, uint64_t total_bytes, int n_chrom, int threads, uint8_t *out) {
  fa_spec_t *sp = fa_spec_new(seed_a, seed_b, total_bytes, n_chrom);
  if (!sp) return -1;
  fa_fill_t F;
  F.sp = sp;
  F.out = out;
  F.next = 0;
  pthread_mutex_init(&F.mu, NULL);
  if (threads < 1) threads = 1;
  if (threads > 64) threads = 64;
  pthread_t th[64];
  for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, fa_fill_worker, &F);
  for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&F.mu);
  fa_spec_free(sp);
  return 0;
}

/* ------------------------------------------------------------- misc draws */

/* n sizes floor(lo * (hi/lo)^u) (log-uniform), seeded */
void synth_loguniform_sizes(uint64_t seed_a, uint64_t seed_b, uint64_t n, double lo, double hi,
                            uint64_t *out) {
  rng_t r;
  rng_seed(&r, seed_a ^ 0x51235ull, seed_b);
  for (uint64_t i = 0; i < n; ++i) out[i] = rng_loguniform(&r, lo, hi);
}

/* n uniform integers in [0, bound) */
void synth_uniform(uint64_t seed_a, uint64_t seed_b, uint64_t n, uint64_t bound, uint64_t *out) {
  rng_t r;
  rng_seed(&r, seed_a ^ 0x0417ull, seed_b);
  for (uint64_t i = 0; i < n; ++i) out[i] = rng_below(&r, bound);
}

/* n uniform random bytes drawn from the first k symbols of alphabet */
void synth_bytes(uint64_t seed_a, uint64_t seed_b, uint64_t n, const uint8_t *alphabet, int k,
                 uint8_t *out) {
  rng_t r;
  rng_seed(&r, seed_a ^ 0xB17E5ull, seed_b);
  for (uint64_t i = 0; i < n; ++i) out[i] = alphabet[rng_below(&r, (uint64_t)k)];
}

/* n bytes of back-to-back quality strings of read_len symbols each (the FASTQ
 * quality model above), with no headers, bases or newlines */
void synth_qualities(uint64_t seed_a, uint64_t seed_b, uint64_t n, uint64_t read_len, uint8_t *out) {
  rng_t r;
  rng_seed(&r, seed_a ^ 0x9A1ull, seed_b);
  for (uint64_t at = 0; at < n; at += read_len) read_qual(&r, n - at < read_len ? n - at : read_len, out + at);
}

/* exponential inter-arrival gaps (Poisson process), in nanoseconds, rate per second */
void synth_poisson_gaps(uint64_t seed_a, uint64_t seed_b, uint64_t n, double rate, uint64_t *out) {
  rng_t r;
  rng_seed(&r, seed_a ^ 0xA331ull, seed_b);
  for (uint64_t i = 0; i < n; ++i) {
    double u = 1.0 - rng_unit(&r);
    out[i] = (uint64_t)(-log(u) / rate * 1e9);
  }
}
