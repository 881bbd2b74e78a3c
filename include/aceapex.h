/*
 * aceapex.h — C ABI of libaceapex.so, a GB300 (sm_103a) decoder for the
 * absolute-offset LZ77 block format of "Compressed-Resident Genomics:
 * Full-Pipeline Device-Resident GPU LZ77 Decode with Position-Invariant
 * Random Access" (arXiv 2606.18900). The byte format is version 1 of the
 * ACEAPEX1 archive format.
 *
 * Conventions
 *  - Every function returns an aceapex_status (0 = ACEAPEX_OK) unless noted.
 *  - Pointers named d_* are device pointers on the archive's device; h_*
 *    are host pointers. Sizes are bytes. Positions are absolute byte offsets
 *    into the decompressed output.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Decode calls are stream-ordered and asynchronous: the returned
 *    status covers argument and host-side validation only. Errors found by
 *    the kernels (a corrupt segment, a dependency wait that ran out of time)
 *    are latched in a device error word and reported by aceapex_last_error.
 *  - The library never writes outside [d_out, d_out + out_cap).
 *  - Calls on one archive handle must be serialised by the caller (one
 *    host thread at a time, and stream-ordered or synchronised between
 *    calls that use different streams): a handle owns one set of work
 *    counters, flags and scratch.
 */
#ifndef ACEAPEX_H
#define ACEAPEX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ACEAPEX_OK = 0,
  ACEAPEX_EINVAL = 1,   /* bad argument */
  ACEAPEX_ECORRUPT = 2, /* archive breaks a rule of the format */
  ACEAPEX_ENOMEM = 3,   /* host or device allocation failed, or over budget */
  ACEAPEX_ECUDA = 4,    /* a CUDA runtime call failed */
  ACEAPEX_ETIMEOUT = 5, /* a dependency wait ran past its time limit */
  ACEAPEX_ERANGE = 6,   /* position or size outside the archive / buffer */
  ACEAPEX_EBUSY = 7     /* admission refused (serving) */
} aceapex_status;

typedef struct aceapex_archive aceapex_archive;

/* Static per-archive byte counts (from the segment directory; no decode). */
typedef struct {
  uint64_t decoded_bytes;    /* U: N, bytes written by a full decode */
  uint64_t compressed_bytes; /* C: payload + directory + tables read by a full decode */
  uint64_t match_bytes;      /* M: sum of match lengths (match-source bytes read) */
  uint64_t literal_bytes;    /* literal bytes (N - M) */
  uint64_t n_commands;       /* matches in the archive */
  uint64_t n_segments;       /* 16 KiB (or smaller) decode units */
  uint64_t n_blocks;         /* B-byte blocks (paper's block size) */
  uint64_t n_deps;           /* dependency-list entries */
  uint64_t n_reads;          /* read-index entries */
  uint32_t max_level;        /* deepest level present */
  uint32_t log2_B, log2_S, W;
} aceapex_stats;

/*
 * Open an archive: validate it on the host (header, tables, directory,
 * dependency lists and read index against the format's rules) and copy the
 * sections the decoder needs into device memory on `device` (paper §3.3:
 * the archive is resident in VRAM before decoding; the copy is outside any
 * decode timer). The host bytes are not retained. On success *out owns the
 * device copies, flags, work counters and scratch; free it with
 * aceapex_close. Errors: EINVAL (null/zero arguments), ECORRUPT, ENOMEM,
 * ECUDA.
 */
int aceapex_open(const void *h_archive, uint64_t nbytes, int device, aceapex_archive **out);

/* Release every device and host resource of the handle (NULL is a no-op).
 * Synchronises the device first so that no kernel still uses them. Device
 * memory goes back to the library's per-device pool, which keeps up to
 * 8 GiB of freed memory for later opens (an open after a close then
 * allocates nothing from the driver); aceapex_release_cached_memory returns
 * it to the driver. */
void aceapex_close(aceapex_archive *a);

/* Return the device memory that the library's pool on `device` keeps for
 * reuse (memory of open handles stays allocated). Errors: ECUDA. */
int aceapex_release_cached_memory(int device);

/* Decompressed size N of the archive (0 for NULL). */
uint64_t aceapex_decoded_size(const aceapex_archive *a);

/* Fill *st with the archive's static counts. */
int aceapex_get_stats(const aceapex_archive *a, aceapex_stats *st);

/*
 * Histogram of the segments' dependency levels (the wavefront depth of paper
 * §2's block DAG under the archive's level cap): h_counts[l] = number of
 * segments at level l, for l < n (levels >= n are not counted). Host only, no
 * GPU work. Errors: EINVAL (NULL pointers).
 */
int aceapex_level_counts(const aceapex_archive *a, uint64_t *h_counts, uint32_t n);

/*
 * Whole-file device-resident decode (paper §3.3, "v4": entropy decode and
 * match resolution both on the GPU, output kept in VRAM). Writes the N
 * decoded bytes to d_out[0..N). One persistent launch: each warp takes the
 * next segment in level order, rANS-decodes its four streams, waits for the
 * segments its matches read (bounded wait), resolves its commands and
 * publishes its ready flag. Errors: EINVAL, ERANGE (out_cap < N), ECUDA.
 * opt_stats, when not NULL, receives aceapex_get_stats.
 */
int aceapex_decode_all(aceapex_archive *a, void *d_out, uint64_t out_cap, void *stream, aceapex_stats *opt_stats);

/*
 * Whole-file decode into host memory (paper §3.3's end-to-end measurement
 * over the host link): the archive decodes into a device buffer owned by the
 * handle, in windows of `window` bytes (0: 64 MiB; rounded to whole
 * segments) taken in order, and each window is copied to h_out[0..N) on a
 * second stream while the next one decodes. A window's segments read only
 * segments of the same or earlier windows, which are complete by then.
 * h_out should be pinned host memory for the copies to overlap. Stream-
 * ordered: work on `stream` after this call starts after the last copy.
 * Errors: EINVAL, ERANGE (out_cap < N), ENOMEM, ECUDA.
 */
int aceapex_decode_all_to_host(aceapex_archive *a, void *h_out, uint64_t out_cap, uint64_t window, void *stream);

/*
 * One call from a host archive to host output (paper §3.3's end-to-end
 * path): open the archive on `device`, decode it as
 * aceapex_decode_all_to_host does, check the decode's error word and close
 * the handle, returning when h_out[0..N) holds the output. The host checks
 * are aceapex_open's without the dependency lists and the read index, which
 * a whole-file decode does not read. Unlike open followed by a decode, the
 * payload goes to the device in 32 MiB pieces that decoding may overtake:
 * the first two while the host checks run, the rest once the small sections
 * are queued; a window's decode starts once the pieces holding its segments
 * have arrived, so the upload, the decodes and the copies back overlap.
 * h_archive (nbytes, caller-owned, read only; pinned
 * memory for the upload to overlap) is read until the call returns. Errors:
 * those of aceapex_open and aceapex_decode_all_to_host, and the device-side
 * ECORRUPT / ETIMEOUT of the decode.
 */
int aceapex_decode_host(const void *h_archive, uint64_t nbytes, int device, void *h_out, uint64_t out_cap,
                        uint64_t window);

/*
 * Range decode (paper §4, "v7-RA"): write exactly the bytes [byte_lo,
 * byte_hi) of the decompressed output to d_out[0 .. byte_hi - byte_lo).
 * Decodes only the covering segments and their transitive source closure
 * (from the stored dependency lists) into the handle's scratch arena, then
 * gathers the requested bytes. Errors: EINVAL, ERANGE (hi > N, lo > hi,
 * out_cap too small), ENOMEM, ECUDA.
 */
int aceapex_decode_range(aceapex_archive *a, uint64_t byte_lo, uint64_t byte_hi, void *d_out, uint64_t out_cap,
                         void *stream);

/*
 * Read-to-block index lookup (paper §4.1): record `read_id` (0-based) covers
 * [*byte_lo, *byte_hi). Host only, O(1), no GPU work. Errors: EINVAL (no
 * index or NULL pointers), ERANGE (read_id >= n_reads).
 */
int aceapex_read_lookup(const aceapex_archive *a, uint64_t read_id, uint64_t *byte_lo, uint64_t *byte_hi);

/*
 * Closure of a range (paper §4 and §4.1: a range or read decodes the blocks
 * that hold it plus the transitive closure of their source blocks): the
 * number of segments that aceapex_decode_range(a, lo, hi, ...) decodes, in
 * *n_segments, and the deepest dependency level among them, in *max_level
 * (may be NULL); the wavefront of that decode has *max_level + 1 steps. Host
 * only, no GPU work; uses the handle's closure scratch, so calls on one
 * handle must not run concurrently. Errors: EINVAL (NULL a or n_segments),
 * ERANGE (lo > hi or hi > N).
 */
int aceapex_range_closure(aceapex_archive *a, uint64_t lo, uint64_t hi, uint64_t *n_segments, uint32_t *max_level);

/*
 * Report the device error word of the handle and clear it. sync != 0 first
 * synchronises `stream` (or the device when stream is NULL) so the word
 * covers every call issued before. Returns ACEAPEX_OK, ECORRUPT, ETIMEOUT or
 * ECUDA.
 */
int aceapex_last_error(aceapex_archive *a, int sync, void *stream);

/*
 * Set the time limit of every dependency wait of later launches, in
 * nanoseconds (default 2e9). A wait that reaches the limit latches ETIMEOUT
 * and the launch finishes without hanging. 0 restores the default.
 */
int aceapex_set_wait_limit(aceapex_archive *a, uint64_t ns);

/*
 * Launch configuration of the handle's later decode calls (the autotuner's
 * knobs): ctas = persistent CTAs (wavefront width, 1..max, one per SM at
 * most), warps_per_cta = warps of each CTA that take work (1..32), stage_bytes
 * = shared-memory staging per warp for the command streams (1..3072; larger
 * segments use the warp's global staging slot). 0 selects the default (the
 * occupancy limit, 32, 3072). Allocates the decode scratch on first use.
 * Errors: EINVAL, ENOMEM, ECUDA. aceapex_get_launch reports the current values
 * and the CTA limit.
 */
int aceapex_set_launch(aceapex_archive *a, uint32_t ctas, uint32_t warps_per_cta, uint32_t stage_bytes);
int aceapex_get_launch(const aceapex_archive *a, uint32_t *ctas, uint32_t *max_ctas, uint32_t *warps_per_cta,
                       uint32_t *stage_bytes);

/*
 * Test hook: segments whose index is in h_segs[0..n) never publish their
 * ready flag in later launches (n = 0 clears the list). Dependent segments
 * then run into the wait limit. Lets the tests exercise ETIMEOUT without
 * faulting or hanging a GPU.
 */
int aceapex_debug_block_segments(aceapex_archive *a, const uint32_t *h_segs, uint32_t n);

/*
 * Streaming range decode through a fixed device ring (paper §5: output size
 * decoupled from device memory). Decodes [byte_lo, byte_hi) window by
 * window; window k covers [byte_lo + k*window_bytes, min(byte_hi, byte_lo +
 * (k+1)*window_bytes)) and its CRC-32 (IEEE, zlib polynomial; replaces the
 * paper's FNV check) is written to d_crc_per_window[k] on the device. Needs
 * an archive with a distance bound D and ring_bytes >= window_bytes + D +
 * 2*S rounded up to a power of two; window_bytes must be a multiple of the
 * segment size. The ring is owned by the handle (allocated on first use).
 * Errors: EINVAL (D == 0, bad sizes), ERANGE, ENOMEM, ECUDA.
 */
int aceapex_stream_range(aceapex_archive *a, uint64_t byte_lo, uint64_t byte_hi, uint64_t ring_bytes,
                         uint64_t window_bytes, uint32_t *d_crc_per_window, void *stream);

/*
 * Batched decode of n archives into n caller buffers (d_outs[i] holds at
 * least aceapex_decoded_size(as[i]) bytes) in one persistent launch; the
 * work list interleaves the archives' segments in level order. All archives
 * must live on the same device. Errors: EINVAL, ECUDA, ENOMEM.
 */
int aceapex_decode_batch(aceapex_archive *const *as, int n, void *const *d_outs, void *stream);

/*
 * Serving engine (continuous batching over device-resident archives; the
 * paper's random access, §4 and §4.1, for many concurrent requests).
 *
 * aceapex_server_create: serve the n archives as[0..n) (same device; the
 * server does not own them and they must outlive it; do not call other
 * decode functions on them while the server runs). mem_budget: device bytes
 * for the server (per-slot page tables and flags, 12 bytes per segment per
 * slot, and the decode arenas, the rest split evenly over the slots). slots:
 * batches that may be in flight at once (1..64), each on its own stream. A
 * worker thread forms batches from the queue in arrival order while the union
 * of the requests' source closures fits a slot's arena, and launches a batch
 * whenever a slot is free, so requests that arrive while batches run are
 * decoded in the next batch, overlapping with them.
 *
 * aceapex_server_submit: queue bytes [byte_lo, byte_hi) of archive `arc`, to
 * be written to the device buffer d_dst (cap bytes, caller-owned, must stay
 * valid until the request completes). Returns a ticket; the request's
 * transitive source closure is walked afterwards by the server's walker
 * threads, so the call itself only enqueues. EBUSY: the range's own segments
 * exceed a slot's arena (admission refused at once); a wider closure that can
 * never fit completes the request with status EBUSY instead. ERANGE, EINVAL.
 *
 * aceapex_server_poll: *done = 1 once the request completed (then the ticket
 * is released, the return value is the request's status and *latency_ms the
 * time from submission to completion); *done = 0 while pending (return
 * ACEAPEX_OK). wait != 0 blocks until completion.
 */
typedef struct aceapex_server aceapex_server;
typedef struct {
  uint64_t submitted, completed, refused, batches, bytes_served;
  uint64_t max_batch;      /* most requests in one batch */
  uint64_t max_inflight;   /* most batches in flight at once */
  uint64_t queued;         /* requests waiting now */
  uint64_t slot_segments;  /* arena capacity of a slot, in segments */
} aceapex_server_stats;

int aceapex_server_create(aceapex_archive *const *as, int n, uint64_t mem_budget, int slots, aceapex_server **out);
void aceapex_server_destroy(aceapex_server *s);
int aceapex_server_submit(aceapex_server *s, int arc, uint64_t byte_lo, uint64_t byte_hi, void *d_dst, uint64_t cap,
                          uint64_t *ticket);
int aceapex_server_poll(aceapex_server *s, uint64_t ticket, int wait, int *done, double *latency_ms);
/*
 * Open-loop arrivals from native code: submits request i (archive arc[i],
 * bytes [lo[i], hi[i]) into d_dst[i], cap[i] bytes) gap_ns[i] nanoseconds
 * after the due time of request i - 1 (the first after gap_ns[0]), waiting on
 * the host clock and never on completions, so a trace of Poisson gaps is
 * offered at its own rate whatever the serving latency. status[i] receives
 * the aceapex_server_submit result and ticket[i] its ticket (0 when refused);
 * *submit_seconds (may be NULL) the time from the call to the last
 * submission. Tickets are then polled as usual. Errors: EINVAL (NULL server
 * or arrays).
 */
int aceapex_server_replay(aceapex_server *s, uint64_t n, const int *arc, const uint64_t *lo, const uint64_t *hi,
                          void *const *d_dst, const uint64_t *cap, const uint64_t *gap_ns, uint64_t *ticket,
                          int *status, double *submit_seconds);
int aceapex_server_get_stats(aceapex_server *s, aceapex_server_stats *out);

/*
 * Allocation-free whole-file decode. The paper has no counterpart; this entry
 * point exists for callers that cannot allocate device memory when they
 * decode: for example a program that gives all device memory to its own pool
 * at start-up and forbids libraries from calling cudaMalloc afterwards, or a
 * real-time pipeline that only allows allocation during initialisation. It
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * d_archive: the complete archive (version 1) in device memory, 16-byte
 * aligned, nbytes long (caller-owned, read only). d_out: out_cap bytes of
 * device memory that receive the decoded output. d_status: one device word
 * that receives 0 or the aceapex_status of a device-side error once the work
 * queued on `stream` has run. The header (128 bytes) is read to the host
 * first, so the call synchronises `stream` once before queuing the decode.
 *
 * Scratch: a fixed array of about 4.6 MiB in the library's device memory,
 * which every GPU that loads the library holds until the process exits. The
 * first call on a device looks up the array's device address (with that
 * device current). Archives
 * of more than 65,536 segments (1 GiB at 16 KiB segments) are rejected with
 * ERANGE. All calls share the array and it keeps the last call's contents;
 * each call resets what must start at zero, but calls that overlap on the
 * GPU race and must not be issued. The decode uses 256 warps, so it is
 * slower than aceapex_decode_all. Errors: EINVAL (null, misaligned or short
 * archive), ECORRUPT (bad header), ERANGE (too many segments, out_cap < N),
 * ECUDA.
 */
int aceapex_decode_all_noalloc(const void *d_archive, uint64_t nbytes, void *d_out, uint64_t out_cap,
                               uint32_t *d_status, void *stream);

/*
 * Host encoder (paper §2: global match search, absolute offsets, fixed
 * blocks; the paper's encoder is CPU-only too). Produces a version-1
 * archive of h_in[0..n) in a malloc'd buffer *h_out (*out_len bytes; free
 * with aceapex_free). log2_B: block size exponent (2..30); min_match: 0 =
 * 4 + W; max_level: level cap; dist_bound: 0 = unbounded; h_reads /
 * n_reads: optional read index (record start offsets); threads: 0 = all
 * cores. Deterministic for any thread count. Errors: EINVAL, ENOMEM.
 */
int aceapex_encode(const void *h_in, uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t max_level,
                   uint64_t dist_bound, const uint64_t *h_reads, uint64_t n_reads, int threads, void **h_out,
                   uint64_t *out_len);

/* Free a buffer returned by aceapex_encode. */
void aceapex_free(void *p);

/* FASTQ record start offsets of h_in (every fourth line starts a record);
 * writes at most cap entries to h_out and returns the total count. */
uint64_t aceapex_fastq_index(const void *h_in, uint64_t n, uint64_t *h_out, uint64_t cap);

/*
 * FASTA coordinate index (the paper's chr:pos index, left there as future
 * work, §4.1): for every record, the offset of its '>' and the offset of its
 * first sequence byte, and one more entry (the offset of the last byte) when
 * the file's last line has no newline; writes at most cap entries to h_out
 * and returns the total count. *line_width (when not NULL) receives the
 * length of the longest sequence line. Stored as an archive's read index (the
 * h_reads of aceapex_encode), it serves aceapex_region_lookup and
 * aceapex_decode_region.
 */
uint64_t aceapex_fasta_index(const void *h_in, uint64_t n, uint64_t *h_out, uint64_t cap, uint32_t *line_width);

/*
 * Coordinates to bytes: bases [pos, pos + len) of record `chrom` (0-based,
 * in file order) of a FASTA archive carrying the coordinate index above,
 * whose sequence lines hold line_width bases each: base p sits at byte
 * seq_start + p + floor(p / line_width). Writes the byte range [*byte_lo,
 * *byte_hi) that covers the bases (with the newlines between them). Host
 * only, O(1). Errors: EINVAL (no coordinate index, len or line_width 0),
 * ERANGE (chrom or the bases outside the record).
 */
int aceapex_region_lookup(const aceapex_archive *a, uint64_t chrom, uint64_t pos, uint64_t len, uint32_t line_width,
                          uint64_t *byte_lo, uint64_t *byte_hi);

/*
 * Region decode by coordinates: writes exactly the len bases of
 * aceapex_region_lookup (newlines dropped) to d_out[0 .. len): the covering
 * segments and their source closure are decoded as in aceapex_decode_range,
 * then a gather kernel skips the newline after every line_width bases.
 * Errors: those of aceapex_region_lookup, ERANGE (out_cap < len), ENOMEM,
 * ECUDA.
 */
int aceapex_decode_region(aceapex_archive *a, uint64_t chrom, uint64_t pos, uint64_t len, uint32_t line_width,
                          void *d_out, uint64_t out_cap, void *stream);

/*
 * FASTQ stream separation (the paper's ids / sequences / qualities split,
 * reported there for +10-11 % ratio): line k of h_in goes to stream k mod 4
 * (headers, sequences, '+' lines, qualities), each line with its newline. The
 * four streams are written back to back to h_out (n bytes, caller-owned) and
 * their lengths to h_lens[0..3]. Returns the number of records. Host only.
 */
uint64_t aceapex_fastq_split(const void *h_in, uint64_t n, void *h_out, uint64_t *h_lens);

/*
 * Whole-file decode of a FASTQ stored as four archives of its line streams
 * (parts[k] holds stream k of aceapex_fastq_split): each part decodes with
 * its own persistent launch into scratch owned by parts[0], a newline index
 * of each stream is built on the device, and one warp per record copies its
 * four lines to d_out[0 .. N), N the sum of the streams' sizes. Stream-
 * ordered; decode errors are latched in each part's error word, and a
 * stream that is not made of FASTQ lines in parts[0]'s. Each stream must be below 4 GiB. Errors:
 * EINVAL, ERANGE (out_cap < N or a stream too large), ENOMEM, ECUDA.
 */
int aceapex_decode_fastq_streams(aceapex_archive *const *parts, void *d_out, uint64_t out_cap, void *stream);

/*
 * GPU encoder (paper §2's global match search run on the device; the paper's
 * encoder is CPU-only and is the bottleneck it names in §8). It applies the
 * rules of aceapex_encode (same hash, chain depth, level schedule, parse and
 * tables) and returns the same archive, byte for byte.
 *
 * aceapex_gpu_encoder_create binds an encoder to a device; it owns a CUDA
 * stream and device scratch that grows on demand and is kept between calls:
 * the input, 16 bytes per position of a chain window (sort keys and values,
 * twice), 8 per position of a parse window (match table), up to 16 KiB of
 * symbols per segment, and the archive; a 1 GiB input takes about 30 GB.
 * aceapex_gpu_encoder_destroy frees it all. Calls on one encoder must be
 * serialised by the caller (one scratch set); separate encoders are
 * independent. Errors: EINVAL, ENOMEM, ECUDA.
 */
typedef struct aceapex_gpu_encoder aceapex_gpu_encoder;

/* Device times of one aceapex_gpu_encode call (CUDA events on its stream). */
typedef struct {
  double ms_total;    /* input copy to archive copy-out, inclusive */
  double ms_h2d;      /* input copy into the encoder's padded buffer */
  double ms_chains;   /* hashing and radix sort (all windows) */
  double ms_match;    /* the match-search kernel (all windows) */
  double ms_parse;    /* match mask, parse, dependency lists, symbols, levels (all windows) */
  double ms_entropy;  /* tables, rANS (two passes), directory and sections */
  double ms_d2h;      /* archive copy to host memory */
  uint64_t input_bytes, archive_bytes, n_segments, n_deps, windows;
  uint64_t kernel_launches; /* kernels the call launched */
} aceapex_encode_stats;

int aceapex_gpu_encoder_create(int device, aceapex_gpu_encoder **out);
void aceapex_gpu_encoder_destroy(aceapex_gpu_encoder *enc);

/*
 * Encode in[0..n) (host memory, or device memory of the encoder's device when
 * in_on_device != 0) into a version-1 archive returned in a malloc'd host
 * buffer *h_out of *out_len bytes (free with aceapex_free). Parameters and
 * their limits are those of aceapex_encode (n < 2^32 when dist_bound = 0,
 * dist_bound < 2^31). Synchronous: returns when the archive is in host
 * memory. opt_stats (may be NULL) receives the phase times. Errors: EINVAL,
 * ENOMEM, ECUDA, ECORRUPT (an internal invariant of the encoder failed; no
 * archive is returned).
 */
int aceapex_gpu_encode(aceapex_gpu_encoder *enc, const void *in, int in_on_device, uint64_t n, uint32_t log2_B,
                       uint32_t min_match, uint32_t max_level, uint64_t dist_bound, const uint64_t *h_reads,
                       uint64_t n_reads, void **h_out, uint64_t *out_len, aceapex_encode_stats *opt_stats);

#ifdef __cplusplus
}
#endif

#endif /* ACEAPEX_H */
