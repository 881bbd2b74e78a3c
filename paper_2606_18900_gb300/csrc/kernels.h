// Device-side data structures and the launchers that host.cpp calls.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "format.h"

namespace aceapex {

// Device error word values (match aceapex_status).
constexpr uint32_t kErrCorrupt = 2;
constexpr uint32_t kErrTimeout = 5;

// A unit of work: archive index (batch) and segment.
struct WorkItem {
  uint32_t arc;
  uint32_t seg;
};

// One archive as the kernels see it (all pointers are device pointers).
struct DevArchive {
  const uint8_t *payload;   // payload section (segment payloads, 16-byte aligned)
  const SegRec *dir;        // segment directory
  const WorkItem *order;    // all segments in level order
  const uint32_t *lut;      // 4 classes x 4096 slots: sym | bias << 8 | (freq - 1) << 20
  uint64_t *flags;          // per segment: its level << 32 | the epoch of the call that completed it
  const uint8_t *blocked;   // test hook: per-segment "never publish" bytes, or nullptr
  uint64_t n;               // decompressed size
  uint64_t D;               // distance bound (0 = none)
  uint32_t log2_S, W, min_match, n_seg;
};

// Where absolute output position p lives.
//  linear / ring: base + ((p - origin) & mask)   (mask = ~0 for linear)
//  paged:         slot_base + page[p >> log2_S] * S + (p & (S - 1))
struct OutView {
  uint8_t *base;
  uint64_t origin;
  uint64_t mask;
  const uint32_t *page;  // non-null selects paged addressing
  uint8_t *slot_base;
};

struct DecodeLaunch {
  DevArchive arc0;          // single-archive launches
  OutView view0;
  const DevArchive *arcs;   // batch launches: device arrays indexed by WorkItem::arc (else nullptr)
  const OutView *views;
  const WorkItem *work;     // device array in dependency-respecting order
  uint32_t n_work;
  const uint32_t *epoch;    // device word written by the begin kernel of this call
  uint32_t *counter;        // work counter, zeroed by the begin kernel
  uint32_t *err;            // device error word
  uint8_t *scratch;         // per-warp staging, kStageBytes each
  uint64_t wait_ns;         // dependency wait limit
  uint32_t scratch_warps;   // number of per-warp staging slots
  uint32_t active_warps;    // warps per CTA that take work (<= kDecodeThreads / 32)
  uint32_t stage_cap;       // bytes of a warp's shared staging to use (<= kSmemStage)
  uint32_t max_stage;       // largest command stage (bytes) of any segment the launch may decode
};

// command stage of a segment: its n_cmd * (4 + W) command symbols plus a
// 4-byte sentinel record; the global slot holds the largest possible one
constexpr uint32_t kStageBytes = kMaxSym + 16;
constexpr uint32_t kDecodeThreads = 1024;  // decode CTA: 32 warps, one CTA per SM
constexpr uint32_t kSmemStage = 3072;      // per-warp shared staging for the command streams
constexpr uint32_t kLutBytes = 4 * kScale * 4;

struct LaunchShape {
  int grid;
  int block;
};

// Start of a decode call: *epoch = ++*global_epoch, *counter = 0 (one thread).
// Keeping the epoch in device memory makes replays of a captured graph use
// fresh epochs.
cudaError_t launch_begin(uint32_t *global_epoch, uint32_t *epoch, uint32_t *counter, cudaStream_t st);

// flags[s] = dir[s].level << 32 for s < n: each segment's flag word with its
// level and no epoch
cudaError_t launch_init_flags(uint64_t *flags, const SegRec *dir, uint64_t n, cudaStream_t st);

// Work lists of windows of `per` segments: out[s0 .. s1) holds window
// [s0, s1)'s segments by (level, index); max_level: the highest level present
cudaError_t launch_window_order(const SegRec *dir, uint64_t n_seg, uint64_t per, uint32_t max_level, WorkItem *out,
                                cudaStream_t st);

// Persistent decode over L.work.
cudaError_t launch_decode(const DecodeLaunch &L, int grid, int block, cudaStream_t st);

// page[work[i].seg] = 0xFFFFFFFF for i < n (undo launch_set_pages)
cudaError_t launch_clear_pages(uint32_t *page, const WorkItem *work, uint32_t n, cudaStream_t st);

// copy [lo, hi) from view src to view dst (both addressed by absolute position)
cudaError_t launch_copy_view(OutView src, OutView dst, uint32_t log2_S, uint64_t lo, uint64_t hi, cudaStream_t st);

// Batch decode: each CTA takes whole archives (L.arcs[0..n_arcs), largest
// first) and decodes each archive's segments in its level order with the
// archive's decode table in shared memory. L.work is unused.
cudaError_t launch_batch(const DecodeLaunch &L, uint32_t n_arcs, int grid, cudaStream_t st);

// Occupancy-derived grid for the decode kernel.
int decode_grid(int device, int block);

// Gather [lo, hi) through a view into a flat buffer.
cudaError_t launch_gather(OutView v, uint32_t log2_S, uint64_t lo, uint64_t hi, uint8_t *dst, cudaStream_t st);

// n FASTA bases from lo (line phase `phase`, lines of line_width bases each
// followed by a newline) into a flat buffer, newlines dropped
cudaError_t launch_gather_bases(OutView v, uint32_t log2_S, uint64_t lo, uint32_t phase, uint32_t line_width,
                                uint64_t n, uint8_t *dst, cudaStream_t st);

// page[work[i].seg] = i for i < n (paged views)
cudaError_t launch_set_pages(uint32_t *page, const WorkItem *work, uint32_t n, cudaStream_t st);

// One request of a served batch: copy [lo, lo + n) of view v to dst.
struct GatherJob {
  OutView v;
  uint64_t lo, n;
  uint8_t *dst;
  uint64_t chunk0;  // first 64 KiB chunk of this job in the launch
  uint32_t log2_S, pad;
};

// All jobs in one launch: the jobs' 64 KiB chunks are spread over the CTAs.
cudaError_t launch_multi_gather(const GatherJob *jobs, uint32_t n_jobs, uint64_t n_chunks, cudaStream_t st);

// Reassembles a FASTQ from its four decoded line streams (base[k], len[k]
// bytes): newline index of each stream (counts: one u32 per 64 KiB chunk of
// the longest stream; offs: chunks + 1 u64 per stream; nl[k]: cap[k] u32
// positions, err latched beyond), then one warp per record copies its four
// lines to out.
cudaError_t launch_fastq_interleave(const uint8_t *const base[4], const uint64_t len[4], uint32_t *counts,
                                    uint64_t *offs, uint32_t *const nl[4], const uint64_t cap[4], uint32_t *err,
                                    uint8_t *out, cudaStream_t st);

// Transitive source closure on the device, for range decodes whose closure
// is too wide to walk on the host (paper §4.1: a read decodes its covering
// blocks plus their sources). mark: one u32 per segment, equal to gen when the
// segment is in the current closure; list: the members in discovery order;
// cnt[0]: their number. Every dependency has a lower level than its reader, so
// expanding the members of level L (max level down to 1) after all higher
// levels visits each member once.
struct ClosureDev {
  const uint64_t *dep_ptr;
  const uint32_t *deps;
  const SegRec *dir;
  uint32_t *mark;
  uint32_t *list;
  uint32_t *cnt;
};
// members := segments [s_lo, s_lo + n)
cudaError_t launch_closure_seed(ClosureDev C, uint32_t s_lo, uint32_t n, uint32_t gen, cudaStream_t st);
// add the unmarked dependencies of every member of level `level`
cudaError_t launch_closure_expand(ClosureDev C, uint32_t level, uint32_t gen, cudaStream_t st);
// members sorted by level into work[0 .. n), page[seg] = its position, n into *n_out
cudaError_t launch_closure_order(ClosureDev C, WorkItem *work, uint32_t *page, uint32_t *n_out, cudaStream_t st);

// CRC-32 of each window [lo + k*window, ...) of the ring view, written to crc[k].
cudaError_t launch_window_crc(OutView v, uint64_t lo, uint64_t hi, uint64_t window, uint32_t *crc, uint32_t *seg_crc,
                              uint32_t log2_S, cudaStream_t st);

}  // namespace aceapex
