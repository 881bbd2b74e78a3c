// Internal: the archive handle and the host helpers shared by host.cpp and
// server.cpp.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "aceapex.h"
#include "format.h"
#include "kernels.h"

namespace aceapex {

constexpr int kBlock = (int)kDecodeThreads;
constexpr uint64_t kDefaultWaitNs = 2000000000ull;

template <class T>
T rd(const uint8_t *p) {
  T v;
  std::memcpy(&v, p, sizeof(T));
  return v;
}

// One library-wide epoch counter per device (host.cpp): epochs never repeat
// on a device, so a ready flag can never be mistaken for one of another call.
uint32_t *global_epoch(int device);

// Device memory of the library's buffers (host.cpp): allocations on the
// current device come from a per-device pool that keeps up to
// kPoolKeepBytes of freed memory for later allocations, so an archive opened
// after another was closed reuses its memory instead of asking the driver;
// dev_free first waits for the whole device, as cudaFree does, since any
// stream may still use the buffer.
constexpr uint64_t kPoolKeepBytes = uint64_t(8) << 30;
cudaError_t dev_alloc(void **p, uint64_t bytes, int *device);
void dev_free(void *p, int device);

// device buffer that owns its memory
template <class T>
struct DBuf {
  T *p = nullptr;
  uint64_t n = 0;
  int dev = 0;
  cudaError_t alloc(uint64_t count) {
    release();
    if (!count) return cudaSuccess;
    const cudaError_t e = dev_alloc(reinterpret_cast<void **>(&p), count * sizeof(T), &dev);
    if (e != cudaSuccess) p = nullptr;
    n = p ? count : 0;
    return e;
  }
  void release() {
    if (p) dev_free(p, dev);
    p = nullptr;
    n = 0;
  }
};

// pinned host staging whose previous async copy is waited for before reuse
struct Staging {
  void *p = nullptr;
  uint64_t bytes = 0;
  cudaEvent_t done = nullptr;
  bool pending = false;
  cudaError_t reserve(uint64_t b) {
    if (pending) cudaEventSynchronize(done), pending = false;
    if (b <= bytes) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMallocHost(&p, b);
    if (e == cudaSuccess) bytes = b;
    if (!done) cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    return e;
  }
  void mark(cudaStream_t st) {
    cudaEventRecord(done, st);
    pending = true;
  }
  void release() {
    if (pending) cudaEventSynchronize(done);
    if (p) cudaFreeHost(p);
    if (done) cudaEventDestroy(done);
    p = nullptr;
    done = nullptr;
    bytes = 0;
    pending = false;
  }
};

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? ACEAPEX_OK : ACEAPEX_ECUDA; }

// host array whose storage is not initialised on allocation (the archive's
// index sections are copied into it once, in parallel pieces)
template <class T>
struct HostArray {
  std::unique_ptr<T[]> p;
  uint64_t n = 0;
  bool alloc(uint64_t count) {
    p.reset(count ? new (std::nothrow) T[count] : nullptr);
    n = count;
    return !count || p != nullptr;
  }
  T &operator[](uint64_t i) { return p[i]; }
  const T &operator[](uint64_t i) const { return p[i]; }
  T *data() { return p.get(); }
  uint64_t size() const { return n; }
};

}  // namespace aceapex

// (internal header: the handle's members use the library namespace)
using namespace aceapex;

struct aceapex_archive {
  int device = 0;
  Header h{};
  std::vector<SegRec> dir;
  HostArray<uint64_t> dep_ptr;
  HostArray<uint32_t> deps;
  HostArray<uint64_t> reads;
  aceapex_stats stats{};

  DBuf<uint8_t> d_payload;
  DBuf<SegRec> d_dir;
  DBuf<uint32_t> d_lut;
  DBuf<uint64_t> d_flags;   // level << 32 | epoch of the call that completed the segment
  DBuf<WorkItem> d_order;    // all segments in level order
  DBuf<uint32_t> d_words;    // [0] err, [1] epoch, [2] counter
  DBuf<uint8_t> d_blocked;
  DBuf<uint8_t> d_scratch;
  uint32_t scratch_warps = 0;
  int grid = 0;       // CTAs of the current launch configuration
  int max_grid = 0;   // occupancy limit (scratch is sized for it)
  uint32_t active_warps = kDecodeThreads / 32;
  uint32_t stage_cap = kSmemStage;
  uint32_t max_cmd_syms = 0;  // largest command stage of any segment: n_cmd * (4 + W) + 4 bytes
  uint64_t wait_ns = kDefaultWaitNs;
  bool any_blocked = false;

  // range decode: page table, arena of slots, work list
  DBuf<uint32_t> d_page;
  DBuf<uint8_t> d_arena;
  DBuf<WorkItem> d_work;
  Staging stage_work;
  std::vector<uint32_t> mark;
  uint32_t mark_gen = 0;
  // device closures (wide dependency lists): the lists on the device, tagged
  // marks, the member list, counters, and a pinned word for the member count
  DBuf<uint64_t> d_dep_ptr;
  DBuf<uint32_t> d_deps, d_cmark, d_clist, d_ccnt;
  Staging stage_cnt;
  uint32_t cgen = 0;

  // ring streaming
  DBuf<uint8_t> d_ring;
  DBuf<uint32_t> d_seg_crc;
  // batch
  std::vector<uint8_t> batch_desc;  // host copy of what d_batch_arcs / d_batch_views hold
  DBuf<DevArchive> d_batch_arcs;
  DBuf<OutView> d_batch_views;
  Staging stage_batch;
  // decode to host: device output buffer, window work lists, copy stream
  DBuf<uint8_t> d_host_out;
  DBuf<WorkItem> d_win_work;
  std::vector<uint64_t> win_start;  // work-list offset of each window
  uint64_t win_bytes = 0;
  cudaStream_t copy_st = nullptr;
  std::vector<cudaEvent_t> win_ev;
  // a payload upload still in flight after the open (aceapex_decode_host):
  // its stream, an event after each piece and the payload bytes then present
  cudaStream_t up_st = nullptr;
  std::vector<cudaEvent_t> up_ev;
  std::vector<uint64_t> up_end;
  // FASTQ stream reassembly (when this handle is a set's first part)
  DBuf<uint8_t> d_fq_streams;
  DBuf<uint32_t> d_fq_counts, d_fq_nl;
  DBuf<uint64_t> d_fq_offs;

  uint32_t *err() const { return d_words.p; }
  uint32_t *epoch() const { return d_words.p + 1; }
  uint32_t *counter() const { return d_words.p + 2; }

  DevArchive dev() const {
    DevArchive A{};
    A.payload = d_payload.p;
    A.dir = d_dir.p;
    A.order = d_order.p;
    A.lut = d_lut.p;
    A.flags = d_flags.p;
    A.blocked = any_blocked ? d_blocked.p : nullptr;
    A.n = h.n;
    A.D = h.D;
    A.log2_S = h.log2_S;
    A.W = h.W;
    A.min_match = h.min_match;
    A.n_seg = (uint32_t)h.n_seg;
    return A;
  }

  void end_upload() {
    if (up_st) cudaStreamSynchronize(up_st);
    for (cudaEvent_t e : up_ev) cudaEventDestroy(e);
    up_ev.clear();
    up_end.clear();
    if (up_st) cudaStreamDestroy(up_st);
    up_st = nullptr;
  }

  void release() {
    end_upload();
    d_payload.release(); d_dir.release(); d_lut.release(); d_flags.release(); d_order.release();
    d_words.release(); d_blocked.release(); d_scratch.release(); d_page.release(); d_arena.release();
    d_work.release(); d_ring.release(); d_seg_crc.release(); d_batch_arcs.release(); d_batch_views.release();
    d_fq_streams.release(); d_fq_counts.release(); d_fq_nl.release(); d_fq_offs.release();
    d_host_out.release(); d_win_work.release();
    d_dep_ptr.release(); d_deps.release(); d_cmark.release(); d_clist.release(); d_ccnt.release();
    stage_cnt.release();
    for (cudaEvent_t e : win_ev) cudaEventDestroy(e);
    win_ev.clear();
    if (copy_st) cudaStreamDestroy(copy_st);
    copy_st = nullptr;
    stage_work.release();
    stage_batch.release();
  }
};

namespace aceapex {

// segments sorted by (level, index), appended to out with archive index arc
void level_order(const std::vector<SegRec> &dir, const uint32_t *segs, uint64_t n, uint32_t arc,
                 std::vector<WorkItem> &out);
// launch shape and (when an archive needs it) the global staging slots
int ensure_scratch(aceapex_archive *A, uint32_t need_cmd_syms);
int ensure_scratch(aceapex_archive *A);
// a DecodeLaunch with the handle's control words, scratch and knobs
DecodeLaunch base_launch(aceapex_archive *A);
OutView linear_view(uint8_t *base, uint64_t origin);
// transitive source closure of segments [s_lo, s_hi] from the stored lists;
// with max_edges > 0, gives up (returns false) after visiting that many
// dependency entries
bool closure(aceapex_archive *A, uint64_t s_lo, uint64_t s_hi, std::vector<uint32_t> &out, uint64_t max_edges = 0);
// the same walk with caller-owned marks (one set per thread that walks)
bool closure_with(const aceapex_archive *A, uint64_t s_lo, uint64_t s_hi, std::vector<uint32_t> &mark, uint32_t &gen,
                  std::vector<uint32_t> &out, uint64_t max_edges = 0);
// the same for a list of seed segments; marks with a fresh generation of A->mark
void closure_of(aceapex_archive *A, const uint32_t *seeds, uint64_t n, std::vector<uint32_t> &out);

}  // namespace aceapex
