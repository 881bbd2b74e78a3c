// Host side of libaceapex.so: archive validation (header, tables, directory,
// dependency lists), device residency (paper §3.3), work lists in level order,
// source closures for range decode (paper §4), the ring streamer (paper §5),
// batching, and the C ABI declared in include/aceapex.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "archive.h"

namespace aceapex {
int encode_archive(const uint8_t *in, uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t cap, uint64_t D,
                   const uint64_t *reads, uint64_t n_reads, int threads, uint8_t **out, uint64_t *out_len);
uint64_t fastq_index(const uint8_t *in, uint64_t n, uint64_t *out, uint64_t cap);
uint64_t fasta_index(const uint8_t *in, uint64_t n, uint64_t *out, uint64_t cap, uint32_t *line_width);
uint64_t fastq_split(const uint8_t *in, uint64_t n, uint8_t *out, uint64_t len[4]);
}  // namespace aceapex

using namespace aceapex;

namespace aceapex {

// One library-wide epoch counter per device: epochs never repeat on a device,
// so a ready flag can never be mistaken for one of another call.
struct DeviceState {
  uint32_t *d_global_epoch = nullptr;
};
std::mutex g_dev_mu;
std::map<int, DeviceState> g_dev;

uint32_t *global_epoch(int device) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceState &d = g_dev[device];
  if (!d.d_global_epoch) {
    if (cudaMalloc(&d.d_global_epoch, sizeof(uint32_t)) != cudaSuccess) return nullptr;
    if (cudaMemset(d.d_global_epoch, 0, sizeof(uint32_t)) != cudaSuccess) return nullptr;
  }
  return d.d_global_epoch;
}

// The per-device memory pools behind dev_alloc: created on first use, with a
// private stream that orders their allocations and frees (each is waited
// for, so a buffer is usable on any stream when dev_alloc returns). Devices
// without stream-ordered allocation fall back to cudaMalloc / cudaFree.
struct DevPool {
  std::once_flag once;
  cudaMemPool_t pool = nullptr;
  cudaStream_t st = nullptr;
};
constexpr int kMaxPoolDevices = 64;
DevPool g_pool[kMaxPoolDevices];

DevPool *pool_of(int dev) {
  if (dev < 0 || dev >= kMaxPoolDevices) return nullptr;
  DevPool &P = g_pool[dev];
  std::call_once(P.once, [&] {
    int supported = 0;
    if (cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev) != cudaSuccess || !supported) return;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return;
    uint64_t keep = kPoolKeepBytes;
    cudaStream_t st = nullptr;
    int cur = 0;
    cudaGetDevice(&cur);
    const bool same = cur == dev || cudaSetDevice(dev) == cudaSuccess;
    if (!same || cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      if (cur != dev) cudaSetDevice(cur);
      return;
    }
    if (cur != dev) cudaSetDevice(cur);
    P.pool = pool;
    P.st = st;
  });
  return P.pool ? &P : nullptr;
}

cudaError_t dev_alloc(void **p, uint64_t bytes, int *device) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  *device = dev;
  DevPool *P = pool_of(dev);
  if (!P) return cudaMalloc(p, bytes);
  e = cudaMallocFromPoolAsync(p, bytes, P->pool, P->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);
  return e;
}

void dev_free(void *p, int device) {
  DevPool *P = pool_of(device);
  if (!P) {
    cudaFree(p);
    return;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != device) cudaSetDevice(device);
  cudaDeviceSynchronize();
  cudaFreeAsync(p, P->st);
  cudaStreamSynchronize(P->st);
  if (cur != device) cudaSetDevice(cur);
}

}  // namespace aceapex


namespace aceapex {

// Host-side checks of the format (header, tables, directory, dependency lists,
// read index); fills h, dir, dep_ptr, deps, reads, stats.
// f(0) .. f(n - 1) on up to 16 host threads
template <class F>
void parallel_for(uint64_t n, F f) {
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  const uint64_t nt = std::min<uint64_t>(n, hw);
  if (nt <= 1) {
    for (uint64_t k = 0; k < n; ++k) f(k);
    return;
  }
  std::atomic<uint64_t> next{0};
  std::vector<std::thread> ts;
  for (uint64_t t = 0; t < nt; ++t)
    ts.emplace_back([&] {
      for (uint64_t k; (k = next.fetch_add(1)) < n;) f(k);
    });
  for (auto &t : ts) t.join();
}

int fill_stats(aceapex_archive *A, uint64_t n_lit, uint64_t n_cmd, uint32_t max_lv);

// (lists = false: the dependency lists and the read index are neither checked
// nor copied; a whole-file decode reads neither)
int validate(const uint8_t *a, uint64_t len, aceapex_archive *A, bool lists = true) {
  if (len < kHeaderBytes + kTablesBytes || std::memcmp(a, "ACEAPEX1", 8) != 0) return ACEAPEX_ECORRUPT;
  if (rd<uint32_t>(a + 8) != 1 || rd<uint32_t>(a + 12) != kHeaderBytes) return ACEAPEX_ECORRUPT;
  Header &h = A->h;
  h.n = rd<uint64_t>(a + 16);
  h.log2_B = a[24];
  h.log2_S = a[25];
  h.W = a[26];
  h.min_match = a[27];
  h.max_level = a[30];
  h.flags = a[31];
  if (a[28] != kScaleBits || a[29] != kLanes || (h.flags & ~1u)) return ACEAPEX_ECORRUPT;
  if (h.log2_B < 2 || h.log2_B > 30 || h.log2_S != std::min<uint32_t>(h.log2_B, kMaxLog2S)) return ACEAPEX_ECORRUPT;
  if (h.W != offset_width(h.n) || h.min_match < 1) return ACEAPEX_ECORRUPT;
  h.D = rd<uint64_t>(a + 32);
  h.n_seg = rd<uint64_t>(a + 40);
  h.n_deps = rd<uint64_t>(a + 48);
  h.n_reads = rd<uint64_t>(a + 56);
  const uint64_t S = uint64_t(1) << h.log2_S;
  if (h.n_seg != (h.n + S - 1) / S || h.n_seg >= (uint64_t(1) << 32)) return ACEAPEX_ECORRUPT;
  if (!(h.flags & 1) && h.n_reads) return ACEAPEX_ECORRUPT;
  if (h.n_seg > len / 24 || h.n_deps > len / 4 || h.n_reads > len / 8) return ACEAPEX_ECORRUPT;
  h.off_tables = rd<uint64_t>(a + 64);
  h.off_dir = rd<uint64_t>(a + 72);
  h.off_dep_ptr = rd<uint64_t>(a + 80);
  h.off_deps = rd<uint64_t>(a + 88);
  h.off_reads = rd<uint64_t>(a + 96);
  h.off_payload = rd<uint64_t>(a + 104);
  h.payload_bytes = rd<uint64_t>(a + 112);
  h.total_bytes = rd<uint64_t>(a + 120);
  if (h.off_tables != kHeaderBytes || h.off_dir != kHeaderBytes + kTablesBytes ||
      h.off_dep_ptr != round16(h.off_dir + 24 * h.n_seg) ||
      h.off_deps != round16(h.off_dep_ptr + 8 * (h.n_seg + 1)) ||
      h.off_reads != round16(h.off_deps + 4 * h.n_deps) || h.off_payload != round16(h.off_reads + 8 * h.n_reads) ||
      h.total_bytes != h.off_payload + h.payload_bytes || h.total_bytes != len)
    return ACEAPEX_ECORRUPT;
  // tables
  for (int c = 0; c < 4; ++c) {
    uint32_t sum = 0;
    for (int s = 0; s < 256; ++s) sum += rd<uint16_t>(a + kHeaderBytes + 512 * c + 2 * s);
    if (sum != 0 && sum != kScale) return ACEAPEX_ECORRUPT;
  }
  // directory
  A->dir.resize(h.n_seg);
  if (h.n_seg) std::memcpy(A->dir.data(), a + h.off_dir, 24 * h.n_seg);
  uint64_t po = 0, n_lit = 0, n_cmd = 0;
  uint32_t max_lv = 0;
  for (uint64_t s = 0; s < h.n_seg; ++s) {
    const SegRec &r = A->dir[s];
    if (r.payload_off != po || r.zero != 0) return ACEAPEX_ECORRUPT;
    if ((uint64_t)r.n_cmd * (4 + h.W) + r.n_lit > kMaxSym) return ACEAPEX_ECORRUPT;
    if (r.level > h.max_level) return ACEAPEX_ECORRUPT;
    const uint64_t out_size = std::min<uint64_t>(S, h.n - s * S);
    if (r.n_lit > out_size || (uint64_t)r.n_cmd * h.min_match > out_size - r.n_lit) return ACEAPEX_ECORRUPT;
    po = round16(po + 128 + 2 * (uint64_t)r.n_words);
    A->max_cmd_syms = std::max<uint32_t>(A->max_cmd_syms, r.n_cmd * (4 + h.W) + 4);
    n_lit += r.n_lit;
    n_cmd += r.n_cmd;
    max_lv = std::max<uint32_t>(max_lv, r.level);
  }
  if (po != h.payload_bytes) return ACEAPEX_ECORRUPT;
  if (!lists) return fill_stats(A, n_lit, n_cmd, max_lv);
  // dependency lists (ascending, below their segment, level consistent) and
  // the read index (ascending, below N): copied and checked in parallel
  // pieces, since at gigabyte sizes these are millions of entries
  std::vector<uint8_t> lvl(h.n_seg);
  for (uint64_t s = 0; s < h.n_seg; ++s) lvl[s] = (uint8_t)std::min<uint32_t>(A->dir[s].level, 255);
  if (!A->dep_ptr.alloc(h.n_seg + 1) || !A->deps.alloc(h.n_deps) || !A->reads.alloc(h.n_reads))
    return ACEAPEX_ENOMEM;
  std::memcpy(A->dep_ptr.data(), a + h.off_dep_ptr, 8 * (h.n_seg + 1));
  if (A->dep_ptr[0] != 0 || A->dep_ptr[h.n_seg] != h.n_deps) return ACEAPEX_ECORRUPT;
  for (uint64_t s = 0; s < h.n_seg; ++s)
    if (A->dep_ptr[s + 1] < A->dep_ptr[s]) return ACEAPEX_ECORRUPT;
  const uint64_t seg_per = std::max<uint64_t>(4096, (h.n_seg + 63) / 64);
  const uint64_t seg_pieces = (h.n_seg + seg_per - 1) / seg_per;
  const uint64_t read_per = std::max<uint64_t>(1 << 16, (h.n_reads + 63) / 64);
  const uint64_t read_pieces = (h.n_reads + read_per - 1) / read_per;
  std::vector<uint8_t> bad(seg_pieces + read_pieces, 0);
  parallel_for(seg_pieces + read_pieces, [&](uint64_t k) {
    if (k < seg_pieces) {
      const uint64_t s0 = k * seg_per, s1 = std::min(h.n_seg, s0 + seg_per);
      const uint64_t b0 = A->dep_ptr[s0], b1 = A->dep_ptr[s1];
      if (b1 > b0) std::memcpy(A->deps.data() + b0, a + h.off_deps + 4 * b0, 4 * (b1 - b0));
      for (uint64_t s = s0; s < s1; ++s) {
        const uint64_t b = A->dep_ptr[s], e = A->dep_ptr[s + 1];
        uint32_t lv = 0;
        for (uint64_t i = b; i < e; ++i) {
          const uint32_t d = A->deps[i];
          if (d >= s || (i > b && d <= A->deps[i - 1])) {
            bad[k] = 1;
            return;
          }
          lv = std::max<uint32_t>(lv, lvl[d] + 1u);
        }
        if (lv != A->dir[s].level) {
          bad[k] = 1;
          return;
        }
      }
    } else {
      const uint64_t r0 = (k - seg_pieces) * read_per, r1 = std::min(h.n_reads, r0 + read_per);
      std::memcpy(A->reads.data() + r0, a + h.off_reads + 8 * r0, 8 * (r1 - r0));
      uint64_t prev = r0 ? rd<uint64_t>(a + h.off_reads + 8 * (r0 - 1)) : 0;
      for (uint64_t r = r0; r < r1; ++r) {
        if (A->reads[r] >= h.n || (r && A->reads[r] <= prev)) {
          bad[k] = 1;
          return;
        }
        prev = A->reads[r];
      }
    }
  });
  for (uint8_t b : bad)
    if (b) return ACEAPEX_ECORRUPT;
  return fill_stats(A, n_lit, n_cmd, max_lv);
}

int fill_stats(aceapex_archive *A, uint64_t n_lit, uint64_t n_cmd, uint32_t max_lv) {
  const Header &h = A->h;
  aceapex_stats &st = A->stats;
  st.decoded_bytes = h.n;
  st.compressed_bytes = h.payload_bytes + 24 * h.n_seg + kTablesBytes;
  st.literal_bytes = n_lit;
  st.match_bytes = h.n - n_lit;
  st.n_commands = n_cmd;
  st.n_segments = h.n_seg;
  st.n_blocks = (h.n + (uint64_t(1) << h.log2_B) - 1) >> h.log2_B;
  st.n_deps = h.n_deps;
  st.n_reads = h.n_reads;
  st.max_level = max_lv;
  st.log2_B = h.log2_B;
  st.log2_S = h.log2_S;
  st.W = h.W;
  return ACEAPEX_OK;
}

// decode table: slot -> sym | (slot - cum) << 8 | (freq - 1) << 20
void build_lut(const uint8_t *a, std::vector<uint32_t> &lut) {
  lut.assign(4 * kScale, 0);
  for (int c = 0; c < 4; ++c) {
    uint32_t cum = 0;
    for (int s = 0; s < 256; ++s) {
      uint32_t f = rd<uint16_t>(a + kHeaderBytes + 512 * c + 2 * s);
      for (uint32_t k = 0; k < f; ++k) lut[c * kScale + cum + k] = (uint32_t)s | (k << 8) | ((f - 1) << 20);
      cum += f;
    }
  }
}

// segments sorted by (level, index)
void level_order(const std::vector<SegRec> &dir, const uint32_t *segs, uint64_t n, uint32_t arc,
                 std::vector<WorkItem> &out) {
  uint32_t cnt[257] = {};
  for (uint64_t i = 0; i < n; ++i) cnt[dir[segs ? segs[i] : i].level + 1]++;
  for (int l = 0; l < 256; ++l) cnt[l + 1] += cnt[l];
  size_t base = out.size();
  out.resize(base + n);
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t s = segs ? segs[i] : (uint32_t)i;
    out[base + cnt[dir[s].level]++] = WorkItem{arc, s};
  }
}

// Launch shape, and the per-warp global staging slots, which only segments
// whose command streams exceed the shared stage use: they are allocated only
// when the archive (or, for a batch, any archive) has such a segment.
int ensure_scratch(aceapex_archive *A, uint32_t need_cmd_syms) {
  if (!A->max_grid) {
    // (looked up once per device: the lookup sets kernel attributes and asks
    // the driver for the occupancy, and every open needs it)
    static std::mutex grid_mu;
    static std::map<int, int> grid_of;
    {
      std::lock_guard<std::mutex> lk(grid_mu);
      auto it = grid_of.find(A->device);
      A->max_grid = it != grid_of.end() ? it->second : (grid_of[A->device] = decode_grid(A->device, kBlock));
    }
    if (A->grid <= 0 || A->grid > A->max_grid) A->grid = A->max_grid;
    A->scratch_warps = (uint32_t)A->max_grid * (kBlock / 32);
  }
  if (need_cmd_syms > A->stage_cap && !A->d_scratch.p) {
    if (A->d_scratch.alloc((uint64_t)A->scratch_warps * kStageBytes) != cudaSuccess) return ACEAPEX_ENOMEM;
  }
  return ACEAPEX_OK;
}

int ensure_scratch(aceapex_archive *A) { return ensure_scratch(A, A->max_cmd_syms); }

DecodeLaunch base_launch(aceapex_archive *A) {
  DecodeLaunch L{};
  L.arc0 = A->dev();
  L.epoch = A->epoch();
  L.counter = A->counter();
  L.err = A->err();
  L.scratch = A->d_scratch.p;
  L.scratch_warps = A->scratch_warps;
  L.wait_ns = A->wait_ns;
  L.active_warps = A->active_warps;
  L.stage_cap = A->stage_cap;
  L.max_stage = A->max_cmd_syms;
  return L;
}

OutView linear_view(uint8_t *base, uint64_t origin) {
  OutView v{};
  v.base = base;
  v.origin = origin;
  v.mask = ~uint64_t(0);
  return v;
}

// transitive source closure of segments [s_lo, s_hi] (host, from the stored lists)
bool closure_with(const aceapex_archive *A, uint64_t s_lo, uint64_t s_hi, std::vector<uint32_t> &mark, uint32_t &gen,
                  std::vector<uint32_t> &out, uint64_t max_edges) {
  if (mark.size() != A->h.n_seg) mark.assign(A->h.n_seg, 0);
  if (++gen == 0) {
    std::fill(mark.begin(), mark.end(), 0);
    gen = 1;
  }
  const uint32_t g = gen;
  out.clear();
  std::vector<uint32_t> stack;
  for (uint64_t s = s_lo; s <= s_hi; ++s)
    if (mark[s] != g) {
      mark[s] = g;
      stack.push_back((uint32_t)s);
    }
  uint64_t edges = 0;
  while (!stack.empty()) {
    uint32_t s = stack.back();
    stack.pop_back();
    out.push_back(s);
    edges += A->dep_ptr[s + 1] - A->dep_ptr[s];
    if (max_edges && edges > max_edges) return false;
    for (uint64_t i = A->dep_ptr[s]; i < A->dep_ptr[s + 1]; ++i) {
      uint32_t d = A->deps[i];
      if (mark[d] != g) {
        mark[d] = g;
        stack.push_back(d);
      }
    }
  }
  return true;
}

bool closure(aceapex_archive *A, uint64_t s_lo, uint64_t s_hi, std::vector<uint32_t> &out, uint64_t max_edges) {
  return closure_with(A, s_lo, s_hi, A->mark, A->mark_gen, out, max_edges);
}

void closure_of(aceapex_archive *A, const uint32_t *seeds, uint64_t n, std::vector<uint32_t> &out) {
  if (A->mark.size() != A->h.n_seg) A->mark.assign(A->h.n_seg, 0);
  if (++A->mark_gen == 0) {
    std::fill(A->mark.begin(), A->mark.end(), 0);
    A->mark_gen = 1;
  }
  const uint32_t g = A->mark_gen;
  out.clear();
  std::vector<uint32_t> stack;
  for (uint64_t i = 0; i < n; ++i)
    if (A->mark[seeds[i]] != g) {
      A->mark[seeds[i]] = g;
      stack.push_back(seeds[i]);
    }
  while (!stack.empty()) {
    uint32_t s = stack.back();
    stack.pop_back();
    out.push_back(s);
    for (uint64_t i = A->dep_ptr[s]; i < A->dep_ptr[s + 1]; ++i) {
      uint32_t d = A->deps[i];
      if (A->mark[d] != g) {
        A->mark[d] = g;
        stack.push_back(d);
      }
    }
  }
}

// Host walks stop after this many dependency entries (tens of microseconds);
// wider closures are found on the device.
constexpr uint64_t kHostClosureEdges = 16384;

// The closure of [s_lo, s_hi] found on the device: the lists are uploaded on
// first use; the members of each level from the seeds' deepest level down to 1
// add their dependencies, then the members are sorted by level into d_work
// with their page-table slots. The member count comes back to the host (one
// stream synchronisation) so that the arena can be sized for it.
int device_closure(aceapex_archive *A, uint64_t s_lo, uint64_t s_hi, cudaStream_t st, uint32_t *n_out) {
  const uint64_t ns = A->h.n_seg;
  if (!A->d_dep_ptr.p) {
    if (A->d_dep_ptr.alloc(ns + 1) != cudaSuccess || A->d_deps.alloc(std::max<uint64_t>(A->h.n_deps, 1)) != cudaSuccess ||
        A->d_cmark.alloc(ns) != cudaSuccess || A->d_clist.alloc(ns) != cudaSuccess ||
        A->d_ccnt.alloc(4) != cudaSuccess || A->stage_cnt.reserve(16) != cudaSuccess)
      return ACEAPEX_ENOMEM;
    if (cudaMemcpy(A->d_dep_ptr.p, A->dep_ptr.data(), 8 * (ns + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        (A->h.n_deps &&
         cudaMemcpy(A->d_deps.p, A->deps.data(), 4 * A->h.n_deps, cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(A->d_cmark.p, 0, 4 * ns) != cudaSuccess ||
        cudaStreamSynchronize(0) != cudaSuccess)  // (st need not wait for the legacy stream)
      return ACEAPEX_ECUDA;
    A->cgen = 0;
  }
  if (A->d_work.n < ns) {
    cudaStreamSynchronize(st);
    if (A->d_work.alloc(ns) != cudaSuccess) return ACEAPEX_ENOMEM;
  }
  if (++A->cgen == 0) {  // tags wrapped: clear the marks
    if (cudaMemsetAsync(A->d_cmark.p, 0, 4 * ns, st) != cudaSuccess) return ACEAPEX_ECUDA;
    A->cgen = 1;
  }
  ClosureDev C{A->d_dep_ptr.p, A->d_deps.p, A->d_dir.p, A->d_cmark.p, A->d_clist.p, A->d_ccnt.p};
  uint32_t top = 0;
  for (uint64_t s = s_lo; s <= s_hi; ++s) top = std::max<uint32_t>(top, A->dir[s].level);
  cudaError_t e = launch_closure_seed(C, (uint32_t)s_lo, (uint32_t)(s_hi - s_lo + 1), A->cgen, st);
  for (uint32_t l = top; e == cudaSuccess && l >= 1; --l) e = launch_closure_expand(C, l, A->cgen, st);
  if (e == cudaSuccess) e = launch_closure_order(C, A->d_work.p, A->d_page.p, A->d_ccnt.p + 1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A->stage_cnt.p, A->d_ccnt.p + 1, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ACEAPEX_ECUDA;
  *n_out = *static_cast<const uint32_t *>(A->stage_cnt.p);
  return *n_out <= ns ? ACEAPEX_OK : ACEAPEX_ECUDA;
}

// decode the closure of [s_lo, s_hi] into arena slots (paged view); returns the view
int decode_closure(aceapex_archive *A, uint64_t s_lo, uint64_t s_hi, cudaStream_t st, OutView *view_out,
                   uint32_t *n_out, bool begin) {
  const uint64_t S = uint64_t(1) << A->h.log2_S;
  if (!A->d_page.p) {
    if (A->d_page.alloc(A->h.n_seg) != cudaSuccess) return ACEAPEX_ENOMEM;
    if (cudaMemsetAsync(A->d_page.p, 0xFF, 4 * A->h.n_seg, st) != cudaSuccess) return ACEAPEX_ECUDA;
  }
  std::vector<uint32_t> segs;
  if (!closure(A, s_lo, s_hi, segs, kHostClosureEdges)) {
    uint32_t n = 0;
    int rc = device_closure(A, s_lo, s_hi, st, &n);
    if (rc) return rc;
    if (A->d_arena.n < n * S) {
      cudaStreamSynchronize(st);
      if (A->d_arena.alloc(std::max<uint64_t>(n, 64) * S) != cudaSuccess) return ACEAPEX_ENOMEM;
    }
    uint32_t *ge = global_epoch(A->device);
    if (!ge) return ACEAPEX_ECUDA;
    cudaError_t e = begin ? launch_begin(ge, A->epoch(), A->counter(), st) : cudaMemsetAsync(A->counter(), 0, 4, st);
    if (e != cudaSuccess) return ACEAPEX_ECUDA;
    DecodeLaunch L = base_launch(A);
    OutView v{};
    v.page = A->d_page.p;
    v.slot_base = A->d_arena.p;
    L.view0 = v;
    L.work = A->d_work.p;
    L.n_work = n;
    if ((e = launch_decode(L, A->grid, kBlock, st)) != cudaSuccess) return ACEAPEX_ECUDA;
    *view_out = v;
    *n_out = n;
    return ACEAPEX_OK;
  }
  std::vector<WorkItem> work;
  level_order(A->dir, segs.data(), segs.size(), 0, work);
  if (A->d_arena.n < work.size() * S) {
    cudaStreamSynchronize(st);
    uint64_t slots = std::max<uint64_t>(work.size(), 64);
    if (A->d_arena.alloc(slots * S) != cudaSuccess) return ACEAPEX_ENOMEM;
  }
  if (A->d_work.n < work.size()) {
    cudaStreamSynchronize(st);
    if (A->d_work.alloc(std::max<uint64_t>(work.size(), 1024)) != cudaSuccess) return ACEAPEX_ENOMEM;
  }
  if (A->stage_work.reserve(work.size() * sizeof(WorkItem)) != cudaSuccess) return ACEAPEX_ENOMEM;
  std::memcpy(A->stage_work.p, work.data(), work.size() * sizeof(WorkItem));
  cudaError_t e = cudaMemcpyAsync(A->d_work.p, A->stage_work.p, work.size() * sizeof(WorkItem),
                                  cudaMemcpyHostToDevice, st);
  A->stage_work.mark(st);
  if (e != cudaSuccess) return ACEAPEX_ECUDA;
  if ((e = launch_set_pages(A->d_page.p, A->d_work.p, (uint32_t)work.size(), st)) != cudaSuccess) return ACEAPEX_ECUDA;
  uint32_t *ge = global_epoch(A->device);
  if (!ge) return ACEAPEX_ECUDA;
  if (begin && (e = launch_begin(ge, A->epoch(), A->counter(), st)) != cudaSuccess) return ACEAPEX_ECUDA;
  if (!begin && (e = cudaMemsetAsync(A->counter(), 0, 4, st)) != cudaSuccess) return ACEAPEX_ECUDA;
  DecodeLaunch L = base_launch(A);
  OutView v{};
  v.page = A->d_page.p;
  v.slot_base = A->d_arena.p;
  L.view0 = v;
  L.work = A->d_work.p;
  L.n_work = (uint32_t)work.size();
  if ((e = launch_decode(L, A->grid, kBlock, st)) != cudaSuccess) return ACEAPEX_ECUDA;
  *view_out = v;
  *n_out = (uint32_t)work.size();
  return ACEAPEX_OK;
}

}  // namespace aceapex

// ====================================================================== C ABI

extern "C" {

}  // extern "C"

namespace aceapex {

// Payload pieces of an upload that decoding may overtake (aceapex_decode_host).
constexpr uint64_t kUploadPiece = uint64_t(32) << 20;
// Default window of a decode to host memory: the first window's decode is
// all that precedes the first copy back, so windows are kept short.
constexpr uint64_t kHostWindow = uint64_t(64) << 20;

int upload_pieces(aceapex_archive *A, const uint8_t *src, uint64_t bytes, uint64_t limit);

// Payload bytes a one-call decode uploads before its host checks: what the
// first windows read, so that their decodes need not wait for the rest
constexpr uint64_t kEarlyUpload = 2 * kUploadPiece;

// aceapex_open. With defer_payload (aceapex_decode_host) the host checks
// leave out the dependency lists and the read index, which a whole-file
// decode does not read, no whole-file work list is made (the windows have
// their own), and only the payload's first pieces are copied while the host
// checks run: start_payload_upload copies the rest afterwards, once the small
// sections are on their way, so that their copies do not queue behind it.
int open_archive(const void *h_archive, uint64_t nbytes, int device, aceapex_archive **out, bool defer_payload) {
  if (!h_archive || !out || nbytes == 0) return ACEAPEX_EINVAL;
  *out = nullptr;
  aceapex_archive *A = new (std::nothrow) aceapex_archive();
  if (!A) return ACEAPEX_ENOMEM;
  const uint8_t *a = static_cast<const uint8_t *>(h_archive);
  A->device = device;
  const bool dev_ok = cudaSetDevice(device) == cudaSuccess;  // reported after validation
  // Unless deferred, the payload (almost all of the archive) goes to the
  // device while the host checks the rest: its place and size come from the
  // header, checked against the buffer size first; the copy is waited for
  // before any return.
  uint64_t pay_off = 0, pay_bytes = 0;
  if (nbytes >= kHeaderBytes) {
    pay_off = rd<uint64_t>(a + 104);
    pay_bytes = rd<uint64_t>(a + 112);
    if (pay_off > nbytes || pay_bytes > nbytes - pay_off) pay_off = pay_bytes = 0;
  }
  cudaStream_t up = nullptr;
  bool uploading = false;
  if (!defer_payload && dev_ok && pay_bytes && cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) == cudaSuccess &&
      A->d_payload.alloc(pay_bytes) == cudaSuccess &&
      cudaMemcpyAsync(A->d_payload.p, a + pay_off, pay_bytes, cudaMemcpyHostToDevice, up) == cudaSuccess)
    uploading = true;
  bool early = false;
  if (defer_payload && dev_ok && pay_bytes && A->d_payload.alloc(pay_bytes) == cudaSuccess &&
      upload_pieces(A, a + pay_off, pay_bytes, kEarlyUpload) == ACEAPEX_OK)
    early = true;
  int rc = validate(a, nbytes, A, !defer_payload);
  const bool upload_ok = !uploading || cudaStreamSynchronize(up) == cudaSuccess;
  if (up) cudaStreamDestroy(up);
  if (rc || !upload_ok || !dev_ok) {
    A->release();
    delete A;
    return rc ? rc : ACEAPEX_ECUDA;
  }
  std::vector<uint32_t> lut;
  build_lut(a, lut);
  std::vector<WorkItem> order;
  if (!defer_payload) level_order(A->dir, nullptr, A->h.n_seg, 0, order);
  const Header &h = A->h;
  // (the payload buffer is the uploaded one when the header's payload fields
  // were what validation accepted, else it is allocated and copied now)
  const bool have_payload = (uploading || early) && pay_off == h.off_payload && pay_bytes == h.payload_bytes;
  bool okm = (have_payload || A->d_payload.alloc(std::max<uint64_t>(h.payload_bytes, 16)) == cudaSuccess) &&
             A->d_dir.alloc(std::max<uint64_t>(h.n_seg, 1)) == cudaSuccess &&
             A->d_lut.alloc(4 * kScale) == cudaSuccess && A->d_flags.alloc(std::max<uint64_t>(h.n_seg, 1)) == cudaSuccess &&
             (defer_payload || A->d_order.alloc(std::max<uint64_t>(h.n_seg, 1)) == cudaSuccess) &&
             A->d_words.alloc(4) == cudaSuccess &&
             A->d_blocked.alloc(std::max<uint64_t>(h.n_seg, 1)) == cudaSuccess;
  if (!okm || !global_epoch(device)) {
    A->release();
    delete A;
    return ACEAPEX_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  if (h.payload_bytes && !have_payload && !defer_payload)
    e = cudaMemcpy(A->d_payload.p, a + h.off_payload, h.payload_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && h.n_seg) e = cudaMemcpy(A->d_dir.p, A->dir.data(), 24 * h.n_seg, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(A->d_lut.p, lut.data(), 4 * lut.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && h.n_seg && !defer_payload)
    e = cudaMemcpy(A->d_order.p, order.data(), sizeof(WorkItem) * h.n_seg, cudaMemcpyHostToDevice);
  // each segment's flag word starts with its level and no epoch (made on the
  // device from the directory copied above, on the legacy stream, which
  // orders it before the synchronous copies below)
  if (e == cudaSuccess) e = launch_init_flags(A->d_flags.p, A->d_dir.p, h.n_seg, 0);
  if (e == cudaSuccess) e = cudaMemset(A->d_words.p, 0, 16);
  if (e == cudaSuccess) e = cudaMemset(A->d_blocked.p, 0, std::max<uint64_t>(h.n_seg, 1));
  // (the caller's streams need not synchronise with the legacy stream)
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    A->release();
    delete A;
    return ACEAPEX_ECUDA;
  }
  *out = A;
  return ACEAPEX_OK;
}

// Payload bytes [issued, min(limit, bytes)) of a handle opened with
// defer_payload, in pieces on the handle's upload stream, each followed by an
// event (up_ev / up_end); src is the payload in host memory.
int upload_pieces(aceapex_archive *A, const uint8_t *src, uint64_t bytes, uint64_t limit) {
  if (!bytes) return ACEAPEX_OK;
  if (!A->up_st && cudaStreamCreateWithFlags(&A->up_st, cudaStreamNonBlocking) != cudaSuccess) return ACEAPEX_ECUDA;
  const uint64_t end = std::min(limit, bytes);
  for (uint64_t o = A->up_end.empty() ? 0 : A->up_end.back(); o < end; o += kUploadPiece) {
    const uint64_t n = std::min(kUploadPiece, bytes - o);
    cudaEvent_t ev = nullptr;
    if (cudaMemcpyAsync(A->d_payload.p + o, src + o, n, cudaMemcpyHostToDevice, A->up_st) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return ACEAPEX_ECUDA;
    A->up_ev.push_back(ev);
    A->up_end.push_back(o + n);
    if (cudaEventRecord(ev, A->up_st) != cudaSuccess) return ACEAPEX_ECUDA;
  }
  return ACEAPEX_OK;
}

// the rest of the payload of a handle opened with defer_payload
int start_payload_upload(aceapex_archive *A, const void *h_archive) {
  return upload_pieces(A, static_cast<const uint8_t *>(h_archive) + A->h.off_payload, A->h.payload_bytes,
                       ~uint64_t(0));
}


// What a decode to host memory needs besides the archive, for windows of
// `window` bytes (a multiple of the segment size): scratch, the device
// output buffer, the copy stream, the windows' work lists in level order
// (built once per window size) and their events.
int prepare_windows(aceapex_archive *a, uint64_t window, cudaStream_t st) {
  const uint64_t S = uint64_t(1) << a->h.log2_S;
  int rc = ensure_scratch(a);
  if (rc) return rc;
  if (a->d_host_out.n < a->h.n) {
    cudaStreamSynchronize(st);
    if (a->d_host_out.alloc(a->h.n) != cudaSuccess) return ACEAPEX_ENOMEM;
  }
  if (!a->copy_st && cudaStreamCreateWithFlags(&a->copy_st, cudaStreamNonBlocking) != cudaSuccess)
    return ACEAPEX_ECUDA;
  if (a->win_bytes != window) {
    // (work made for another window size may still be queued)
    cudaStreamSynchronize(st);
    // window k is segments [k per, (k + 1) per), and its work list sits at
    // the same place of the window lists, made on the device
    const uint64_t per = window / S;
    a->win_start.clear();
    for (uint64_t s = 0; s < a->h.n_seg; s += per) a->win_start.push_back(s);
    a->win_start.push_back(a->h.n_seg);
    if (a->d_win_work.alloc(std::max<uint64_t>(a->h.n_seg, 1)) != cudaSuccess) return ACEAPEX_ENOMEM;
    if (launch_window_order(a->d_dir.p, a->h.n_seg, per, a->stats.max_level, a->d_win_work.p, st) != cudaSuccess)
      return ACEAPEX_ECUDA;
    a->win_bytes = window;
  }
  const size_t nwin = a->win_start.size() - 1;
  while (a->win_ev.size() < nwin + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return ACEAPEX_ECUDA;
    a->win_ev.push_back(e);
  }
  return ACEAPEX_OK;
}

}  // namespace aceapex

extern "C" {

int aceapex_open(const void *h_archive, uint64_t nbytes, int device, aceapex_archive **out) {
  return open_archive(h_archive, nbytes, device, out, false);
}

void aceapex_close(aceapex_archive *a) {
  if (!a) return;
  cudaSetDevice(a->device);
  cudaDeviceSynchronize();
  a->release();
  delete a;
}

int aceapex_release_cached_memory(int device) {
  DevPool *P = pool_of(device);
  if (!P) return ACEAPEX_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != device && cudaSetDevice(device) != cudaSuccess) return ACEAPEX_ECUDA;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(P->pool, 0);
  if (cur != device) cudaSetDevice(cur);
  return cuda_status(e);
}

uint64_t aceapex_decoded_size(const aceapex_archive *a) { return a ? a->h.n : 0; }

int aceapex_level_counts(const aceapex_archive *a, uint64_t *h_counts, uint32_t n) {
  if (!a || (!h_counts && n)) return ACEAPEX_EINVAL;
  for (uint32_t l = 0; l < n; ++l) h_counts[l] = 0;
  for (const SegRec &r : a->dir)
    if (r.level < n) h_counts[r.level]++;
  return ACEAPEX_OK;
}

int aceapex_get_stats(const aceapex_archive *a, aceapex_stats *st) {
  if (!a || !st) return ACEAPEX_EINVAL;
  *st = a->stats;
  return ACEAPEX_OK;
}

int aceapex_decode_all(aceapex_archive *a, void *d_out, uint64_t out_cap, void *stream, aceapex_stats *opt_stats) {
  if (!a || (!d_out && a->h.n)) return ACEAPEX_EINVAL;
  if (out_cap < a->h.n) return ACEAPEX_ERANGE;
  if (opt_stats) *opt_stats = a->stats;
  if (a->h.n == 0) return ACEAPEX_OK;
  if (cudaSetDevice(a->device) != cudaSuccess) return ACEAPEX_ECUDA;
  int rc = ensure_scratch(a);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t *ge = global_epoch(a->device);
  if (!ge) return ACEAPEX_ECUDA;
  cudaError_t e = launch_begin(ge, a->epoch(), a->counter(), st);
  if (e != cudaSuccess) return ACEAPEX_ECUDA;
  DecodeLaunch L = base_launch(a);
  L.view0 = linear_view(static_cast<uint8_t *>(d_out), 0);
  L.work = a->d_order.p;
  L.n_work = (uint32_t)a->h.n_seg;
  return cuda_status(launch_decode(L, a->grid, kBlock, st));
}

int aceapex_decode_all_to_host(aceapex_archive *a, void *h_out, uint64_t out_cap, uint64_t window, void *stream) {
  if (!a || (!h_out && a->h.n)) return ACEAPEX_EINVAL;
  if (out_cap < a->h.n) return ACEAPEX_ERANGE;
  if (a->h.n == 0) return ACEAPEX_OK;
  const uint64_t S = uint64_t(1) << a->h.log2_S;
  if (window == 0) window = kHostWindow;
  window = std::max<uint64_t>(S, window / S * S);
  if (cudaSetDevice(a->device) != cudaSuccess) return ACEAPEX_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = prepare_windows(a, window, st);
  if (rc) return rc;
  const size_t nwin = a->win_start.size() - 1;
  uint32_t *ge = global_epoch(a->device);
  if (!ge) return ACEAPEX_ECUDA;
  // the copy stream starts after the caller's earlier work
  cudaError_t e = cudaEventRecord(a->win_ev[nwin], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(a->copy_st, a->win_ev[nwin], 0);
  DecodeLaunch L = base_launch(a);
  L.view0 = linear_view(a->d_host_out.p, 0);
  uint8_t *host = static_cast<uint8_t *>(h_out);
  // window k decodes on `stream` (its sources lie in windows <= k, already
  // complete with this call's epoch) while window k - 1 is copied out
  for (size_t k = 0; k < nwin && e == cudaSuccess; ++k) {
    e = k == 0 ? launch_begin(ge, a->epoch(), a->counter(), st) : cudaMemsetAsync(a->counter(), 0, 4, st);
    if (e != cudaSuccess) break;
    L.work = a->d_win_work.p + a->win_start[k];
    L.n_work = (uint32_t)(a->win_start[k + 1] - a->win_start[k]);
    if (!a->up_ev.empty()) {
      // a payload upload still in flight: wait for the piece that completes
      // this window's payload (segments are laid out in order; the last one's
      // words end the window's part)
      const uint64_t s_last = std::min<uint64_t>(a->h.n_seg, (k + 1) * window / S + ((k + 1) * window % S ? 1 : 0)) - 1;
      const SegRec &r = a->dir[s_last];
      const uint64_t need = (r.payload_off + 128 + 2 * (uint64_t)r.n_words + 15) & ~uint64_t(15);
      size_t i = 0;
      while (i + 1 < a->up_end.size() && a->up_end[i] < need) ++i;
      if ((e = cudaStreamWaitEvent(st, a->up_ev[i], 0)) != cudaSuccess) break;
    }
    if ((e = launch_decode(L, a->grid, kBlock, st)) != cudaSuccess) break;
    if ((e = cudaEventRecord(a->win_ev[k], st)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(a->copy_st, a->win_ev[k], 0)) != cudaSuccess) break;
    const uint64_t lo = (uint64_t)k * window, hi = std::min(a->h.n, lo + window);
    e = cudaMemcpyAsync(host + lo, a->d_host_out.p + lo, hi - lo, cudaMemcpyDeviceToHost, a->copy_st);
  }
  // the caller's stream waits for the last copy
  if (e == cudaSuccess) e = cudaEventRecord(a->win_ev[nwin], a->copy_st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, a->win_ev[nwin], 0);
  return cuda_status(e);
}

int aceapex_decode_host(const void *h_archive, uint64_t nbytes, int device, void *h_out, uint64_t out_cap,
                        uint64_t window) {
  if (!h_archive || nbytes == 0) return ACEAPEX_EINVAL;
  aceapex_archive *A = nullptr;
  int rc = open_archive(h_archive, nbytes, device, &A, true);
  if (rc) return rc;
  if (!h_out && A->h.n) rc = ACEAPEX_EINVAL;
  else if (out_cap < A->h.n) rc = ACEAPEX_ERANGE;
  cudaStream_t st = nullptr;
  if (!rc && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = ACEAPEX_ECUDA;
  if (rc) {
    aceapex_close(A);
    return rc;
  }
  // everything the windows need goes to the device before the payload, whose
  // pieces the window decodes then follow
  const uint64_t S = uint64_t(1) << A->h.log2_S;
  const uint64_t win = std::max<uint64_t>(S, (window ? window : kHostWindow) / S * S);
  if (A->h.n) rc = prepare_windows(A, win, st);
  if (!rc) rc = start_payload_upload(A, h_archive);
  if (!rc) rc = aceapex_decode_all_to_host(A, h_out, out_cap, window, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (!rc) rc = e == cudaSuccess ? aceapex_last_error(A, 0, nullptr) : ACEAPEX_ECUDA;
  cudaStreamDestroy(st);
  aceapex_close(A);
  return rc;
}

int aceapex_decode_range(aceapex_archive *a, uint64_t lo, uint64_t hi, void *d_out, uint64_t out_cap, void *stream) {
  if (!a || (!d_out && hi > lo)) return ACEAPEX_EINVAL;
  if (lo > hi || hi > a->h.n || out_cap < hi - lo) return ACEAPEX_ERANGE;
  if (hi == lo) return ACEAPEX_OK;
  if (cudaSetDevice(a->device) != cudaSuccess) return ACEAPEX_ECUDA;
  int rc = ensure_scratch(a);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  OutView v;
  uint32_t n = 0;
  rc = decode_closure(a, lo >> a->h.log2_S, (hi - 1) >> a->h.log2_S, st, &v, &n, true);
  if (rc) return rc;
  cudaError_t e = launch_gather(v, a->h.log2_S, lo, hi, static_cast<uint8_t *>(d_out), st);
  if (e == cudaSuccess) e = launch_clear_pages(a->d_page.p, a->d_work.p, n, st);
  return cuda_status(e);
}

int aceapex_range_closure(aceapex_archive *a, uint64_t lo, uint64_t hi, uint64_t *n_segments, uint32_t *max_level) {
  if (!a || !n_segments) return ACEAPEX_EINVAL;
  if (lo > hi || hi > a->h.n) return ACEAPEX_ERANGE;
  *n_segments = 0;
  if (max_level) *max_level = 0;
  if (hi == lo) return ACEAPEX_OK;
  std::vector<uint32_t> segs;
  closure(a, lo >> a->h.log2_S, (hi - 1) >> a->h.log2_S, segs);
  uint32_t lv = 0;
  for (uint32_t s : segs) lv = std::max<uint32_t>(lv, a->dir[s].level);
  *n_segments = segs.size();
  if (max_level) *max_level = lv;
  return ACEAPEX_OK;
}

int aceapex_read_lookup(const aceapex_archive *a, uint64_t read_id, uint64_t *byte_lo, uint64_t *byte_hi) {
  if (!a || !byte_lo || !byte_hi || a->h.n_reads == 0) return ACEAPEX_EINVAL;
  if (read_id >= a->h.n_reads) return ACEAPEX_ERANGE;
  *byte_lo = a->reads[read_id];
  *byte_hi = read_id + 1 < a->h.n_reads ? a->reads[read_id + 1] : a->h.n;
  return ACEAPEX_OK;
}

int aceapex_region_lookup(const aceapex_archive *a, uint64_t chrom, uint64_t pos, uint64_t len, uint32_t line_width,
                          uint64_t *byte_lo, uint64_t *byte_hi) {
  if (!a || !byte_lo || !byte_hi || line_width == 0 || len == 0) return ACEAPEX_EINVAL;
  const uint64_t n_idx = a->h.n_reads, n_rec = n_idx / 2;
  if (n_rec == 0) return ACEAPEX_EINVAL;  // not a coordinate index
  if (chrom >= n_rec) return ACEAPEX_ERANGE;
  const uint64_t seq = a->reads[2 * chrom + 1];
  const bool last_rec = chrom + 1 == n_rec;
  const uint64_t end = last_rec ? a->h.n : a->reads[2 * chrom + 2];
  if (end < seq) return ACEAPEX_ECORRUPT;
  // B bases in lines of line_width, each line ending in a newline, take
  // B + ceil(B / line_width) bytes; when the file's last line has no
  // newline (an odd entry count marks it), the last record takes
  // B + floor(B / line_width) bytes, less one if B is a whole number of lines
  const uint64_t bytes = end - seq;
  const uint64_t bases = last_rec && (n_idx & 1) ? bytes - bytes / (line_width + 1)
                                             : bytes - (bytes + line_width) / (line_width + 1);
  if (pos >= bases || len > bases - pos) return ACEAPEX_ERANGE;
  const uint64_t last = pos + len - 1;
  *byte_lo = seq + pos + pos / line_width;
  *byte_hi = seq + last + last / line_width + 1;
  return ACEAPEX_OK;
}

int aceapex_decode_region(aceapex_archive *a, uint64_t chrom, uint64_t pos, uint64_t len, uint32_t line_width,
                          void *d_out, uint64_t out_cap, void *stream) {
  uint64_t lo = 0, hi = 0;
  int rc = aceapex_region_lookup(a, chrom, pos, len, line_width, &lo, &hi);
  if (rc) return rc;
  if (!d_out) return ACEAPEX_EINVAL;
  if (out_cap < len) return ACEAPEX_ERANGE;
  if (cudaSetDevice(a->device) != cudaSuccess) return ACEAPEX_ECUDA;
  if ((rc = ensure_scratch(a))) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  OutView v;
  uint32_t n = 0;
  rc = decode_closure(a, lo >> a->h.log2_S, (hi - 1) >> a->h.log2_S, st, &v, &n, true);
  if (rc) return rc;
  cudaError_t e = launch_gather_bases(v, a->h.log2_S, lo, (uint32_t)(pos % line_width), line_width, len,
                                      static_cast<uint8_t *>(d_out), st);
  if (e == cudaSuccess) e = launch_clear_pages(a->d_page.p, a->d_work.p, n, st);
  return cuda_status(e);
}

int aceapex_last_error(aceapex_archive *a, int sync, void *stream) {
  if (!a) return ACEAPEX_EINVAL;
  if (cudaSetDevice(a->device) != cudaSuccess) return ACEAPEX_ECUDA;
  cudaError_t e = sync ? (stream ? cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) : cudaDeviceSynchronize())
                       : cudaSuccess;
  if (e != cudaSuccess) return ACEAPEX_ECUDA;
  uint32_t v = 0;
  if (cudaMemcpy(&v, a->err(), 4, cudaMemcpyDeviceToHost) != cudaSuccess) return ACEAPEX_ECUDA;
  // (cleared on the legacy stream, which later non-blocking streams do not wait for)
  if (v && (cudaMemset(a->err(), 0, 4) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess))
    return ACEAPEX_ECUDA;
  return v == 0 ? ACEAPEX_OK : (int)v;
}

int aceapex_set_wait_limit(aceapex_archive *a, uint64_t ns) {
  if (!a) return ACEAPEX_EINVAL;
  a->wait_ns = ns ? ns : kDefaultWaitNs;
  return ACEAPEX_OK;
}

int aceapex_set_launch(aceapex_archive *a, uint32_t ctas, uint32_t warps_per_cta, uint32_t stage_bytes) {
  if (!a || warps_per_cta > kDecodeThreads / 32 || stage_bytes > kSmemStage) return ACEAPEX_EINVAL;
  if (cudaSetDevice(a->device) != cudaSuccess) return ACEAPEX_ECUDA;
  int rc = ensure_scratch(a, 0);
  if (rc) return rc;
  a->grid = (ctas == 0 || (int)ctas > a->max_grid) ? a->max_grid : (int)ctas;
  a->active_warps = warps_per_cta ? warps_per_cta : kDecodeThreads / 32;
  a->stage_cap = stage_bytes ? stage_bytes : kSmemStage;
  return ensure_scratch(a);
}

int aceapex_get_launch(const aceapex_archive *a, uint32_t *ctas, uint32_t *max_ctas, uint32_t *warps_per_cta,
                       uint32_t *stage_bytes) {
  if (!a || !ctas || !max_ctas || !warps_per_cta || !stage_bytes) return ACEAPEX_EINVAL;
  *ctas = (uint32_t)a->grid;
  *max_ctas = (uint32_t)a->max_grid;
  *warps_per_cta = a->active_warps;
  *stage_bytes = a->stage_cap;
  return ACEAPEX_OK;
}

int aceapex_debug_block_segments(aceapex_archive *a, const uint32_t *segs, uint32_t n) {
  if (!a || (n && !segs)) return ACEAPEX_EINVAL;
  for (uint32_t i = 0; i < n; ++i)
    if (segs[i] >= a->h.n_seg) return ACEAPEX_ERANGE;
  if (cudaSetDevice(a->device) != cudaSuccess) return ACEAPEX_ECUDA;
  std::vector<uint8_t> b(std::max<uint64_t>(a->h.n_seg, 1), 0);
  for (uint32_t i = 0; i < n; ++i) b[segs[i]] = 1;
  if (cudaMemcpy(a->d_blocked.p, b.data(), b.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess)
    return ACEAPEX_ECUDA;
  a->any_blocked = n != 0;
  return ACEAPEX_OK;
}

int aceapex_stream_range(aceapex_archive *a, uint64_t lo, uint64_t hi, uint64_t ring_bytes, uint64_t window,
                         uint32_t *d_crc, void *stream) {
  if (!a || !d_crc) return ACEAPEX_EINVAL;
  const Header &h = a->h;
  const uint64_t S = uint64_t(1) << h.log2_S;
  if (h.D == 0 || window == 0 || window % S || lo % S) return ACEAPEX_EINVAL;
  if (lo > hi || hi > h.n) return ACEAPEX_ERANGE;
  if (hi == lo) return ACEAPEX_OK;
  if (ring_bytes & (ring_bytes - 1)) return ACEAPEX_EINVAL;
  if (ring_bytes < window + round16(h.D) + 2 * S) return ACEAPEX_EINVAL;
  if (cudaSetDevice(a->device) != cudaSuccess) return ACEAPEX_ECUDA;
  int rc = ensure_scratch(a);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (a->d_ring.n != ring_bytes) {
    cudaStreamSynchronize(st);
    if (a->d_ring.alloc(ring_bytes) != cudaSuccess) return ACEAPEX_ENOMEM;
  }
  const uint64_t seg_per_win = window / S + 1;
  if (a->d_seg_crc.n < seg_per_win) {
    cudaStreamSynchronize(st);
    if (a->d_seg_crc.alloc(seg_per_win) != cudaSuccess) return ACEAPEX_ENOMEM;
  }
  OutView ring{};
  ring.base = a->d_ring.p;
  ring.origin = 0;
  ring.mask = ring_bytes - 1;
  uint32_t *ge = global_epoch(a->device);
  if (!ge) return ACEAPEX_ECUDA;
  cudaError_t e = cudaSuccess;
  bool begun = false;
  // prime: bytes [lo - D, lo) must be in the ring with this call's epoch
  if (lo > 0) {
    uint64_t p0 = lo > h.D ? ((lo - h.D) & ~(S - 1)) : 0;
    OutView v;
    uint32_t n = 0;
    rc = decode_closure(a, p0 >> h.log2_S, (lo - 1) >> h.log2_S, st, &v, &n, true);
    if (rc) return rc;
    begun = true;
    if ((e = launch_copy_view(v, ring, h.log2_S, p0, lo, st)) != cudaSuccess) return ACEAPEX_ECUDA;
    if ((e = launch_clear_pages(a->d_page.p, a->d_work.p, n, st)) != cudaSuccess) return ACEAPEX_ECUDA;
  }
  // all windows' work lists, uploaded once
  const uint64_t s_lo = lo >> h.log2_S, s_hi = (hi - 1) >> h.log2_S, ns = s_hi - s_lo + 1;
  std::vector<WorkItem> work;
  work.reserve(ns);
  std::vector<uint64_t> wstart;
  std::vector<uint32_t> segs;
  for (uint64_t wa = lo; wa < hi; wa += window) {
    uint64_t wb = std::min(hi, wa + window);
    segs.clear();
    for (uint64_t s = wa >> h.log2_S; s <= (wb - 1) >> h.log2_S; ++s) segs.push_back((uint32_t)s);
    wstart.push_back(work.size());
    level_order(a->dir, segs.data(), segs.size(), 0, work);
  }
  wstart.push_back(work.size());
  if (a->d_work.n < work.size()) {
    cudaStreamSynchronize(st);
    if (a->d_work.alloc(work.size()) != cudaSuccess) return ACEAPEX_ENOMEM;
  }
  if (a->stage_work.reserve(work.size() * sizeof(WorkItem)) != cudaSuccess) return ACEAPEX_ENOMEM;
  std::memcpy(a->stage_work.p, work.data(), work.size() * sizeof(WorkItem));
  e = cudaMemcpyAsync(a->d_work.p, a->stage_work.p, work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, st);
  a->stage_work.mark(st);
  if (e != cudaSuccess) return ACEAPEX_ECUDA;
  DecodeLaunch L = base_launch(a);
  L.view0 = ring;
  for (size_t k = 0; k + 1 < wstart.size(); ++k) {
    uint64_t wa = lo + k * window, wb = std::min(hi, wa + window);
    if (!begun) {
      e = launch_begin(ge, a->epoch(), a->counter(), st);
      begun = true;
    } else {
      e = cudaMemsetAsync(a->counter(), 0, 4, st);
    }
    if (e != cudaSuccess) return ACEAPEX_ECUDA;
    L.work = a->d_work.p + wstart[k];
    L.n_work = (uint32_t)(wstart[k + 1] - wstart[k]);
    if ((e = launch_decode(L, a->grid, kBlock, st)) != cudaSuccess) return ACEAPEX_ECUDA;
    if ((e = launch_window_crc(ring, wa, wb, window, d_crc + k, a->d_seg_crc.p, h.log2_S, st)) != cudaSuccess)
      return ACEAPEX_ECUDA;
  }
  return ACEAPEX_OK;
}

int aceapex_decode_batch(aceapex_archive *const *as, int n, void *const *d_outs, void *stream) {
  if (!as || !d_outs || n <= 0) return ACEAPEX_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!as[i] || as[i]->device != as[0]->device || (!d_outs[i] && as[i]->h.n)) return ACEAPEX_EINVAL;
  aceapex_archive *A = as[0];
  if (cudaSetDevice(A->device) != cudaSuccess) return ACEAPEX_ECUDA;
  uint32_t need = 0;
  for (int i = 0; i < n; ++i) need = std::max(need, as[i]->max_cmd_syms);
  int rc = ensure_scratch(A, need);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // largest archives first, so the last CTAs to finish hold small ones
  std::vector<int> perm;
  for (int i = 0; i < n; ++i)
    if (as[i]->h.n_seg) perm.push_back(i);
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return as[x]->h.n_seg > as[y]->h.n_seg; });
  const uint32_t m = (uint32_t)perm.size();
  if (m == 0) return ACEAPEX_OK;
  std::vector<DevArchive> arcs(m);
  std::vector<OutView> views(m);
  for (uint32_t k = 0; k < m; ++k) {
    arcs[k] = as[perm[k]]->dev();
    views[k] = linear_view(static_cast<uint8_t *>(d_outs[perm[k]]), 0);
  }
  // the device copy of the batch description is reused while it is unchanged,
  // so a repeated call (or its capture into a CUDA graph) issues kernels only
  const uint64_t bytes = (sizeof(DevArchive) + sizeof(OutView)) * m;
  std::vector<uint8_t> desc(bytes);
  std::memcpy(desc.data(), arcs.data(), sizeof(DevArchive) * m);
  std::memcpy(desc.data() + sizeof(DevArchive) * m, views.data(), sizeof(OutView) * m);
  if (desc != A->batch_desc) {
    if (A->d_batch_arcs.n < m) {
      cudaStreamSynchronize(st);
      if (A->d_batch_arcs.alloc(m) != cudaSuccess || A->d_batch_views.alloc(m) != cudaSuccess) return ACEAPEX_ENOMEM;
    }
    if (A->stage_batch.reserve(bytes) != cudaSuccess) return ACEAPEX_ENOMEM;
    uint8_t *p = static_cast<uint8_t *>(A->stage_batch.p);
    std::memcpy(p, desc.data(), bytes);
    cudaError_t e = cudaMemcpyAsync(A->d_batch_arcs.p, p, sizeof(DevArchive) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(A->d_batch_views.p, p + sizeof(DevArchive) * m, sizeof(OutView) * m,
                          cudaMemcpyHostToDevice, st);
    A->stage_batch.mark(st);
    if (e != cudaSuccess) return ACEAPEX_ECUDA;
    A->batch_desc.swap(desc);
  }
  uint32_t *ge = global_epoch(A->device);
  if (!ge || launch_begin(ge, A->epoch(), A->counter(), st) != cudaSuccess) return ACEAPEX_ECUDA;
  DecodeLaunch L = base_launch(A);
  L.arcs = A->d_batch_arcs.p;
  L.views = A->d_batch_views.p;
  return cuda_status(launch_batch(L, m, A->grid, st));
}

int aceapex_encode(const void *h_in, uint64_t n, uint32_t log2_B, uint32_t min_match, uint32_t max_level,
                   uint64_t dist_bound, const uint64_t *h_reads, uint64_t n_reads, int threads, void **h_out,
                   uint64_t *out_len) {
  if (!h_out || !out_len || (n && !h_in) || (n_reads && !h_reads)) return ACEAPEX_EINVAL;
  uint8_t *o = nullptr;
  int rc = encode_archive(static_cast<const uint8_t *>(h_in), n, log2_B, min_match, max_level, dist_bound, h_reads,
                          n_reads, threads, &o, out_len);
  *h_out = o;
  return rc;
}

void aceapex_free(void *p) { std::free(p); }

uint64_t aceapex_fastq_split(const void *h_in, uint64_t n, void *h_out, uint64_t *h_lens) {
  if (!h_in || !h_out || !h_lens) return 0;
  return fastq_split(static_cast<const uint8_t *>(h_in), n, static_cast<uint8_t *>(h_out), h_lens);
}

int aceapex_decode_fastq_streams(aceapex_archive *const *parts, void *d_out, uint64_t out_cap, void *stream) {
  if (!parts) return ACEAPEX_EINVAL;
  for (int k = 0; k < 4; ++k)
    if (!parts[k] || parts[k]->device != parts[0]->device) return ACEAPEX_EINVAL;
  aceapex_archive *A = parts[0];
  uint64_t len[4], N = 0, chunks_max = 0, offs_n = 0, cap[4], nl_n = 0;
  for (int k = 0; k < 4; ++k) {
    len[k] = parts[k]->h.n;
    if (len[k] >= (uint64_t(1) << 32)) return ACEAPEX_ERANGE;  // u32 newline positions
    N += len[k];
    const uint64_t chunks = (len[k] + 65535) / 65536;
    chunks_max = std::max(chunks_max, chunks);
    offs_n += chunks + 1;
    cap[k] = len[k] / 2 + 1;  // FASTQ lines are at least 2 bytes long
    nl_n += cap[k];
  }
  if (!d_out && N) return ACEAPEX_EINVAL;
  if (out_cap < N) return ACEAPEX_ERANGE;
  if (N == 0) return ACEAPEX_OK;
  if (cudaSetDevice(A->device) != cudaSuccess) return ACEAPEX_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (A->d_fq_streams.n < N || A->d_fq_counts.n < chunks_max || A->d_fq_offs.n < offs_n || A->d_fq_nl.n < nl_n) {
    cudaStreamSynchronize(st);
    if (A->d_fq_streams.alloc(N) != cudaSuccess || A->d_fq_counts.alloc(std::max<uint64_t>(chunks_max, 1)) != cudaSuccess ||
        A->d_fq_offs.alloc(offs_n) != cudaSuccess || A->d_fq_nl.alloc(nl_n) != cudaSuccess)
      return ACEAPEX_ENOMEM;
  }
  void *outs[4];
  const uint8_t *base[4];
  uint32_t *nl[4];
  uint64_t at = 0, nat = 0;
  for (int k = 0; k < 4; ++k) {
    outs[k] = A->d_fq_streams.p + at;
    base[k] = A->d_fq_streams.p + at;
    nl[k] = A->d_fq_nl.p + nat;
    at += len[k];
    nat += cap[k];
  }
  // each part fills the whole GPU with its own persistent launch (a batch
  // launch would give each of the four archives a single CTA)
  for (int k = 0; k < 4; ++k) {
    if (!len[k]) continue;
    int rc = aceapex_decode_all(parts[k], outs[k], len[k], stream, nullptr);
    if (rc) return rc;
  }
  return cuda_status(launch_fastq_interleave(base, len, A->d_fq_counts.p, A->d_fq_offs.p, nl, cap, A->err(),
                                             static_cast<uint8_t *>(d_out), st));
}

uint64_t aceapex_fasta_index(const void *h_in, uint64_t n, uint64_t *h_out, uint64_t cap, uint32_t *line_width) {
  if (!h_in) return 0;
  return fasta_index(static_cast<const uint8_t *>(h_in), n, h_out, cap, line_width);
}

uint64_t aceapex_fastq_index(const void *h_in, uint64_t n, uint64_t *h_out, uint64_t cap) {
  if (!h_in) return 0;
  return fastq_index(static_cast<const uint8_t *>(h_in), n, h_out, cap);
}

}  // extern "C"
