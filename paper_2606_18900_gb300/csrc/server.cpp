// Serving engine: continuous batching of range and read requests over
// device-resident archives (the serving pattern of the method's random access,
// paper §4 and §4.1, applied to many concurrent requests).
//
// One worker thread owns the GPU side. A submitted request goes to a pool of
// walker threads, which compute its transitive source closure (each with its
// own marks) and then append it to a FIFO queue; a submission itself only
// enqueues, so callers can offer requests at their own rate. Whenever
// one of `slots` batch slots is free, the worker takes requests from the head
// of the queue while the union of their closures fits the slot's decode arena
// (the device-memory budget is split evenly over the slots), then on the
// slot's own stream: uploads the level-ordered work lists, decodes each
// archive's union with one persistent launch through a page table of the
// slot, gathers every request's bytes into its caller buffer with one launch,
// clears the page entries and records an event. Requests that arrive while
// batches run join the next batch on another slot, so several batches overlap
// on the device. Each slot has its own page tables, ready flags and control
// words, so batches never share per-segment state. Completion is observed by
// polling the slots' events; a request's latency runs from submission to the
// moment the worker sees its batch's event complete.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "archive.h"

using namespace aceapex;

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
  int arc;
  uint64_t lo, hi;
  uint8_t *dst;
  std::vector<uint32_t> segs;  // transitive source closure of the covering segments
  double t_submit;
  double latency_ms = 0;
  int status = ACEAPEX_OK;
  bool done = false;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<DBuf<uint32_t>> page;  // per archive
  std::vector<DBuf<uint64_t>> flags;
  DBuf<uint8_t> arena;
  DBuf<WorkItem> work;
  DBuf<GatherJob> jobs;
  DBuf<uint32_t> words;  // err, epoch, counter
  DBuf<uint8_t> scratch;  // global staging, only when an archive needs it
  Staging stage_work, stage_jobs;
  std::vector<uint64_t> reqs;
  bool busy = false;
};

}  // namespace

struct aceapex_server {
  std::vector<aceapex_archive *> arcs;
  int device = 0;
  uint64_t cap_segs = 0;  // arena capacity of a slot, in segments
  std::vector<Slot> slots;
  std::vector<std::vector<uint32_t>> mark;  // per archive, for batch unions
  uint32_t mark_gen = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_pending;
  std::deque<uint64_t> pending;  // submitted, closure not yet walked
  std::deque<uint64_t> queue;    // closure known, waiting for admission
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  std::vector<std::thread> walkers;
  aceapex_server_stats st{};
  uint32_t inflight = 0;
};

namespace {

// Launch one batch on slot s (called by the worker without the lock; the
// requests were moved into the slot under the lock).
int launch_batch_on(aceapex_server *S, Slot &slot, const std::vector<Req *> &batch) {
  const uint32_t n_arc = (uint32_t)S->arcs.size();
  // union of closures per archive
  std::vector<std::vector<uint32_t>> uni(n_arc);
  if (++S->mark_gen == 0) {
    for (auto &m : S->mark) std::fill(m.begin(), m.end(), 0);
    S->mark_gen = 1;
  }
  const uint32_t g = S->mark_gen;
  for (Req *r : batch)
    for (uint32_t seg : r->segs)
      if (S->mark[r->arc][seg] != g) {
        S->mark[r->arc][seg] = g;
        uni[r->arc].push_back(seg);
      }
  std::vector<WorkItem> work;
  std::vector<uint64_t> off(n_arc + 1, 0);
  for (uint32_t a = 0; a < n_arc; ++a) {
    off[a] = work.size();
    level_order(S->arcs[a]->dir, uni[a].data(), uni[a].size(), a, work);
  }
  off[n_arc] = work.size();
  cudaStream_t st = slot.st;
  if (slot.work.n < work.size() && slot.work.alloc(std::max<uint64_t>(work.size(), 4096)) != cudaSuccess)
    return ACEAPEX_ENOMEM;
  if (slot.stage_work.reserve(work.size() * sizeof(WorkItem)) != cudaSuccess) return ACEAPEX_ENOMEM;
  std::memcpy(slot.stage_work.p, work.data(), work.size() * sizeof(WorkItem));
  cudaError_t e = cudaMemcpyAsync(slot.work.p, slot.stage_work.p, work.size() * sizeof(WorkItem),
                                  cudaMemcpyHostToDevice, st);
  slot.stage_work.mark(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(slot.words.p, 0, 4, st);
  if (e != cudaSuccess) return ACEAPEX_ECUDA;
  uint32_t *ge = global_epoch(S->device);
  if (!ge) return ACEAPEX_ECUDA;
  std::vector<OutView> views(n_arc);
  uint64_t arena_off = 0;  // archives may differ in segment size
  for (uint32_t a = 0; a < n_arc; ++a) {
    aceapex_archive *A = S->arcs[a];
    const uint32_t n = (uint32_t)(off[a + 1] - off[a]);
    OutView v{};
    v.page = slot.page[a].p;
    v.slot_base = slot.arena.p + arena_off;
    arena_off += (uint64_t)n << A->h.log2_S;
    views[a] = v;
    if (!n) continue;
    if ((e = launch_set_pages(slot.page[a].p, slot.work.p + off[a], n, st)) != cudaSuccess) return ACEAPEX_ECUDA;
    if ((e = launch_begin(ge, slot.words.p + 1, slot.words.p + 2, st)) != cudaSuccess) return ACEAPEX_ECUDA;
    DecodeLaunch L = base_launch(A);
    L.arc0.flags = slot.flags[a].p;
    L.arc0.blocked = nullptr;
    L.view0 = v;
    L.work = slot.work.p + off[a];
    L.n_work = n;
    L.err = slot.words.p;
    L.epoch = slot.words.p + 1;
    L.counter = slot.words.p + 2;
    L.scratch = slot.scratch.p;
    if ((e = launch_decode(L, A->grid, (int)kDecodeThreads, st)) != cudaSuccess) return ACEAPEX_ECUDA;
  }
  // gather every request into its caller buffer
  std::vector<GatherJob> jobs(batch.size());
  uint64_t chunks = 0;
  for (size_t i = 0; i < batch.size(); ++i) {
    Req *r = batch[i];
    GatherJob j{};
    j.v = views[r->arc];
    j.lo = r->lo;
    j.n = r->hi - r->lo;
    j.dst = r->dst;
    j.chunk0 = chunks;
    j.log2_S = S->arcs[r->arc]->h.log2_S;
    chunks += (j.n + 65535) / 65536;
    jobs[i] = j;
  }
  if (slot.jobs.n < jobs.size() && slot.jobs.alloc(std::max<uint64_t>(jobs.size(), 1024)) != cudaSuccess)
    return ACEAPEX_ENOMEM;
  if (slot.stage_jobs.reserve(jobs.size() * sizeof(GatherJob)) != cudaSuccess) return ACEAPEX_ENOMEM;
  std::memcpy(slot.stage_jobs.p, jobs.data(), jobs.size() * sizeof(GatherJob));
  e = cudaMemcpyAsync(slot.jobs.p, slot.stage_jobs.p, jobs.size() * sizeof(GatherJob), cudaMemcpyHostToDevice, st);
  slot.stage_jobs.mark(st);
  if (e == cudaSuccess) e = launch_multi_gather(slot.jobs.p, (uint32_t)jobs.size(), chunks, st);
  for (uint32_t a = 0; e == cudaSuccess && a < n_arc; ++a)
    e = launch_clear_pages(slot.page[a].p, slot.work.p + off[a], (uint32_t)(off[a + 1] - off[a]), st);
  if (e == cudaSuccess) e = cudaEventRecord(slot.ev, st);
  return e == cudaSuccess ? ACEAPEX_OK : ACEAPEX_ECUDA;
}

// Closure walker: takes submitted requests, walks their closures outside the
// lock with its own marks (one set per archive), and queues them for
// admission, or completes them with EBUSY when the closure can never fit a
// slot's arena.
void walker_loop(aceapex_server *S) {
  std::vector<std::vector<uint32_t>> mark(S->arcs.size());
  std::vector<uint32_t> gen(S->arcs.size(), 0);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_pending.wait(lk, [&] { return S->stop || !S->pending.empty(); });
    if (S->pending.empty()) break;  // stopping
    const uint64_t id = S->pending.front();
    S->pending.pop_front();
    Req *r = &S->reqs[id];
    lk.unlock();
    aceapex_archive *A = S->arcs[r->arc];
    closure_with(A, r->lo >> A->h.log2_S, (r->hi - 1) >> A->h.log2_S, mark[r->arc], gen[r->arc], r->segs);
    lk.lock();
    if (r->segs.size() > S->cap_segs) {
      r->status = ACEAPEX_EBUSY;
      r->latency_ms = now_ms() - r->t_submit;
      r->done = true;
      S->st.refused++;
      S->cv_done.notify_all();
    } else {
      S->queue.push_back(id);
      S->cv_work.notify_one();
    }
  }
}

void worker_loop(aceapex_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progressed = false;
    // completions
    for (Slot &slot : S->slots) {
      if (!slot.busy || cudaEventQuery(slot.ev) != cudaSuccess) continue;
      uint32_t err = 0;
      cudaMemcpy(&err, slot.words.p, 4, cudaMemcpyDeviceToHost);
      const double t = now_ms();
      for (uint64_t id : slot.reqs) {
        Req &r = S->reqs[id];
        r.done = true;
        if (r.status == ACEAPEX_OK && err) r.status = (int)err;
        r.latency_ms = t - r.t_submit;
        S->st.completed++;
        S->st.bytes_served += r.hi - r.lo;
      }
      slot.reqs.clear();
      slot.busy = false;
      S->inflight--;
      progressed = true;
      S->cv_done.notify_all();
    }
    // form and launch a batch on a free slot
    Slot *free_slot = nullptr;
    for (Slot &slot : S->slots)
      if (!slot.busy) {
        free_slot = &slot;
        break;
      }
    if (free_slot && !S->queue.empty()) {
      std::vector<Req *> batch;
      // admission: FIFO while the union of closures fits the slot arena
      std::vector<std::vector<uint32_t>> seen(S->arcs.size());
      uint64_t used = 0;
      if (++S->mark_gen == 0) {
        for (auto &m : S->mark) std::fill(m.begin(), m.end(), 0);
        S->mark_gen = 1;
      }
      const uint32_t g = S->mark_gen;
      while (!S->queue.empty()) {
        Req &r = S->reqs[S->queue.front()];
        uint64_t add = 0;
        for (uint32_t seg : r.segs) add += S->mark[r.arc][seg] != g;
        if (used + add > S->cap_segs && !batch.empty()) break;
        for (uint32_t seg : r.segs) S->mark[r.arc][seg] = g;
        used += add;
        batch.push_back(&r);
        free_slot->reqs.push_back(S->queue.front());
        S->queue.pop_front();
      }
      free_slot->busy = true;
      S->inflight++;
      S->st.batches++;
      S->st.max_batch = std::max<uint64_t>(S->st.max_batch, batch.size());
      S->st.max_inflight = std::max<uint64_t>(S->st.max_inflight, S->inflight);
      lk.unlock();
      int rc = launch_batch_on(S, *free_slot, batch);
      lk.lock();
      if (rc != ACEAPEX_OK) {
        for (Req *r : batch) r->status = rc;
        cudaEventRecord(free_slot->ev, free_slot->st);  // completes with the error status
      }
      progressed = true;
    }
    if (S->stop && S->queue.empty() && S->pending.empty() && S->inflight == 0) break;
    if (!progressed) {
      if (S->inflight) S->cv_work.wait_for(lk, std::chrono::microseconds(20));
      else S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

}  // namespace

extern "C" {

int aceapex_server_create(aceapex_archive *const *as, int n, uint64_t mem_budget, int slots, aceapex_server **out) {
  if (!as || n <= 0 || !out || slots <= 0 || slots > 64) return ACEAPEX_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!as[i] || as[i]->device != as[0]->device) return ACEAPEX_EINVAL;
  aceapex_server *S = new (std::nothrow) aceapex_server();
  if (!S) return ACEAPEX_ENOMEM;
  S->arcs.assign(as, as + n);
  S->device = as[0]->device;
  if (cudaSetDevice(S->device) != cudaSuccess) {
    delete S;
    return ACEAPEX_ECUDA;
  }
  // page tables and flags (12 bytes per segment per slot) come out of the budget
  uint64_t fixed = 0, need_stage = 0, seg_bytes = 0;
  for (aceapex_archive *A : S->arcs) {
    fixed += 12 * A->h.n_seg * (uint64_t)slots;
    seg_bytes = std::max<uint64_t>(seg_bytes, uint64_t(1) << A->h.log2_S);
    int rc = ensure_scratch(A, 0);
    if (rc) {
      delete S;
      return rc;
    }
    if (A->max_cmd_syms > A->stage_cap) need_stage = 1;
  }
  if (mem_budget <= fixed) {
    delete S;
    return ACEAPEX_EINVAL;
  }
  S->cap_segs = (mem_budget - fixed) / (uint64_t)slots / seg_bytes;
  if (S->cap_segs == 0) {
    delete S;
    return ACEAPEX_EINVAL;
  }
  S->mark.resize(n);
  for (int i = 0; i < n; ++i) S->mark[i].assign(S->arcs[i]->h.n_seg, 0);
  S->slots.resize(slots);
  for (Slot &slot : S->slots) {
    bool ok = cudaStreamCreateWithFlags(&slot.st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&slot.ev, cudaEventDisableTiming) == cudaSuccess &&
              slot.arena.alloc(S->cap_segs * seg_bytes) == cudaSuccess && slot.words.alloc(4) == cudaSuccess &&
              cudaMemset(slot.words.p, 0, 16) == cudaSuccess;
    if (ok && need_stage) ok = slot.scratch.alloc((uint64_t)S->arcs[0]->scratch_warps * kStageBytes) == cudaSuccess;
    slot.page.resize(n);
    slot.flags.resize(n);
    for (int i = 0; ok && i < n; ++i) {
      const uint64_t ns = std::max<uint64_t>(S->arcs[i]->h.n_seg, 1);
      // (the flag words start as the archive's: the levels, and epochs of
      // earlier calls, which no later call matches)
      ok = slot.page[i].alloc(ns) == cudaSuccess && slot.flags[i].alloc(ns) == cudaSuccess &&
           cudaMemset(slot.page[i].p, 0xFF, 4 * ns) == cudaSuccess &&
           cudaMemcpy(slot.flags[i].p, S->arcs[i]->d_flags.p, 8 * ns, cudaMemcpyDeviceToDevice) == cudaSuccess;
    }
    if (!ok) {
      aceapex_server_destroy(S);
      return ACEAPEX_ENOMEM;
    }
  }
  // the page-table fills and flag copies above ran on the legacy stream,
  // which the slots' non-blocking streams do not wait for
  if (cudaStreamSynchronize(0) != cudaSuccess) {
    aceapex_server_destroy(S);
    return ACEAPEX_ECUDA;
  }
  S->worker = std::thread(worker_loop, S);
  const unsigned hw = std::thread::hardware_concurrency();
  const unsigned nw = std::max(1u, std::min(8u, hw / 2));
  for (unsigned i = 0; i < nw; ++i) S->walkers.emplace_back(walker_loop, S);
  *out = S;
  return ACEAPEX_OK;
}

void aceapex_server_destroy(aceapex_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->cv_pending.notify_all();
  for (std::thread &t : S->walkers)
    if (t.joinable()) t.join();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  for (Slot &slot : S->slots) {
    if (slot.st) cudaStreamSynchronize(slot.st);
    for (auto &b : slot.page) b.release();
    for (auto &b : slot.flags) b.release();
    slot.arena.release();
    slot.work.release();
    slot.jobs.release();
    slot.words.release();
    slot.scratch.release();
    slot.stage_work.release();
    slot.stage_jobs.release();
    if (slot.ev) cudaEventDestroy(slot.ev);
    if (slot.st) cudaStreamDestroy(slot.st);
  }
  delete S;
}

int aceapex_server_submit(aceapex_server *S, int arc, uint64_t lo, uint64_t hi, void *d_dst, uint64_t cap,
                          uint64_t *ticket) {
  if (!S || !ticket || arc < 0 || arc >= (int)S->arcs.size() || (!d_dst && hi > lo)) return ACEAPEX_EINVAL;
  aceapex_archive *A = S->arcs[arc];
  if (lo >= hi || hi > A->h.n || cap < hi - lo) return ACEAPEX_ERANGE;
  Req r;
  r.arc = arc;
  r.lo = lo;
  r.hi = hi;
  r.dst = static_cast<uint8_t *>(d_dst);
  r.t_submit = now_ms();  // the latency includes the closure walk
  std::unique_lock<std::mutex> lk(S->mu);
  S->st.submitted++;
  // a closure holds at least the range's own segments: a range that alone
  // exceeds a slot's arena can never be admitted (wider closures are found
  // by the walker, which completes the request with EBUSY)
  if (((hi - 1) >> A->h.log2_S) - (lo >> A->h.log2_S) + 1 > S->cap_segs) {
    S->st.refused++;
    return ACEAPEX_EBUSY;
  }
  const uint64_t id = S->next_id++;
  S->reqs.emplace(id, std::move(r));
  S->pending.push_back(id);
  lk.unlock();
  S->cv_pending.notify_one();
  *ticket = id;
  return ACEAPEX_OK;
}

int aceapex_server_replay(aceapex_server *S, uint64_t n, const int *arc, const uint64_t *lo, const uint64_t *hi,
                          void *const *d_dst, const uint64_t *cap, const uint64_t *gap_ns, uint64_t *ticket,
                          int *status, double *submit_seconds) {
  if (!S || (n && (!arc || !lo || !hi || !d_dst || !cap || !gap_ns || !ticket || !status))) return ACEAPEX_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  auto due = t0;
  for (uint64_t i = 0; i < n; ++i) {
    due += std::chrono::nanoseconds(gap_ns[i]);
    while (std::chrono::steady_clock::now() < due) {
    }
    ticket[i] = 0;
    status[i] = aceapex_server_submit(S, arc[i], lo[i], hi[i], d_dst[i], cap[i], ticket + i);
    if (status[i] != ACEAPEX_OK) ticket[i] = 0;
  }
  if (submit_seconds)
    *submit_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return ACEAPEX_OK;
}

int aceapex_server_poll(aceapex_server *S, uint64_t ticket, int wait, int *done, double *latency_ms) {
  if (!S || !done) return ACEAPEX_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return ACEAPEX_EINVAL;
  if (wait)
    S->cv_done.wait(lk, [&] { return it->second.done; });
  *done = it->second.done ? 1 : 0;
  if (!it->second.done) return ACEAPEX_OK;
  if (latency_ms) *latency_ms = it->second.latency_ms;
  const int status = it->second.status;
  S->reqs.erase(it);
  return status;
}

int aceapex_server_get_stats(aceapex_server *S, aceapex_server_stats *out) {
  if (!S || !out) return ACEAPEX_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  out->queued = S->queue.size() + S->pending.size();
  out->slot_segments = S->cap_segs;
  return ACEAPEX_OK;
}

}  // extern "C"
