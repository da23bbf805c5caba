// Query server: continuous batching of segmentation queries over a resident dataset.
//
// Clients submit queries from any thread; one worker thread admits them into launch slots and
// launches each slot's queries as one batch (the batched labelling kernels of k_segment.cu) on
// the slot's own stream. Slots run concurrently on the device, so a batch launched while
// another is still running overlaps with it; queries that arrive meanwhile wait in a FIFO and
// go into the next free slot. A query is admitted only when its labels and its labelling
// scratch fit into the server's device pool, which is allocated once when the server starts:
// nothing is allocated while queries are served. Labels stay in the pool until the client
// releases the query; scratch returns to the pool when the query's batch completes.
//
// Completion is observed through a host function enqueued behind each batch on its stream; it
// stamps the completion time and wakes the worker, which reads the feature counts and hands
// the results to the clients. Results are the canonical labels of each query, so a query gives
// the same labels alone and in any mix.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "msf_internal.cuh"

namespace msf {

static int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over offsets of one device block, 256-byte granules, with coalescing.
class PoolAlloc {
 public:
  void reset(size_t cap) {
    cap_ = cap;
    used_ = peak_ = 0;
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t n, size_t* off) {
    n = round(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n, at = it->first + n;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += n;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = round(n);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  static size_t round(size_t n) { return std::max<size_t>(256, (n + 255) & ~size_t(255)); }
  size_t cap() const { return cap_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes
};

struct Request {
  uint64_t tag = 0;
  msf_criteria crit{};
  int64_t n_labels = 0;
  size_t lab_bytes = 0, scr_bytes = 0;
  size_t lab_off = 0, scr_off = 0;
  int64_t t_submit = 0, t_admit = 0;
};

struct Slot {
  msf_server* srv = nullptr;
  cudaStream_t stream = nullptr;
  StreamPair side;            // second stream of the slot (trajectory joins)
  char* plan_dev = nullptr;   // device plan area (tables and counts)
  char* plan_host = nullptr;  // its pinned host image
  size_t plan_cap = 0;
  bool busy = false;
  bool done = false;          // set by the stream's host function
  int64_t t_done = 0;
  std::vector<Request> reqs;
  BatchJob* job = nullptr;
};

}  // namespace msf

using namespace msf;

struct msf_server {
  msf_ctx* ctx = nullptr;
  int max_batch = 64;
  bool fault_admit = false;   // host-side fault injection: every admission fails
  char* pool = nullptr;
  PoolAlloc alloc;
  std::vector<Slot> slots;
  std::mutex m;
  std::condition_variable cv_work;  // worker: new request, slot done, memory freed, stop
  std::condition_variable cv_done;  // clients: results ready
  std::deque<Request> pending;
  std::deque<msf_server_result> done;
  std::unordered_map<uint64_t, std::pair<size_t, size_t>> held;  // tag -> labels (off, bytes)
  std::unordered_map<uint64_t, int> live;                       // submitted, not yet released
  uint64_t mem_epoch = 0;      // bumped whenever pool memory is freed
  uint64_t blocked_epoch = ~0ull;  // epoch at which the head of the queue did not fit
  bool stop = false;
  std::thread worker;
  msf_server_stats st{};
};

namespace msf {

static void CUDART_CB on_batch_done(void* p) {
  Slot* s = static_cast<Slot*>(p);
  msf_server* srv = s->srv;
  {
    std::lock_guard<std::mutex> lk(srv->m);
    s->done = true;
    s->t_done = now_ns();
  }
  srv->cv_work.notify_one();
}

// Hand a finished (or failed) request to the clients. Under the lock.
static void publish(msf_server* srv, const Request& r, int status, int64_t nf, int batch,
                    int64_t t_done) {
  msf_server_result res{};
  res.tag = r.tag;
  res.status = status;
  res.batch_size = batch;
  res.n_features = status == MSF_OK ? nf : 0;
  res.n_labels = status == MSF_OK ? r.n_labels : 0;
  res.labels = nullptr;
  if (status == MSF_OK && r.lab_bytes) {
    res.labels = reinterpret_cast<int32_t*>(srv->pool + r.lab_off);
    srv->held[r.tag] = {r.lab_off, r.lab_bytes};
  } else if (r.lab_bytes) {
    srv->alloc.release(r.lab_off, r.lab_bytes);
    ++srv->mem_epoch;
  }
  res.t_submit_ns = r.t_submit;
  res.t_admit_ns = r.t_admit;
  res.t_done_ns = t_done;
  srv->done.push_back(res);
  ++srv->st.completed;
}

// Collect the results of finished slots. Under the lock.
static bool harvest(msf_server* srv) {
  bool any = false;
  for (Slot& s : srv->slots) {
    if (!s.busy || !s.done) continue;
    const int n = (int)s.reqs.size();
    std::vector<int64_t> nf(n, 0);
    std::vector<int> status(n, MSF_OK);
    batch_job_finish(s.job, s.plan_host, nf.data(), status.data());
    for (int i = 0; i < n; ++i) {
      const Request& r = s.reqs[i];
      srv->alloc.release(r.scr_off, r.scr_bytes);
      publish(srv, r, status[i], nf[i], n, s.t_done);
    }
    ++srv->mem_epoch;
    batch_job_free(s.job);
    s.job = nullptr;
    s.reqs.clear();
    s.busy = false;
    s.done = false;
    any = true;
  }
  return any;
}

// Move queued requests into a free slot while they fit the pool. Under the lock; returns the
// slot or nullptr.
static Slot* admit(msf_server* srv) {
  if (srv->pending.empty() || srv->blocked_epoch == srv->mem_epoch) return nullptr;
  Slot* slot = nullptr;
  for (Slot& s : srv->slots)
    if (!s.busy) {
      slot = &s;
      break;
    }
  if (!slot) return nullptr;
  const int64_t t = now_ns();
  while (!srv->pending.empty() && (int)slot->reqs.size() < srv->max_batch) {
    Request& r = srv->pending.front();
    if (srv->fault_admit) {  // injected admission failure: the request fails, nothing leaks
      r.lab_bytes = 0;
      r.t_admit = t;
      publish(srv, r, MSF_ERR_OUT_OF_MEMORY, 0, 0, t);
      srv->pending.pop_front();
      continue;
    }
    if (!srv->alloc.alloc(r.lab_bytes, &r.lab_off)) break;
    if (!srv->alloc.alloc(r.scr_bytes, &r.scr_off)) {
      srv->alloc.release(r.lab_off, r.lab_bytes);
      break;
    }
    r.t_admit = t;
    slot->reqs.push_back(r);
    srv->pending.pop_front();
  }
  if (slot->reqs.empty()) {
    if (!srv->pending.empty()) srv->blocked_epoch = srv->mem_epoch;  // wait for memory
    if (!srv->done.empty()) srv->cv_done.notify_all();
    return nullptr;
  }
  srv->blocked_epoch = ~0ull;
  slot->busy = true;
  slot->done = false;
  return slot;
}

// Plan and enqueue one slot's batch. Outside the lock (CUDA calls only on the slot's stream).
static int launch_slot(msf_server* srv, Slot* s) {
  const int n = (int)s->reqs.size();
  std::vector<msf_criteria> crits(n);
  std::vector<int32_t*> labels(n);
  std::vector<char*> scratch(n);
  for (int i = 0; i < n; ++i) {
    crits[i] = s->reqs[i].crit;
    labels[i] = reinterpret_cast<int32_t*>(srv->pool + s->reqs[i].lab_off);
    scratch[i] = srv->pool + s->reqs[i].scr_off;
  }
  BatchJob* job = nullptr;
  MSF_TRY(batch_job_plan(srv->ctx, n, crits.data(), &job));
  s->job = job;
  if (batch_job_plan_bytes(job) > s->plan_cap) return MSF_ERR_INTERNAL;
  for (int i = 0; i < n; ++i)
    if (batch_job_scratch_bytes(job, i) > s->reqs[i].scr_bytes) return MSF_ERR_INTERNAL;
  MSF_TRY(batch_job_launch(srv->ctx, job, labels.data(), scratch.data(), s->plan_dev,
                           s->plan_host, s->stream, s->side, false));
  MSF_CUDA_TRY(cudaLaunchHostFunc(s->stream, on_batch_done, s));
  return MSF_OK;
}

static void worker_main(msf_server* srv) {
  cudaSetDevice(srv->ctx->device);
  std::unique_lock<std::mutex> lk(srv->m);
  for (;;) {
    if (harvest(srv)) srv->cv_done.notify_all();
    int busy = 0;
    for (Slot& s : srv->slots) busy += s.busy;
    if (srv->stop && busy == 0) break;
    Slot* slot = srv->stop ? nullptr : admit(srv);
    if (slot) {
      int in_flight = 0;
      for (Slot& s : srv->slots) in_flight += s.busy;
      srv->st.max_slots_busy = std::max<int64_t>(srv->st.max_slots_busy, in_flight);
      srv->st.max_batch_seen = std::max<int64_t>(srv->st.max_batch_seen, (int64_t)slot->reqs.size());
      ++srv->st.batches;
      lk.unlock();
      const int status = launch_slot(srv, slot);
      lk.lock();
      if (status != MSF_OK) {
        // nothing of this batch runs (a failed launch leaves no host function behind it);
        // wait for the stream so no copy still targets the slot's buffers
        lk.unlock();
        cudaStreamSynchronize(slot->stream);
        cudaGetLastError();
        lk.lock();
        const int64_t t = now_ns();
        for (const Request& r : slot->reqs) {
          srv->alloc.release(r.scr_off, r.scr_bytes);
          publish(srv, r, status, 0, (int)slot->reqs.size(), t);
        }
        ++srv->mem_epoch;
        if (slot->job) batch_job_free(slot->job);
        slot->job = nullptr;
        slot->reqs.clear();
        slot->busy = false;
        srv->cv_done.notify_all();
      }
      continue;  // try to fill another free slot at once
    }
    srv->cv_work.wait(lk, [&] {
      if (srv->stop) return true;
      for (Slot& s : srv->slots)
        if (s.busy && s.done) return true;
      if (srv->pending.empty() || srv->blocked_epoch == srv->mem_epoch) return false;
      for (Slot& s : srv->slots)
        if (!s.busy) return true;
      return false;
    });
  }
}

static void server_free(msf_server* srv) {
  for (Slot& s : srv->slots) {
    if (s.stream) {
      cudaStreamSynchronize(s.stream);
      cudaStreamDestroy(s.stream);
    }
    if (s.plan_dev) cudaFree(s.plan_dev);
    if (s.plan_host) cudaFreeHost(s.plan_host);
    if (s.side.aux) {
      cudaStreamSynchronize(s.side.aux);
      cudaStreamDestroy(s.side.aux);
    }
    if (s.side.ev_fork) cudaEventDestroy(s.side.ev_fork);
    if (s.side.ev_join) cudaEventDestroy(s.side.ev_join);
    if (s.job) batch_job_free(s.job);
  }
  if (srv->pool) cudaFree(srv->pool);
  delete srv;
}

}  // namespace msf

extern "C" int msf_server_create(msf_ctx* ctx, const msf_server_config* cfg, msf_server** out) {
  if (!ctx || !out) return MSF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctx->ds.loaded) return MSF_ERR_NOT_LOADED;
  msf_server_config c{};
  if (cfg) c = *cfg;
  if (c.pool_bytes == 0) c.pool_bytes = (uint64_t)4 << 30;
  if (c.max_batch == 0) c.max_batch = 64;
  if (c.slots == 0) c.slots = 2;
  if (c.max_batch < 1 || c.max_batch > 4096 || c.slots < 1 || c.slots > 16 ||
      c.pool_bytes < 4096)
    return MSF_ERR_INVALID_ARG;
  MSF_CUDA_TRY(cudaSetDevice(ctx->device));
  // the slots' streams read the dataset: everything queued on the context (the field's copy
  // in, binning) completes first
  MSF_TRY(ctx_field_ready(ctx));
  MSF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  msf_server* srv = new msf_server();
  srv->ctx = ctx;
  srv->max_batch = c.max_batch;
  const char* fault = getenv("MSF_FAULT");
  srv->fault_admit = fault && strcmp(fault, "admit") == 0;
  srv->alloc.reset(PoolAlloc::round(c.pool_bytes) == c.pool_bytes ? c.pool_bytes
                                                                   : c.pool_bytes & ~(uint64_t)255);
  srv->slots.resize(c.slots);
  const size_t plan_cap = batch_plan_bound(c.max_batch, ctx->ds.T, ctx->ds.Tp, ctx->ds.nz);
  int st = MSF_OK;
  if (cudaMalloc(&srv->pool, srv->alloc.cap()) != cudaSuccess) st = MSF_ERR_OUT_OF_MEMORY;
  for (Slot& s : srv->slots) {
    if (st != MSF_OK) break;
    s.srv = srv;
    s.plan_cap = plan_cap;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s.side.aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.side.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.side.ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&s.plan_dev, plan_cap) != cudaSuccess ||
        cudaMallocHost(&s.plan_host, plan_cap) != cudaSuccess)
      st = MSF_ERR_OUT_OF_MEMORY;
  }
  if (st != MSF_OK) {
    cudaGetLastError();
    server_free(srv);
    return st;
  }
  srv->st.pool_bytes = srv->alloc.cap();
  ++ctx->servers;
  srv->worker = std::thread(worker_main, srv);
  *out = srv;
  return MSF_OK;
}

extern "C" int msf_server_submit(msf_server* srv, const msf_criteria* crit, uint64_t tag) {
  if (!srv || !crit) return MSF_ERR_INVALID_ARG;
  MSF_TRY(validate_criteria(srv->ctx, crit));
  Request r;
  r.tag = tag;
  r.crit = *crit;
  const Dataset& d = srv->ctx->ds;
  r.n_labels = (int64_t)(crit->t1 - crit->t0) * d.nx * d.ny * d.nz;
  if (r.n_labels > 0) {
    size_t scr = 0;
    MSF_TRY(batch_query_scratch(srv->ctx, crit, &scr));
    r.lab_bytes = PoolAlloc::round(sizeof(int32_t) * (size_t)r.n_labels);
    r.scr_bytes = PoolAlloc::round(scr);
    if (r.lab_bytes + r.scr_bytes > srv->alloc.cap()) return MSF_ERR_TOO_LARGE;
  }
  r.t_submit = now_ns();
  {
    std::lock_guard<std::mutex> lk(srv->m);
    if (srv->stop) return MSF_ERR_INVALID_ARG;
    if (srv->live.count(tag)) return MSF_ERR_INVALID_ARG;
    srv->live[tag] = 1;
    ++srv->st.submitted;
    if (r.n_labels == 0) {  // empty window: done at once, nothing to label
      publish(srv, r, MSF_OK, 0, 0, r.t_submit);
      srv->cv_done.notify_all();
      return MSF_OK;
    }
    srv->pending.push_back(r);
  }
  srv->cv_work.notify_one();
  return MSF_OK;
}

extern "C" int msf_server_poll(msf_server* srv, msf_server_result* out, int cap, int* n_out,
                               int timeout_ms) {
  if (!srv || !n_out || cap < 0 || (cap > 0 && !out)) return MSF_ERR_INVALID_ARG;
  *n_out = 0;
  std::unique_lock<std::mutex> lk(srv->m);
  if (srv->done.empty() && timeout_ms != 0 && cap > 0) {
    auto ready = [&] { return !srv->done.empty(); };
    if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
    else srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  int n = 0;
  while (n < cap && !srv->done.empty()) {
    out[n] = srv->done.front();
    srv->done.pop_front();
    if (!out[n].labels) srv->live.erase(out[n].tag);  // nothing to release
    ++n;
  }
  *n_out = n;
  return MSF_OK;
}

extern "C" int msf_server_release(msf_server* srv, uint64_t tag) {
  if (!srv) return MSF_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(srv->m);
    auto it = srv->held.find(tag);
    if (it == srv->held.end()) return MSF_ERR_INVALID_ARG;
    srv->alloc.release(it->second.first, it->second.second);
    srv->held.erase(it);
    srv->live.erase(tag);
    ++srv->mem_epoch;
  }
  srv->cv_work.notify_one();
  return MSF_OK;
}

extern "C" int msf_server_get_stats(msf_server* srv, msf_server_stats* out) {
  if (!srv || !out) return MSF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->m);
  *out = srv->st;
  out->pending = (int64_t)srv->pending.size();
  int64_t inf = 0;
  for (Slot& s : srv->slots) inf += s.busy ? (int64_t)s.reqs.size() : 0;
  out->in_flight = inf;
  out->pool_used = srv->alloc.used();
  out->pool_peak = srv->alloc.peak();
  return MSF_OK;
}

extern "C" int msf_server_destroy(msf_server* srv) {
  if (!srv) return MSF_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(srv->m);
    srv->stop = true;
  }
  srv->cv_work.notify_one();
  if (srv->worker.joinable()) srv->worker.join();
  cudaSetDevice(srv->ctx->device);
  --srv->ctx->servers;
  server_free(srv);
  return MSF_OK;
}
