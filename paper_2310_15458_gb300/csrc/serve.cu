// Solve server: resident factorizations, continuous batching of solve requests.
//
// A worker thread owns the device side.  Each registered factorization has its
// own CUDA stream and a right-hand-side panel.  Whenever a factorization's
// stream is idle, the worker packs every pending request of that factorization
// (up to a per-batch limit on columns and the server's device-memory budget)
// into one n x sum(nrhs) panel: host-to-device copy, one rss_solve, one copy
// back, one event.  Requests that arrive while a panel is on the GPU wait for the
// next panel of their factorization; panels of different factorizations run
// concurrently on their own streams.  The sweeps treat every column with the
// same sequence of operations, so a request's result does not depend on what it
// was batched with.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket;
  int fid;
  const void* b;
  void* x;
  int64_t nrhs;
  Clock::time_point t_submit, t_done;
  int status = -1;   // -1 pending, else rss_status
};

struct Slot {
  const rss_factorization* f = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  std::deque<Request*> pending;
  std::vector<Request*> inflight;
  int64_t inflight_cols = 0;
  size_t inflight_bytes = 0;
  void* d_panel = nullptr;
  size_t d_cap = 0;
  void* h_panel = nullptr;   // pinned staging
  size_t h_cap = 0;
};

}  // namespace

struct rss_server {
  uint32_t tag = RSS_TAG_SERVER;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  size_t budget = 0, in_use = 0;
  size_t reserved = 0;   // factor caches built for the server's panels (held for its lifetime)
  int64_t max_cols = 256;
  int device = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  // counters
  long long n_req = 0, n_batch = 0, n_cols = 0, max_batch_seen = 0;
  std::string worker_error;
};

namespace {

size_t esz_of(const rss_factorization* f) { return f->is_complex ? 16 : 8; }

// Launch one panel for slot s (worker thread, lock held).  Returns whether it
// launched a panel or retired a request.
bool launch_panel(rss_server* S, Slot& s) {
  const size_t esz = esz_of(s.f);
  const int64_t n = s.f->n;
  std::vector<Request*> batch;
  int64_t cols = 0;
  bool acted = false;
  // device bytes of a panel of c columns: the panel itself plus what the solve
  // allocates for it (working copy and sweep workspace)
  auto need_of = [&](int64_t c) { return esz * (size_t)n * (size_t)c + solve_device_bytes(s.f, c); };
  size_t need = 0;
  while (!s.pending.empty()) {
    Request* r = s.pending.front();
    if (need_of(r->nrhs) > S->budget - S->reserved) {   // can never fit: refuse it
      s.pending.pop_front();
      r->status = RSS_ENOMEM;
      r->t_done = Clock::now();
      S->cv_done.notify_all();
      acted = true;
      continue;
    }
    if (cols + r->nrhs > S->max_cols && !batch.empty()) break;
    const size_t need_next = need_of(cols + r->nrhs);
    if (S->in_use + S->reserved + need_next > S->budget) break;   // wait for memory to free up
    need = need_next;
    batch.push_back(r);
    cols += r->nrhs;
    s.pending.pop_front();
  }
  if (batch.empty()) return acted;
  const size_t bytes = esz * (size_t)n * (size_t)cols;
  auto fail_batch = [&](const char* why) {
    for (Request* r : batch) {
      r->status = RSS_ECUDA;
      r->t_done = Clock::now();
    }
    S->worker_error = why;
    S->cv_done.notify_all();
  };
  if (s.d_cap < bytes) {
    pool_free(s.d_panel, s.stream);   // ordered after the panels already queued on this stream
    s.d_panel = nullptr;
    s.d_cap = 0;
    if (pool_malloc(&s.d_panel, bytes, s.stream) != cudaSuccess) {
      fail_batch("panel allocation failed");
      return true;
    }
    s.d_cap = bytes;
  }
  if (s.h_cap < bytes) {
    if (s.h_panel) cudaFreeHost(s.h_panel);
    s.h_panel = nullptr;
    s.h_cap = 0;
    if (cudaHostAlloc(&s.h_panel, bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      fail_batch("staging allocation failed");
      return true;
    }
    s.h_cap = bytes;
  }
  int64_t col = 0;
  for (Request* r : batch) {
    std::memcpy(static_cast<char*>(s.h_panel) + esz * n * col, r->b, esz * n * r->nrhs);
    col += r->nrhs;
  }
  cudaError_t e = cudaMemcpyAsync(s.d_panel, s.h_panel, bytes, cudaMemcpyHostToDevice, s.stream);
  rss_status st = RSS_OK;
  if (e == cudaSuccess)
    st = s.f->is_complex ? solve_impl<zd>(s.f, static_cast<zd*>(s.d_panel), cols, n, s.stream)
                         : solve_impl<double>(s.f, static_cast<double*>(s.d_panel), cols, n, s.stream);
  if (e == cudaSuccess && st == RSS_OK)
    e = cudaMemcpyAsync(s.h_panel, s.d_panel, bytes, cudaMemcpyDeviceToHost, s.stream);
  if (e == cudaSuccess && st == RSS_OK) e = cudaEventRecord(s.done, s.stream);
  if (e != cudaSuccess || st != RSS_OK) {
    cudaGetLastError();
    fail_batch("panel launch failed");
    return true;
  }
  s.inflight = std::move(batch);
  s.inflight_cols = cols;
  s.inflight_bytes = need;
  S->in_use += s.inflight_bytes;
  S->n_batch += 1;
  S->n_cols += cols;
  S->max_batch_seen = std::max<long long>(S->max_batch_seen, (long long)s.inflight.size());
  return true;
}

// Retire slot s's panel if its event completed (worker thread, lock held).
bool retire_panel(rss_server* S, Slot& s) {
  if (s.inflight.empty()) return false;
  const cudaError_t q = cudaEventQuery(s.done);
  if (q == cudaErrorNotReady) return false;
  const size_t esz = esz_of(s.f);
  const int64_t n = s.f->n;
  int64_t col = 0;
  const auto now = Clock::now();
  for (Request* r : s.inflight) {
    if (q == cudaSuccess) {
      std::memcpy(r->x, static_cast<char*>(s.h_panel) + esz * n * col, esz * n * r->nrhs);
      r->status = RSS_OK;
    } else {
      r->status = RSS_ECUDA;
    }
    r->t_done = now;
    col += r->nrhs;
  }
  if (q != cudaSuccess) cudaGetLastError();
  s.inflight.clear();
  S->in_use -= s.inflight_bytes;
  s.inflight_bytes = 0;
  S->cv_done.notify_all();
  return true;
}

void worker_main(rss_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    bool progress = false;
    for (auto& sp : S->slots) progress |= retire_panel(S, *sp);
    for (auto& sp : S->slots)
      if (sp->inflight.empty() && !sp->pending.empty()) progress |= launch_panel(S, *sp);
    bool busy = false;
    for (auto& sp : S->slots) busy |= !sp->inflight.empty();
    if (!progress) {
      if (busy) {   // poll the panels' events (requests waiting for memory wait for them too)
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        S->cv_work.wait(lk);
      }
    }
  }
}

rss_status fail(rss_status s, const std::string& msg) {
  rss_set_error(msg);
  return s;
}

}  // namespace

extern "C" {

rss_status rss_server_create(size_t device_bytes, int64_t max_batch_rhs, rss_server** out) {
  if (!out) return fail(RSS_EINVAL, "rss_server_create: out is NULL");
  *out = nullptr;
  if (device_bytes == 0 || max_batch_rhs <= 0) return fail(RSS_EINVAL, "rss_server_create: empty budget");
  rss_server* S = new (std::nothrow) rss_server();
  if (!S) return fail(RSS_ENOMEM, "rss_server_create: host allocation failed");
  S->budget = device_bytes;
  S->max_cols = max_batch_rhs;
  cudaGetDevice(&S->device);
  try {
    S->worker = std::thread(worker_main, S);
  } catch (...) {
    delete S;
    return fail(RSS_ENOMEM, "rss_server_create: could not start the worker thread");
  }
  *out = S;
  return RSS_OK;
}

rss_status rss_server_add(rss_server* S, const rss_factorization* f, int32_t* factor_id) {
  if (!S || S->tag != RSS_TAG_SERVER || !f || f->tag != RSS_TAG_FACTOR || !factor_id)
    return fail(RSS_EINVAL, "rss_server_add: bad arguments");
  auto s = std::make_unique<Slot>();
  s->f = f;
  // the factor caches the panels' solves would build on first use (outside any
  // budget) are built here and charged to the budget for the server's lifetime
  const size_t cache = solve_cache_bytes(f, S->max_cols);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->reserved + cache + solve_device_bytes(f, 1) + (f->is_complex ? 16 : 8) * (size_t)f->n > S->budget)
      return fail(RSS_ENOMEM, "rss_server_add: the factorization's solve caches (" + std::to_string(cache) +
                                  " bytes) and one column do not fit the server's device budget");
    S->reserved += cache;
  }
  auto unreserve = [&] {
    std::lock_guard<std::mutex> lk(S->mu);
    S->reserved -= cache;
  };
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (s->stream) cudaStreamDestroy(s->stream);
    unreserve();
    return fail(RSS_ECUDA, "rss_server_add: stream or event creation failed");
  }
  const rss_status cs = prepare_solve_caches(f, S->max_cols, s->stream);
  if (cs != RSS_OK) {
    cudaEventDestroy(s->done);
    cudaStreamDestroy(s->stream);
    unreserve();
    return cs;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  *factor_id = (int32_t)S->slots.size();
  S->slots.push_back(std::move(s));
  return RSS_OK;
}

rss_status rss_server_submit(rss_server* S, int32_t factor_id, const void* b, void* x, int64_t nrhs,
                             int64_t* ticket) {
  if (!S || S->tag != RSS_TAG_SERVER || !b || !x || nrhs <= 0 || !ticket)
    return fail(RSS_EINVAL, "rss_server_submit: bad arguments");
  std::lock_guard<std::mutex> lk(S->mu);
  if (factor_id < 0 || factor_id >= (int32_t)S->slots.size())
    return fail(RSS_EINVAL, "rss_server_submit: unknown factor id");
  auto r = std::make_unique<Request>();
  r->ticket = S->next_ticket++;
  r->fid = factor_id;
  r->b = b;
  r->x = x;
  r->nrhs = nrhs;
  r->t_submit = Clock::now();
  S->slots[factor_id]->pending.push_back(r.get());
  *ticket = r->ticket;
  S->reqs.emplace(r->ticket, std::move(r));
  S->n_req += 1;
  S->cv_work.notify_one();
  return RSS_OK;
}

rss_status rss_server_wait(rss_server* S, int64_t ticket, double timeout_s, double* latency_s) {
  if (!S || S->tag != RSS_TAG_SERVER) return fail(RSS_EINVAL, "rss_server_wait: bad server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(RSS_EINVAL, "rss_server_wait: unknown ticket");
  Request* r = it->second.get();
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
  while (r->status < 0)
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->status < 0)
      return fail(RSS_ETIMEOUT, "rss_server_wait: request still pending at the deadline");
  const rss_status st = (rss_status)r->status;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  S->reqs.erase(it);
  if (st != RSS_OK) return fail(st, "rss_server_wait: the request failed: " + S->worker_error);
  return RSS_OK;
}

rss_status rss_server_stats(rss_server* S, char* buf, size_t len) {
  if (!S || S->tag != RSS_TAG_SERVER || !buf || !len) return fail(RSS_EINVAL, "rss_server_stats: bad arguments");
  std::ostringstream o;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    o << "{\"requests\": " << S->n_req << ", \"batches\": " << S->n_batch << ", \"columns\": " << S->n_cols
      << ", \"max_requests_per_batch\": " << S->max_batch_seen << ", \"factors\": " << S->slots.size()
      << ", \"device_bytes_in_use\": " << S->in_use << ", \"device_bytes_reserved\": " << S->reserved
      << ", \"budget\": " << S->budget << "}";
  }
  const std::string s = o.str();
  if (s.size() + 1 > len) return fail(RSS_EINVAL, "rss_server_stats: buffer too small");
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return RSS_OK;
}

}  // extern "C"

void free_server(rss_server* S) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  for (auto& sp : S->slots) {
    if (sp->stream) cudaStreamSynchronize(sp->stream);
    pool_free(sp->d_panel, sp->stream);
    if (sp->stream) cudaStreamSynchronize(sp->stream);
    if (sp->h_panel) cudaFreeHost(sp->h_panel);
    if (sp->done) cudaEventDestroy(sp->done);
    if (sp->stream) cudaStreamDestroy(sp->stream);
  }
  S->tag = 0;
  delete S;
}
