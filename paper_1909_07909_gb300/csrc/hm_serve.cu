// Serving runtime: resident HODLR/HSS matrices, admission of product requests
// by free slots and a memory budget, and continuous batching.
//
// A worker thread takes whatever requests are queued, merges the requests of
// one matrix into a single product with the requests' columns side by side
// (up to r_cap columns), launches it on that matrix's stream and records an
// event; requests arriving meanwhile are admitted and merged into the next
// launches without waiting for earlier ones, and products of different
// matrices overlap on the device (one stream per matrix slot, round robin).
// Each registered matrix's kernel family is fixed at registration (tensor
// cores for BF16/BF16X2 storage, SIMT otherwise) and every kernel treats
// columns independently, so a request's result does not depend on what it was
// merged with.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hm_api_internal.h"

namespace hmi {

static hm_status sfail(hm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_error("%s", buf);
  return s;
}

static int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct SrvMatrix {
  hm_matrix* A = nullptr;
  int stream = 0;
  float* xbuf = nullptr;   // merged right-hand sides, n x r_cap
  float* ybuf = nullptr;   // merged results, n x r_cap
  size_t bytes = 0;        // budget charged at registration
};

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct SrvReq {
  int id = 0;
  int64_t r = 0;
  const void* X = nullptr;
  void* Y = nullptr;
  int64_t t_submit = 0;
  int64_t t_done = 0;
  int state = RQ_QUEUED;
  hm_status status = HM_OK;
  size_t transient = 0;   // budget held while admitted
};

struct SrvBatch {
  cudaEvent_t ev = nullptr;
  std::vector<uint64_t> tickets;
  double bytes = 0;
};

}  // namespace hmi

struct hm_server {
  uint32_t magic = 0;
  int device = 0;
  size_t budget = 0;
  size_t resident = 0;      // registered matrices and their buffers
  size_t transient = 0;     // admitted requests' share
  int32_t max_slots = 0;
  int64_t r_cap = 64;      // most columns merged into one product
  int pending = 0;          // admitted and not yet completed
  std::vector<hmi::SrvMatrix> mats;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> event_pool;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, hmi::SrvReq> reqs;
  std::deque<hmi::SrvBatch> inflight;
  std::vector<double> lat_us;
  int64_t submitted = 0, admitted = 0, rejected = 0, completed = 0, launches = 0;
  double bytes_done = 0;
  int64_t t_first = 0, t_last = 0;
  int max_merge = 0;
  uint64_t next_ticket = 1;
  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<bool> paused{false};   // hm_serve_pause: the worker takes no queued request
};

namespace hmi {

static cudaEvent_t get_event(hm_server* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

// Completes every in-flight batch whose event has fired (in launch order per
// stream is not required: each batch is checked on its own).
static void reap(hm_server* s) {
  std::vector<SrvBatch> done;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->inflight.begin(); it != s->inflight.end();) {
      if (cudaEventQuery(it->ev) == cudaSuccess) {
        done.push_back(*it);
        it = s->inflight.erase(it);
      } else {
        cudaGetLastError();
        ++it;
      }
    }
    if (done.empty()) return;
    const int64_t t = now_ns();
    for (auto& b : done) {
      for (uint64_t tk : b.tickets) {
        auto f = s->reqs.find(tk);
        if (f == s->reqs.end()) continue;
        f->second.state = RQ_DONE;
        f->second.t_done = t;
        s->transient -= f->second.transient;
        s->pending -= 1;
        s->completed += 1;
        if (s->lat_us.size() < (size_t(1) << 22)) s->lat_us.push_back((t - f->second.t_submit) * 1e-3);
      }
      s->bytes_done += b.bytes;
      s->t_last = t;
      s->event_pool.push_back(b.ev);
    }
  }
  s->cv_done.notify_all();
}

// Launches one merged product for requests `tk` of matrix `id`.
static void launch_group(hm_server* s, int id, const std::vector<uint64_t>& tk) {
  SrvMatrix& M = s->mats[id];
  hm_matrix* A = M.A;
  const int64_t n = A->n;
  cudaStream_t st = s->streams[M.stream];
  std::vector<SrvReq> rq;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (uint64_t t : tk) {
      s->reqs[t].state = RQ_RUNNING;
      rq.push_back(s->reqs[t]);
    }
  }
  int64_t rtot = 0;
  for (auto& q : rq) rtot += q.r;
  hm_status st_prod = HM_OK;
  if (rq.size() == 1) {
    st_prod = run_product(A, A->kind, rq[0].r, rq[0].X, n, HM_F32, rq[0].Y, n, HM_F32, st);
  } else {
    int64_t off = 0;
    for (auto& q : rq) {
      if (cudaMemcpyAsync(M.xbuf + off * n, q.X, sizeof(float) * n * q.r, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        st_prod = HM_ECUDA;
      off += q.r;
    }
    if (st_prod == HM_OK) st_prod = run_product(A, A->kind, rtot, M.xbuf, n, HM_F32, M.ybuf, n, HM_F32, st);
    off = 0;
    for (auto& q : rq) {
      if (st_prod == HM_OK &&
          cudaMemcpyAsync(q.Y, M.ybuf + off * n, sizeof(float) * n * q.r, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        st_prod = HM_ECUDA;
      off += q.r;
    }
  }
  SrvBatch b;
  b.tickets = tk;
  b.bytes = static_cast<double>(A->gen_bytes) + 8.0 * static_cast<double>(n) * rtot;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    b.ev = get_event(s);
    s->launches += 1;
    s->max_merge = std::max(s->max_merge, static_cast<int>(tk.size()));
    if (st_prod != HM_OK) {
      for (uint64_t t : tk) s->reqs[t].status = st_prod;
    }
  }
  cudaEventRecord(b.ev, st);
  std::lock_guard<std::mutex> lk(s->mu);
  s->inflight.push_back(b);
}

static void worker_main(hm_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    reap(s);
    // take the queue: group by matrix, up to r_cap columns per product
    std::vector<std::pair<int, std::vector<uint64_t>>> groups;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->queue.empty() || s->paused.load()) {
        if (s->inflight.empty())
          s->cv_work.wait_for(lk, std::chrono::microseconds(200));
        else
          s->cv_work.wait_for(lk, std::chrono::microseconds(10));
        if (s->queue.empty() || s->paused.load()) continue;
      }
      std::unordered_map<int, size_t> at;
      std::unordered_map<int, int64_t> cols;
      while (!s->queue.empty()) {
        const uint64_t t = s->queue.front();
        s->queue.pop_front();
        SrvReq& q = s->reqs[t];
        q.state = RQ_RUNNING;   // taken: no longer cancellable
        auto f = at.find(q.id);
        if (f == at.end() || cols[q.id] + q.r > s->r_cap) {
          at[q.id] = groups.size();
          cols[q.id] = 0;
          groups.push_back({q.id, {}});
        }
        groups[at[q.id]].second.push_back(t);
        cols[q.id] += q.r;
      }
    }
    for (auto& g : groups) launch_group(s, g.first, g.second);
  }
}

void destroy_server(void* any) {
  hm_server* s = static_cast<hm_server*>(any);
  s->stop.store(true);
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != s->device) cudaSetDevice(s->device);
  for (auto st : s->streams) cudaStreamSynchronize(st);
  reap(s);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->reqs)
      if (kv.second.state != RQ_DONE) {
        kv.second.state = RQ_DONE;
        kv.second.status = HM_ECUDA;
      }
  }
  s->cv_done.notify_all();
  for (auto& m : s->mats) {
    if (m.xbuf) cudaFree(m.xbuf);
    if (m.ybuf) cudaFree(m.ybuf);
  }
  for (auto e : s->event_pool) cudaEventDestroy(e);
  for (auto st : s->streams) cudaStreamDestroy(st);
  if (dev_prev != s->device) cudaSetDevice(dev_prev);
  s->magic = 0;
  delete s;
}

}  // namespace hmi

using namespace hmi;

extern "C" hm_status hm_serve_create(size_t mem_budget, int32_t max_slots, hm_server** out) {
  if (!out) return sfail(HM_EINVAL, "out is NULL");
  *out = nullptr;
  if (mem_budget == 0 || max_slots < 1) return sfail(HM_EINVAL, "need a positive budget and at least one slot");
  hm_server* s = new (std::nothrow) hm_server();
  if (!s) return sfail(HM_ENOMEM, "host allocation failed");
  s->magic = kMagicServer;
  cudaGetDevice(&s->device);
  s->budget = mem_budget;
  s->max_slots = max_slots;
  for (int i = 0; i < 4; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      destroy_server(s);
      return sfail(HM_ECUDA, "stream creation failed");
    }
    s->streams.push_back(st);
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return HM_OK;
}

extern "C" hm_status hm_serve_register(hm_server* s, hm_matrix* A, int32_t* id) {
  if (!s || s->magic != kMagicServer) return sfail(HM_EINVAL, "not a server handle");
  if (!A || A->magic != kMagicMatrix || !id) return sfail(HM_EINVAL, "need a matrix handle and an id pointer");
  if (A->device != s->device) return sfail(HM_EINVAL, "matrix lives on another device");
  if (A->storage == HM_F64) return sfail(HM_EUNSUPPORTED, "the server takes F32 right-hand sides: F64 storage is not served");
  const int64_t n = std::max<int64_t>(A->n, 1);
  const MatView mv = A->view();
  const size_t scratch = scratch_elems(mv, s->r_cap) * 4 + counter_count(mv, s->r_cap) * sizeof(int);
  const size_t bufs = 2 * sizeof(float) * static_cast<size_t>(n) * s->r_cap;
  const size_t need = A->dev_bytes + scratch + bufs;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->resident + need > s->budget)
    return sfail(HM_ENOMEM, "registering needs %zu bytes; %zu of the %zu-byte budget are in use", need, s->resident,
                 s->budget);
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != s->device) cudaSetDevice(s->device);
  SrvMatrix M;
  M.A = A;
  M.stream = static_cast<int>(s->mats.size() % s->streams.size());
  hm_status st = ensure_scratch(A, s->r_cap);
  if (st == HM_OK && (dev_malloc(reinterpret_cast<void**>(&M.xbuf), bufs / 2) != cudaSuccess || dev_malloc(reinterpret_cast<void**>(&M.ybuf), bufs / 2) != cudaSuccess))
    st = sfail(HM_ENOMEM, "merge buffers");
  if (dev_prev != s->device) cudaSetDevice(dev_prev);
  if (st != HM_OK) {
    if (M.xbuf) cudaFree(M.xbuf);
    if (M.ybuf) cudaFree(M.ybuf);
    return st;
  }
  // results must not depend on how requests are merged: fix the kernel family
  A->path = (A->storage == HM_BF16 || A->storage == HM_BF16X2) ? 2 : 1;
  M.bytes = need;
  s->resident += need;
  *id = static_cast<int32_t>(s->mats.size());
  s->mats.push_back(M);
  return HM_OK;
}

extern "C" hm_status hm_serve_submit(hm_server* s, int32_t id, int64_t r, const void* X, void* Y, uint64_t* ticket) {
  if (!s || s->magic != kMagicServer) return sfail(HM_EINVAL, "not a server handle");
  if (!ticket || !X || !Y) return sfail(HM_EINVAL, "X, Y and ticket are required");
  std::unique_lock<std::mutex> lk(s->mu);
  if (id < 0 || id >= static_cast<int32_t>(s->mats.size())) return sfail(HM_EINVAL, "unknown matrix id %d", id);
  if (r < 1 || r > s->r_cap) return sfail(HM_EINVAL, "r must be in [1, %lld]", static_cast<long long>(s->r_cap));
  s->submitted += 1;
  const hm_matrix* A = s->mats[id].A;
  const size_t tbytes = 2 * sizeof(float) * static_cast<size_t>(std::max<int64_t>(A->n, 1)) * r;
  if (s->pending >= s->max_slots || s->resident + s->transient + tbytes > s->budget) {
    s->rejected += 1;
    return sfail(HM_EBUSY, "no free slot or budget (%d pending of %d slots)", s->pending, s->max_slots);
  }
  const uint64_t t = s->next_ticket++;
  SrvReq q;
  q.id = id;
  q.r = r;
  q.X = X;
  q.Y = Y;
  q.t_submit = now_ns();
  q.transient = tbytes;
  if (s->t_first == 0) s->t_first = q.t_submit;
  s->reqs[t] = q;
  s->queue.push_back(t);
  s->pending += 1;
  s->transient += tbytes;
  s->admitted += 1;
  *ticket = t;
  lk.unlock();
  s->cv_work.notify_one();
  return HM_OK;
}

extern "C" hm_status hm_serve_wait(hm_server* s, uint64_t ticket, int32_t timeout_ms) {
  if (!s || s->magic != kMagicServer) return sfail(HM_EINVAL, "not a server handle");
  std::unique_lock<std::mutex> lk(s->mu);
  auto f = s->reqs.find(ticket);
  if (f == s->reqs.end()) return sfail(HM_EINVAL, "unknown ticket %llu", static_cast<unsigned long long>(ticket));
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(timeout_ms, 0));
  while (s->reqs[ticket].state != RQ_DONE) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->reqs[ticket].state != RQ_DONE)
      return sfail(HM_ETIMEOUT, "request %llu not finished after %d ms", static_cast<unsigned long long>(ticket),
                   timeout_ms);
  }
  const hm_status st = s->reqs[ticket].status;
  s->reqs.erase(ticket);
  return st;
}

extern "C" hm_status hm_serve_poll(hm_server* s, uint64_t ticket) {
  if (!s || s->magic != kMagicServer) return sfail(HM_EINVAL, "not a server handle");
  std::lock_guard<std::mutex> lk(s->mu);
  auto f = s->reqs.find(ticket);
  if (f == s->reqs.end()) return sfail(HM_EINVAL, "unknown ticket");
  if (f->second.state != RQ_DONE) return HM_EBUSY;
  const hm_status st = f->second.status;
  s->reqs.erase(f);
  return st;
}

extern "C" hm_status hm_serve_cancel(hm_server* s, uint64_t ticket) {
  if (!s || s->magic != kMagicServer) return sfail(HM_EINVAL, "not a server handle");
  std::lock_guard<std::mutex> lk(s->mu);
  auto f = s->reqs.find(ticket);
  if (f == s->reqs.end()) return sfail(HM_EINVAL, "unknown ticket %llu", static_cast<unsigned long long>(ticket));
  if (f->second.state != RQ_QUEUED)
    return sfail(HM_EBUSY, "request %llu is already running or finished", static_cast<unsigned long long>(ticket));
  auto q = std::find(s->queue.begin(), s->queue.end(), ticket);
  if (q != s->queue.end()) s->queue.erase(q);
  s->pending -= 1;
  s->transient -= f->second.transient;
  s->reqs.erase(f);
  return HM_OK;
}

extern "C" hm_status hm_serve_pause(hm_server* s, int32_t pause) {
  if (!s || s->magic != kMagicServer) return sfail(HM_EINVAL, "not a server handle");
  s->paused.store(pause != 0);
  s->cv_work.notify_all();
  return HM_OK;
}

extern "C" hm_status hm_serve_stats(hm_server* s, hm_serve_stats_t* out) {
  if (!s || s->magic != kMagicServer) return sfail(HM_EINVAL, "not a server handle");
  if (!out) return sfail(HM_EINVAL, "out is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->rejected = s->rejected;
  out->completed = s->completed;
  out->launches = s->launches;
  out->pending = s->pending;
  out->max_merged = s->max_merge;
  out->resident_bytes = s->resident;
  if (!s->lat_us.empty()) {
    std::vector<double> v = s->lat_us;
    auto pct = [&](double p) {
      const size_t k = std::min(v.size() - 1, static_cast<size_t>(p * (v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + k, v.end());
      return v[k];
    };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    double sum = 0;
    for (double x : s->lat_us) sum += x;
    out->mean_us = sum / s->lat_us.size();
  }
  const double span = (s->t_last > s->t_first) ? (s->t_last - s->t_first) * 1e-9 : 0.0;
  if (span > 0) {
    out->throughput_rps = s->completed / span;
    out->gbs = s->bytes_done / span / 1e9;
  }
  return HM_OK;
}

extern "C" hm_status hm_serve_reset_stats(hm_server* s) {
  if (!s || s->magic != kMagicServer) return sfail(HM_EINVAL, "not a server handle");
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_us.clear();
  s->submitted = s->admitted = s->rejected = s->completed = s->launches = 0;
  s->bytes_done = 0;
  s->t_first = s->t_last = 0;
  s->max_merge = 0;
  return HM_OK;
}
