// Serving loop (host runtime): request queue, admission by HBM footprint, a device
// arena for the packed operands (first-fit free list with coalescing), priority
// streams for overlapping work, and completion tracking with CUDA events.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "plan.h"
#include "../../include/mxgemm.h"

namespace mxg {
extern thread_local int g_last_cuda_error;
}

using namespace mxg;

namespace {

size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// First-fit allocator over [0, size) with coalescing of freed neighbours.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = al256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t o = it->first, rem = it->second - bytes;
      free_.erase(it);
      if (rem) free_[o + bytes] = rem;
      *off = o;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al256(bytes);
    auto it = free_.emplace(off, bytes).first;
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

 private:
  std::map<size_t, size_t> free_;
};


struct Req {
  uint64_t id = 0;
  Plan P;
  int status = MXG_OK;
  double arrival = 0, admit = 0, done = 0, flops = 0;
  size_t footprint = 0, ws_off = 0, ws_bytes = 0;
  bool small = false;
  int stream = -1;
  cudaEvent_t ev = nullptr;
};

}  // namespace

struct mxg_server_s {
  int device = 0;
  int flags = 0;
  double small_flops = 0;
  int method_s = 0, method_d = 0;
  std::vector<cudaStream_t> streams;
  int rr = 0;
  size_t budget = 0;
  char* arena_base = nullptr;
  Arena arena;
  int* dev_err = nullptr;
  cudaEvent_t t0_ev = nullptr;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<Req*> incoming;              // guarded by mu
  std::deque<mxg_completion> completed;   // guarded by mu
  uint64_t next_id = 1;                   // guarded by mu
  mxg_server_stats st{};                  // guarded by mu
  bool stop = false;                      // guarded by mu
  std::deque<Req*> pending;               // worker only
  std::vector<Req*> inflight;             // worker only
  std::vector<cudaEvent_t> ev_pool;       // worker only
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

cudaEvent_t take_ev(mxg_server_s* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void finish(mxg_server_s* s, Req* r) {
  if (r->ws_bytes) s->arena.release(r->ws_off, r->ws_bytes);
  if (r->ev) s->ev_pool.push_back(r->ev);
  mxg_completion c{};
  c.id = r->id; c.status = r->status; c.stream = r->stream;
  c.arrival = r->arrival; c.admit = r->admit; c.done = r->done;
  c.flops = r->flops; c.footprint = r->footprint;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->stream >= 0) s->st.bytes_in_flight -= r->footprint;
    s->st.completed++;
    if (r->status != MXG_OK) s->st.failed++;
    s->completed.push_back(c);
  }
  s->cv_done.notify_all();
  delete r;
}

// Enqueue r; returns false if it does not fit now (budget or arena).
bool try_launch(mxg_server_s* s, Req* r, size_t bytes_in_flight) {
  const bool nothing_in_flight = s->inflight.empty();
  if (!nothing_in_flight && bytes_in_flight + r->footprint > s->budget) return false;
  if (r->P.kind == PLAN_GEMM) {
    if (r->P.workspace > s->budget) {   // can never fit in the arena
      r->status = MXG_ENOMEM;
      r->admit = r->done = s->now();
      finish(s, r);
      return true;
    }
    if (!s->arena.alloc(r->P.workspace, &r->ws_off)) return false;
    r->ws_bytes = r->P.workspace;
  }
  const int ns = static_cast<int>(s->streams.size());
  int si = 0;
  if (!(s->flags & MXG_SERVE_FIFO) && ns > 1) si = r->small ? 0 : 1 + (s->rr++ % (ns - 1));
  r->stream = si;
  r->ev = take_ev(s);
  r->admit = s->now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.admitted++;
    s->st.bytes_in_flight += r->footprint;
    s->st.peak_bytes_in_flight = std::max(s->st.peak_bytes_in_flight, s->st.bytes_in_flight);
  }
  int st = r->ev ? MXG_OK : MXG_ECUDA;
  if (st == MXG_OK) st = enqueue_plan(r->P, s->arena_base + r->ws_off, s->streams[si], nullptr, s->dev_err);
  if (st == MXG_OK && cudaEventRecord(r->ev, s->streams[si]) != cudaSuccess) st = MXG_ECUDA;
  if (st != MXG_OK) {
    cudaGetLastError();
    r->status = st;
    r->done = s->now();
    finish(s, r);
    return true;
  }
  s->inflight.push_back(r);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.max_in_flight = std::max<int64_t>(s->st.max_in_flight, static_cast<int64_t>(s->inflight.size()));
  }
  return true;
}

void worker_main(mxg_server_s* s) {
  cudaSetDevice(s->device);
  for (;;) {
    bool progress = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->incoming.empty()) {
        s->pending.push_back(s->incoming.front());
        s->incoming.pop_front();
        progress = true;
      }
      s->st.queue_len = static_cast<int64_t>(s->pending.size());
      if (s->stop && s->pending.empty() && s->inflight.empty()) break;
    }
    // completions
    for (size_t i = 0; i < s->inflight.size();) {
      Req* r = s->inflight[i];
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (q == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->t0_ev, r->ev) == cudaSuccess) r->done = ms / 1e3;
        else { cudaGetLastError(); r->done = s->now(); }
      } else {
        g_last_cuda_error = static_cast<int>(q);
        cudaGetLastError();
        r->status = MXG_ECUDA;
        r->done = s->now();
      }
      s->inflight[i] = s->inflight.back();
      s->inflight.pop_back();
      finish(s, r);
      progress = true;
    }
    // admission: head first; past a blocked head only small requests (bounded scan)
    size_t bif;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      bif = s->st.bytes_in_flight;
    }
    while (!s->pending.empty()) {
      Req* r = s->pending.front();
      if (r->P.kind == PLAN_NOOP || r->status != MXG_OK) {
        s->pending.pop_front();
        r->admit = r->done = s->now();
        finish(s, r);
        progress = true;
        continue;
      }
      if (!try_launch(s, r, bif)) break;
      s->pending.pop_front();
      progress = true;
      std::lock_guard<std::mutex> lk(s->mu);
      bif = s->st.bytes_in_flight;
    }
    if (!(s->flags & MXG_SERVE_FIFO) && s->pending.size() > 1) {
      int scanned = 0;
      for (auto it = std::next(s->pending.begin()); it != s->pending.end() && scanned < 256; ++scanned) {
        Req* r = *it;
        if (r->small && r->P.kind != PLAN_NOOP && r->status == MXG_OK && try_launch(s, r, bif)) {
          it = s->pending.erase(it);
          progress = true;
          std::lock_guard<std::mutex> lk(s->mu);
          bif = s->st.bytes_in_flight;
        } else {
          ++it;
        }
      }
    }
    if (!progress) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_submit.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 2000 : 20));
    }
  }
}

void destroy_server(mxg_server_s* s) {
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_submit.notify_all();
    s->worker.join();
  }
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->t0_ev) cudaEventDestroy(s->t0_ev);
  if (s->arena_base) cudaFree(s->arena_base);
  if (s->dev_err) cudaFree(s->dev_err);
  delete s;
}

}  // namespace

extern "C" {

int mxg_server_create(int n_streams, size_t hbm_budget_bytes, double small_flops, int method_s, int method_d,
                      int flags, mxg_server* out) {
  if (!out || n_streams < 1 || n_streams > 64 || hbm_budget_bytes == 0) return MXG_EINVAL;
  if (method_s < MXG_METHOD_AUTO || method_s > MXG_METHOD_DFMA || method_d < MXG_METHOD_AUTO ||
      method_d > MXG_METHOD_DFMA)
    return MXG_EINVAL;
  mxg_server_s* s = new (std::nothrow) mxg_server_s();
  if (!s) return MXG_ENOMEM;
  s->flags = flags;
  s->small_flops = small_flops;
  s->method_s = method_s;
  s->method_d = method_d;
  s->budget = hbm_budget_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  int lo = 0, hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  for (int i = 0; e == cudaSuccess && i < n_streams; ++i) {
    cudaStream_t st = nullptr;
    const int prio = ((flags & MXG_SERVE_FIFO) || i > 0) ? lo : hi;   // stream 0: high priority
    e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio);
    if (e == cudaSuccess) s->streams.push_back(st);
  }
  if (e == cudaSuccess) e = cudaMalloc(&s->arena_base, al256(hbm_budget_bytes));
  if (e == cudaSuccess) e = cudaMalloc(&s->dev_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(s->dev_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&s->t0_ev);
  if (e == cudaSuccess) e = cudaEventRecord(s->t0_ev, s->streams[0]);
  if (e == cudaSuccess) e = cudaEventSynchronize(s->t0_ev);
  if (e != cudaSuccess) {
    g_last_cuda_error = static_cast<int>(e);
    cudaGetLastError();
    destroy_server(s);
    return e == cudaErrorMemoryAllocation ? MXG_ENOMEM : MXG_ECUDA;
  }
  s->t0 = std::chrono::steady_clock::now();
  s->arena.init(al256(hbm_budget_bytes));
  s->st.budget = hbm_budget_bytes;
  s->worker = std::thread(worker_main, s);
  *out = s;
  return MXG_OK;
}

int mxg_server_submit(mxg_server s, const mxg_problem* p, uint64_t* id) {
  if (!s || !p) return MXG_EINVAL;
  Req* r = new (std::nothrow) Req();
  if (!r) return MXG_ENOMEM;
  r->arrival = s->now();
  Call c{};
  c.transa = p->transa; c.transb = p->transb; c.m = p->m; c.n = p->n; c.k = p->k;
  c.alpha_re = p->alpha_re; c.alpha_im = p->alpha_im; c.beta_re = p->beta_re; c.beta_im = p->beta_im;
  c.A = p->A; c.dtA = p->dtA; c.rsA = p->rsA; c.csA = p->csA;
  c.B = p->B; c.dtB = p->dtB; c.rsB = p->rsB; c.csB = p->csB;
  c.C = p->C; c.dtC = p->dtC; c.rsC = p->rsC; c.csC = p->csC; c.comp = p->comp_prec;
  Plan probe;
  int st = make_plan(c, MXG_METHOD_AUTO, &probe);
  if (st == MXG_OK) st = make_plan(c, probe.comp_double ? s->method_d : s->method_s, &r->P);
  if (st == MXG_OK && r->P.kind != PLAN_NOOP && !c.C) st = MXG_EINVAL;
  if (st == MXG_OK && r->P.kind == PLAN_GEMM && (!c.A || !c.B)) st = MXG_EINVAL;
  r->status = st;
  if (st == MXG_OK) {
    r->flops = 2.0 * static_cast<double>(c.m) * c.n * c.k * r->P.real_products;
    r->small = r->flops <= s->small_flops;
    r->footprint = static_cast<size_t>(c.m * c.k) * dt_bytes(c.dtA) + static_cast<size_t>(c.k * c.n) * dt_bytes(c.dtB) +
                   static_cast<size_t>(c.m * c.n) * dt_bytes(c.dtC) + (r->P.kind == PLAN_GEMM ? r->P.workspace : 0);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->st.submitted++;
    s->incoming.push_back(r);
  }
  if (id) *id = r->id;
  s->cv_submit.notify_one();
  return MXG_OK;
}

int mxg_server_poll(mxg_server s, mxg_completion* out, int max, int* n) {
  if (!s || !n || (max > 0 && !out)) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  int k = 0;
  while (k < max && !s->completed.empty()) {
    out[k++] = s->completed.front();
    s->completed.pop_front();
  }
  *n = k;
  return MXG_OK;
}

int mxg_server_drain(mxg_server s, double timeout_s) {
  if (!s) return MXG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [s] { return s->st.completed == s->st.submitted; });
  return ok ? MXG_OK : MXG_ETIMEOUT;
}

int mxg_server_get_stats(mxg_server s, mxg_server_stats* st) {
  if (!s || !st) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->st;
  return MXG_OK;
}

int mxg_server_check_device_error(mxg_server s, int* flag) {
  if (!s || !flag) return MXG_EINVAL;
  for (cudaStream_t st : s->streams) {   // the work already enqueued by the worker
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      g_last_cuda_error = static_cast<int>(e);
      cudaGetLastError();
      return MXG_ECUDA;
    }
  }
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(s->dev_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    g_last_cuda_error = static_cast<int>(e);
    cudaGetLastError();
    return MXG_ECUDA;
  }
  *flag = v;
  return MXG_OK;
}

double mxg_server_now(mxg_server s) { return s ? s->now() : 0.0; }

int mxg_server_destroy(mxg_server s) {
  if (!s) return MXG_EINVAL;
  destroy_server(s);
  return MXG_OK;
}

}  // extern "C"
