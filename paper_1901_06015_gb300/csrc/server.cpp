// Serving loop (host runtime): request queue, admission by HBM footprint, a device
// arena for the packed operands (first-fit free list with coalescing), priority
// streams for overlapping work, waves that batch the small requests admitted while the
// previous wave ran into one grouped launch, and completion tracking with CUDA events.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "grouped.h"
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
  bool wave_ok = false;   // may join a wave (a plain FFMA / DFMA / DMMA gemm)
  int stream = -1;
};

// Work in flight: one request on its own, or a wave of small requests in one grouped
// launch. The requests complete with the job's event.
struct Job {
  std::vector<Req*> reqs;
  cudaEvent_t ev = nullptr;
  bool wave = false;                      // holds the wave slot of stream 0
  size_t dev_off = 0, dev_bytes = 0;      // the wave's work lists in the arena
  size_t host_off = 0, host_bytes = 0;    // their pinned staging copy
};

constexpr size_t kHostStageBytes = 16u << 20;   // pinned staging for the waves' work lists
constexpr double kHeadAgeS = 0.05;              // a blocked head stops small requests passing it after this

}  // namespace

struct mxg_server_s {
  int device = 0;
  int flags = 0;
  int sm_count = 152;
  double small_flops = 0;
  int method_s = 0, method_d = 0;
  std::vector<cudaStream_t> streams;
  int rr = 0;
  size_t budget = 0;
  char* arena_base = nullptr;
  Arena arena;
  char* host_stage = nullptr;             // pinned
  Arena host_arena;
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
  std::vector<Job*> inflight;             // worker only
  std::vector<Req*> batch;                // worker only: admitted, waiting for the next wave
  bool wave_busy = false;                 // worker only: a wave (or a lone small request) runs on stream 0
  uint64_t head_id = 0;                   // worker only: the blocked head request and since when
  double head_since = 0;
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

// Finish every request of a job (done time and status already set) and free its
// resources.
void finish_job(mxg_server_s* s, Job* j) {
  for (Req* r : j->reqs) finish(s, r);
  if (j->dev_bytes) s->arena.release(j->dev_off, j->dev_bytes);
  if (j->host_bytes) s->host_arena.release(j->host_off, j->host_bytes);
  if (j->ev) s->ev_pool.push_back(j->ev);
  if (j->wave) s->wave_busy = false;
  delete j;
}

void fail_job(mxg_server_s* s, Job* j, int st) {
  cudaGetLastError();
  const double t = s->now();
  for (Req* r : j->reqs) {
    r->status = st;
    r->done = t;
  }
  finish_job(s, j);
}

void track(mxg_server_s* s, Job* j) {
  s->inflight.push_back(j);
  int64_t n = 0;
  for (const Job* x : s->inflight) n += static_cast<int64_t>(x->reqs.size());
  std::lock_guard<std::mutex> lk(s->mu);
  s->st.max_in_flight = std::max<int64_t>(s->st.max_in_flight, n);
}

// Reserve r's packed-operand space and count its footprint; false if it does not fit
// now. A request whose packs can never fit the arena completes at once with
// MXG_ENOMEM (*done_now).
bool admit(mxg_server_s* s, Req* r, size_t bytes_in_flight, bool* done_now) {
  *done_now = false;
  const bool nothing_in_flight = s->inflight.empty() && s->batch.empty();
  if (!nothing_in_flight && bytes_in_flight + r->footprint > s->budget) return false;
  if (r->P.kind == PLAN_GEMM) {
    if (r->P.workspace > s->budget) {   // can never fit in the arena
      r->status = MXG_ENOMEM;
      r->admit = r->done = s->now();
      finish(s, r);
      *done_now = true;
      return true;
    }
    if (!s->arena.alloc(r->P.workspace, &r->ws_off)) return false;
    r->ws_bytes = r->P.workspace;
  }
  r->admit = s->now();
  r->stream = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  s->st.admitted++;
  s->st.bytes_in_flight += r->footprint;
  s->st.peak_bytes_in_flight = std::max(s->st.peak_bytes_in_flight, s->st.bytes_in_flight);
  return true;
}

// Enqueue one admitted request on its own on stream si.
void launch_one(mxg_server_s* s, Req* r, int si, bool holds_wave) {
  Job* j = new Job();
  j->reqs.push_back(r);
  j->wave = holds_wave;
  if (holds_wave) s->wave_busy = true;
  r->stream = si;
  j->ev = take_ev(s);
  int st = j->ev ? MXG_OK : MXG_ECUDA;
  if (st == MXG_OK) st = enqueue_plan(r->P, s->arena_base + r->ws_off, s->streams[si], nullptr, s->dev_err);
  if (st == MXG_OK && cudaEventRecord(j->ev, s->streams[si]) != cudaSuccess) st = MXG_ECUDA;
  if (st != MXG_OK) {
    // part of the request may be enqueued: let it finish before its arena space is reused
    cudaStreamSynchronize(s->streams[si]);
    fail_job(s, j, st);
    return;
  }
  track(s, j);
}

// One bucket of a wave (single or double computation precision): its problems, pack
// tasks and tile work list, laid out contiguously for one host-to-device copy.
struct WaveBucket {
  int comp_double = 0, variant = -1;
  std::vector<GroupProb> probs;
  std::vector<PackArgs> tasks;
  std::vector<int64_t> tile_start{0};
  std::vector<GroupTile> tiles;
  size_t off_probs = 0, off_tiles = 0, off_tasks = 0, off_start = 0, off_counter = 0;
};

// Launch the batch as one wave on stream 0: per precision bucket one grouped pack launch
// and one persistent grouped contraction over all of the batch's tiles (the same
// kernels as mxg_group_run, so the results are those of separate calls bit for bit).
// Falls back to separate launches when the work lists do not fit.
void launch_wave(mxg_server_s* s, std::vector<Req*>& batch) {
  WaveBucket wb[2];
  wb[0].comp_double = 0;
  wb[1].comp_double = 1;
  for (Req* r : batch) {
    WaveBucket& b = wb[r->P.comp_double ? 1 : 0];
    GroupProb gp{};
    PackArgs ta{}, tb{};
    group_describe_problem(r->P, s->arena_base + r->ws_off, &gp, &ta, &tb, s->dev_err);
    b.probs.push_back(gp);
    for (const PackArgs& t : {ta, tb}) {
      b.tasks.push_back(t);
      b.tile_start.push_back(b.tile_start.back() + pack_tiles(t));
    }
  }
  size_t bytes = 0;
  for (WaveBucket& b : wb) {
    if (b.probs.empty()) continue;
    if (b.comp_double) {
      // DFMA on 32 x 32 tiles once they fill the device, else 16 x 16 for more CTAs
      const size_t t32 = group_tiles(b.probs, VAR_DFMA_32).size();
      b.variant = (s->method_d == MXG_METHOD_DMMA) ? VAR_DMMA_64
                  : (t32 >= static_cast<size_t>(2 * s->sm_count)) ? VAR_DFMA_32 : VAR_DFMA_16;
    } else {
      // 64 x 64 tiles once they fill the device, else 32 x 32 for more CTAs
      const size_t t64 = group_tiles(b.probs, VAR_FFMA_64).size();
      b.variant = (t64 >= static_cast<size_t>(2 * s->sm_count)) ? VAR_FFMA_64 : VAR_FFMA_32;
    }
    b.tiles = group_tiles(b.probs, b.variant);
    b.off_probs = bytes; bytes += al256(b.probs.size() * sizeof(GroupProb));
    b.off_tiles = bytes; bytes += al256(b.tiles.size() * sizeof(GroupTile));
    b.off_tasks = bytes; bytes += al256(b.tasks.size() * sizeof(PackArgs));
    b.off_start = bytes; bytes += al256(b.tile_start.size() * sizeof(int64_t));
    b.off_counter = bytes; bytes += 256;
  }
  Job* j = new Job();
  j->wave = true;
  j->reqs = batch;
  batch.clear();
  bool fits = bytes <= kHostStageBytes && s->host_arena.alloc(bytes, &j->host_off);
  if (fits) {
    j->host_bytes = bytes;
    fits = s->arena.alloc(bytes, &j->dev_off);
    if (fits) j->dev_bytes = bytes;
  }
  if (!fits) {
    // no room for the work lists now: the batch runs as separate launches on stream 0
    std::vector<Req*> reqs = j->reqs;
    j->reqs.clear();
    finish_job(s, j);   // releases the partial reservation and the wave slot; no requests attached
    for (size_t i = 0; i < reqs.size(); ++i) launch_one(s, reqs[i], 0, i + 1 == reqs.size());
    return;
  }
  char* h = s->host_stage + j->host_off;
  char* d = s->arena_base + j->dev_off;
  std::memset(h, 0, bytes);
  for (const WaveBucket& b : wb) {
    if (b.probs.empty()) continue;
    std::memcpy(h + b.off_probs, b.probs.data(), b.probs.size() * sizeof(GroupProb));
    std::memcpy(h + b.off_tiles, b.tiles.data(), b.tiles.size() * sizeof(GroupTile));
    std::memcpy(h + b.off_tasks, b.tasks.data(), b.tasks.size() * sizeof(PackArgs));
    std::memcpy(h + b.off_start, b.tile_start.data(), b.tile_start.size() * sizeof(int64_t));
  }
  const cudaStream_t st0 = s->streams[0];
  for (Req* r : j->reqs) r->stream = 0;
  j->ev = take_ev(s);
  cudaError_t e = j->ev ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st0) : cudaErrorMemoryAllocation;
  for (const WaveBucket& b : wb) {
    if (e != cudaSuccess || b.probs.empty()) continue;
    e = launch_pack_grouped(reinterpret_cast<const PackArgs*>(d + b.off_tasks),
                            reinterpret_cast<const int64_t*>(d + b.off_start), static_cast<int>(b.tasks.size()),
                            b.tile_start.back(), b.comp_double, st0);
  }
  for (const WaveBucket& b : wb) {
    if (e != cudaSuccess || b.probs.empty()) continue;
    const int ntiles = static_cast<int>(b.tiles.size());
    const int grid = std::min(grouped_blocks_per_sm(b.variant) * s->sm_count, ntiles);
    e = launch_gemm_grouped(b.variant, reinterpret_cast<const GroupProb*>(d + b.off_probs),
                            reinterpret_cast<const GroupTile*>(d + b.off_tiles), ntiles,
                            reinterpret_cast<int*>(d + b.off_counter), SCHED_DYNAMIC, grid, st0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(j->ev, st0);
  if (e != cudaSuccess) {
    g_last_cuda_error = static_cast<int>(e);
    // part of the wave may be enqueued: let it finish before its arena space is reused
    cudaStreamSynchronize(st0);
    fail_job(s, j, MXG_ECUDA);
    return;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.waves++;
    s->st.wave_requests += j->reqs.size();
  }
  track(s, j);
}

// Place an admitted request: small wave-eligible ones wait for the next wave, the rest
// run on their own (small ones on the high-priority stream 0, large ones round-robin
// over the others; the serial form puts everything on stream 0 in order).
void place(mxg_server_s* s, Req* r) {
  const int ns = static_cast<int>(s->streams.size());
  if (s->flags & MXG_SERVE_FIFO) { launch_one(s, r, 0, false); return; }
  if (r->small && r->wave_ok) { s->batch.push_back(r); return; }
  launch_one(s, r, (r->small || ns == 1) ? 0 : 1 + (s->rr++ % (ns - 1)), false);
}

// Start the next wave when stream 0 has no wave running: a lone request runs on its
// own, two or more as one grouped launch.
void flush_batch(mxg_server_s* s) {
  if (s->batch.empty() || s->wave_busy) return;
  s->wave_busy = true;
  if (s->batch.size() == 1) {
    Req* r = s->batch.front();
    s->batch.clear();
    launch_one(s, r, 0, true);
    return;
  }
  launch_wave(s, s->batch);
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
      s->st.queue_len = static_cast<int64_t>(s->pending.size() + s->batch.size());
      if (s->stop && s->pending.empty() && s->inflight.empty() && s->batch.empty()) break;
    }
    // completions
    for (size_t i = 0; i < s->inflight.size();) {
      Job* j = s->inflight[i];
      const cudaError_t q = cudaEventQuery(j->ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      double done = s->now();
      int st = MXG_OK;
      if (q == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->t0_ev, j->ev) == cudaSuccess) done = ms / 1e3;
        else cudaGetLastError();
      } else {
        g_last_cuda_error = static_cast<int>(q);
        cudaGetLastError();
        st = MXG_ECUDA;
      }
      for (Req* r : j->reqs) {
        r->done = done;
        if (st != MXG_OK) r->status = st;
      }
      s->inflight[i] = s->inflight.back();
      s->inflight.pop_back();
      finish_job(s, j);
      progress = true;
    }
    // admission: head first; past a blocked head only small requests (bounded scan),
    // and only while the head has waited less than kHeadAgeS
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
      bool done_now = false;
      if (!admit(s, r, bif, &done_now)) break;
      s->pending.pop_front();
      if (!done_now) place(s, r);
      progress = true;
      std::lock_guard<std::mutex> lk(s->mu);
      bif = s->st.bytes_in_flight;
    }
    const double t = s->now();
    if (s->pending.empty()) {
      s->head_id = 0;
    } else if (s->pending.front()->id != s->head_id) {
      s->head_id = s->pending.front()->id;
      s->head_since = t;
    }
    const bool head_young = s->head_id == 0 || t - s->head_since < kHeadAgeS;
    if (!(s->flags & MXG_SERVE_FIFO) && s->pending.size() > 1 && head_young) {
      int scanned = 0;
      for (auto it = std::next(s->pending.begin()); it != s->pending.end() && scanned < 256; ++scanned) {
        Req* r = *it;
        bool done_now = false;
        if (r->small && r->P.kind != PLAN_NOOP && r->status == MXG_OK && admit(s, r, bif, &done_now)) {
          it = s->pending.erase(it);
          if (!done_now) place(s, r);
          progress = true;
          std::lock_guard<std::mutex> lk(s->mu);
          bif = s->st.bytes_in_flight;
        } else {
          ++it;
        }
      }
    }
    if (!s->batch.empty() && !s->wave_busy) {
      flush_batch(s);
      progress = true;
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
  if (s->host_stage) cudaFreeHost(s->host_stage);
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
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->arena_base, al256(hbm_budget_bytes));
  if (e == cudaSuccess) e = cudaMallocHost(&s->host_stage, kHostStageBytes);
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
  s->host_arena.init(kHostStageBytes);
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
    const int m = r->P.method;
    r->wave_ok = r->P.kind == PLAN_GEMM && r->P.split == SPLIT_NONE && r->P.splits == 1 && !r->P.fold_a &&
                 !r->P.fold_b && (m == MXG_METHOD_FFMA || m == MXG_METHOD_DFMA || m == MXG_METHOD_DMMA);
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
