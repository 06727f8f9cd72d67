// Grouped persistent launch (host side): plan every problem, lay out one device arena
// (packed operands, work lists, counters), autotune each bucket's kernel and tile
// schedule, and optionally capture the run in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "context.h"
#include "grouped.h"
#include "plan.h"
#include "../../include/mxgemm.h"

namespace mxg {
extern thread_local int g_last_cuda_error;
}

namespace mxg {

std::vector<GroupTile> group_tiles(const std::vector<GroupProb>& probs, int variant) {
  const int T = variant_tile(variant);
  std::vector<std::pair<int64_t, GroupTile>> v;
  for (size_t i = 0; i < probs.size(); ++i) {
    const GroupProb& p = probs[i];
    // logical extent of the real product: the epilogue's C extent times the pairing
    const int64_t Mr = p.e.m * (p.mode == OUT_ROWPAIR ? 2 : 1);
    const int64_t Nr = p.e.n * (p.mode == OUT_COLPAIR ? 2 : 1);
    const int tm = static_cast<int>((Mr + T - 1) / T), tn = static_cast<int>((Nr + T - 1) / T);
    for (int x = 0; x < tm; ++x)
      for (int y = 0; y < tn; ++y) v.push_back({p.Kp, GroupTile{static_cast<int>(i), x, y}});
  }
  std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<GroupTile> out;
  out.reserve(v.size());
  for (auto& e : v) out.push_back(e.second);
  return out;
}

void group_describe_problem(const Plan& P, char* pa, GroupProb* gp, PackArgs* ta, PackArgs* tb, int* dbg) {
  const Call& w = P.work;
  char* pb = pa + P.bytes_a;
  *gp = GroupProb{};
  gp->A = pa; gp->B = pb;
  gp->lda = P.Mp; gp->ldb = P.Np; gp->Kp = P.Kp;
  gp->e = plan_epilogue(P);
  gp->cdt = w.dtC;
  gp->mode = P.mode;
  *ta = PackArgs{};
  ta->src = w.A; ta->src_dt = w.dtA;
  if (w.transa == MXG_TRANS || w.transa == MXG_CONJTRANS) { ta->smn = w.csA; ta->sk = w.rsA; }
  else { ta->smn = w.rsA; ta->sk = w.csA; }
  ta->MN = w.m; ta->K = w.k; ta->pattern = P.pat_a; ta->conj = P.conj_a;
  ta->dst = pa; ta->ld = P.Mp; ta->MNp = P.Mp; ta->Kp = P.Kp; ta->layout = LAYOUT_MN_MAJOR; ta->split = SPLIT_NONE;
  *tb = PackArgs{};
  tb->src = w.B; tb->src_dt = w.dtB;
  if (w.transb == MXG_TRANS || w.transb == MXG_CONJTRANS) { tb->smn = w.rsB; tb->sk = w.csB; }
  else { tb->smn = w.csB; tb->sk = w.rsB; }
  tb->MN = w.n; tb->K = w.k; tb->pattern = P.pat_b; tb->conj = P.conj_b;
  tb->dst = pb; tb->ld = P.Np; tb->MNp = P.Np; tb->Kp = P.Kp; tb->layout = LAYOUT_MN_MAJOR; tb->split = SPLIT_NONE;
  gp->e.dbg = ta->dbg = tb->dbg = dbg;
}

}  // namespace mxg

using namespace mxg;

namespace {

int cstat(cudaError_t e) {
  if (e == cudaSuccess) return MXG_OK;
  g_last_cuda_error = static_cast<int>(e);
  return e == cudaErrorMemoryAllocation ? MXG_ENOMEM : MXG_ECUDA;
}

size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct TuneRec { int variant, sched; double ms; };
std::mutex g_tune_mu;
std::map<std::string, TuneRec> g_tune;

struct Bucket {
  int comp_double = 0;
  int plan_method = 0;              // method whose padding the packs use
  std::vector<int> candidates;      // GroupVariant
  int variant = -1, sched = SCHED_DYNAMIC;
  double tuned_ms = -1.0;
  bool from_cache = false;
  std::vector<int> members;         // indices into plans (GEMM problems of this bucket)
  std::vector<GroupProb> probs;     // host copy, same order as members
  std::vector<PackArgs> tasks;
  std::vector<int64_t> tile_start;  // ntasks + 1
  int ntiles = 0;                   // for the chosen variant
  int max_tiles = 0;                // over the candidates
  // device pointers into the arena
  GroupProb* d_probs = nullptr;
  GroupTile* d_tiles = nullptr;
  PackArgs* d_tasks = nullptr;
  int64_t* d_tile_start = nullptr;
  int* d_counter = nullptr;
  std::string signature;
  // tensor-core buckets (split forms, TC16): plane format, problems with their maps
  int tc_split = SPLIT_NONE;
  std::vector<TcGroupProb> tcprobs;
  std::vector<GroupTile> tctiles;
  TcGroupProb* d_tcprobs = nullptr;
};

// Buckets of a group: plain single and double precision (SIMT / DMMA kernels), and the
// tensor-core ones: single precision on the split method the caller chose, and the two
// 16-bit computation precisions.
enum { BK_S = 0, BK_D = 1, BK_S_TC = 2, BK_H = 3, BK_B = 4, NBUCKETS = 5 };

// (problem, tile) work list of a tensor-core bucket: 128 x 256 tiles of each problem's
// padded real product, longest K' first.
std::vector<GroupTile> tc_tiles(const std::vector<Plan>& plans, const std::vector<int>& members) {
  std::vector<std::pair<int64_t, GroupTile>> v;
  for (size_t j = 0; j < members.size(); ++j) {
    const Plan& P = plans[members[j]];
    for (int64_t x = 0; x < P.Mp / 128; ++x)
      for (int64_t y = 0; y < P.Np / 256; ++y)
        v.push_back({P.Kp, GroupTile{static_cast<int>(j), static_cast<int>(x), static_cast<int>(y)}});
  }
  std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<GroupTile> out;
  out.reserve(v.size());
  for (auto& e : v) out.push_back(e.second);
  return out;
}

std::vector<GroupTile> make_tiles(const Bucket& b, int variant) { return group_tiles(b.probs, variant); }

}  // namespace

struct mxg_group_s {
  mxg_context* h = nullptr;
  int sm_count = 152;
  std::vector<Plan> plans;
  std::vector<int> scale_list;      // PLAN_SCALE problems
  Bucket buckets[NBUCKETS];         // BK_*
  std::vector<int> bucket_of;       // bucket of each GEMM problem
  void* arena = nullptr;
  size_t arena_bytes = 0;
  size_t counters_off = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int enqueue_run(mxg_group_s* g, cudaStream_t s, bool packs, bool gemms, const Bucket* only = nullptr) {
  if (gemms && !only) {
    cudaError_t e = cudaMemsetAsync(static_cast<char*>(g->arena) + g->counters_off, 0, NBUCKETS * 64, s);
    if (e != cudaSuccess) return cstat(e);
  }
  for (const Bucket& b : g->buckets) {
    if (only && &b != only) continue;
    if (packs && !b.tasks.empty()) {
      const int nt = static_cast<int>(b.tasks.size());
      int st = cstat(b.tc_split != SPLIT_NONE
                         ? launch_pack_grouped_tc(b.d_tasks, b.d_tile_start, nt, b.tile_start.back(), b.tc_split, s)
                         : launch_pack_grouped(b.d_tasks, b.d_tile_start, nt, b.tile_start.back(), b.comp_double, s));
      if (st) return st;
    }
  }
  if (gemms) {
    for (const Bucket& b : g->buckets) {
      if (only && &b != only) continue;
      if (b.ntiles == 0) continue;
      if (b.tc_split != SPLIT_NONE) {
        int st = cstat(launch_gemm_tc_grouped(b.tc_split, b.d_tcprobs, b.d_tiles, b.ntiles, g->h->dev_err, s));
        if (st) return st;
        continue;
      }
      const int grid = grouped_blocks_per_sm(b.variant) * g->sm_count;
      int st = cstat(launch_gemm_grouped(b.variant, b.d_probs, b.d_tiles, b.ntiles, b.d_counter, b.sched,
                                         std::min(grid, b.ntiles), s));
      if (st) return st;
    }
    if (!only) {
      for (int i : g->scale_list) {
        const Plan& P = g->plans[i];
        EpiArgs e = plan_epilogue(P);
        e.ar = 0.0; e.ai = 0.0;
        e.dbg = g->h->dev_err;
        int st = cstat(launch_scale_c(e, P.call.dtC, s));
        if (st) return st;
      }
    }
  }
  return MXG_OK;
}

std::string bucket_signature(const Bucket& b, const std::vector<Plan>& plans) {
  // problems count, total useful flops and mean K' on a log2 scale
  double fl = 0.0, kk = 0.0;
  for (int i : b.members) {
    const Plan& P = plans[i];
    fl += 2.0 * P.Mr * P.Nr * P.Kr;
    kk += static_cast<double>(P.Kr);
  }
  const int n = static_cast<int>(b.members.size());
  char buf[160];
  std::snprintf(buf, sizeof(buf), "d%d-m%d-n%d-f%d-k%d", b.comp_double, b.plan_method,
                n > 0 ? static_cast<int>(std::lround(std::log2(static_cast<double>(n)) * 2)) : -1,
                fl > 0 ? static_cast<int>(std::lround(std::log2(fl) * 2)) : -1,
                n > 0 ? static_cast<int>(std::lround(std::log2(kk / n + 1) * 2)) : -1);
  return buf;
}

// Time every candidate (variant, schedule) of bucket b, writing into scratch C, and
// keep the fastest.
int tune_bucket(mxg_group_s* g, Bucket& b) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(b.signature);
    if (it != g_tune.end() &&
        std::find(b.candidates.begin(), b.candidates.end(), it->second.variant) != b.candidates.end()) {
      b.variant = it->second.variant;
      b.sched = it->second.sched;
      b.tuned_ms = it->second.ms;
      b.from_cache = true;
      return MXG_OK;
    }
  }
  // scratch C: a dense column-major copy-sized buffer per problem, zeroed
  size_t bytes = 0;
  std::vector<size_t> off(b.probs.size());
  for (size_t i = 0; i < b.probs.size(); ++i) {
    const GroupProb& p = b.probs[i];
    const size_t es = dt_bytes(p.cdt);
    off[i] = bytes;
    bytes += al256(static_cast<size_t>(p.e.m) * p.e.n * es);
  }
  const size_t probs_bytes = al256(b.probs.size() * sizeof(GroupProb));
  const size_t tiles_bytes = al256(static_cast<size_t>(b.max_tiles) * sizeof(GroupTile));
  char* scratch = nullptr;
  cudaError_t e = cudaMalloc(&scratch, bytes + probs_bytes + tiles_bytes + 256);
  if (e != cudaSuccess) return cstat(e);
  std::vector<GroupProb> sp = b.probs;
  for (size_t i = 0; i < sp.size(); ++i) {
    sp[i].e.C = scratch + off[i];
    sp[i].e.rs = 1;
    sp[i].e.cs = sp[i].e.m;
  }
  GroupProb* d_sp = reinterpret_cast<GroupProb*>(scratch + bytes);
  GroupTile* d_st = reinterpret_cast<GroupTile*>(scratch + bytes + probs_bytes);
  int* d_cnt = reinterpret_cast<int*>(scratch + bytes + probs_bytes + tiles_bytes);
  cudaStream_t s = g->cap_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = MXG_OK;
  if ((e = cudaMemsetAsync(scratch, 0, bytes, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_sp, sp.data(), sp.size() * sizeof(GroupProb), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = cstat(e);
  }
  double best = 1e30;
  int best_v = b.candidates.empty() ? -1 : b.candidates[0], best_s = SCHED_DYNAMIC;
  for (int v : b.candidates) {
    if (st) break;
    std::vector<GroupTile> tl = make_tiles(b, v);
    if ((e = cudaMemcpyAsync(d_st, tl.data(), tl.size() * sizeof(GroupTile), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
      st = cstat(e);
      break;
    }
    const int grid = std::min(grouped_blocks_per_sm(v) * g->sm_count, static_cast<int>(tl.size()));
    for (int sched : {SCHED_DYNAMIC, SCHED_STATIC}) {
      double t_best = 1e30;
      for (int rep = 0; rep < 3 && !st; ++rep) {
        cudaMemsetAsync(d_cnt, 0, sizeof(int), s);
        cudaEventRecord(e0, s);
        e = launch_gemm_grouped(v, d_sp, d_st, static_cast<int>(tl.size()), d_cnt, sched, grid, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { st = cstat(e); break; }
        if (rep > 0) t_best = std::min(t_best, static_cast<double>(ms));   // first run warms up
      }
      if (!st && t_best < best) {
        best = t_best;
        best_v = v;
        best_s = sched;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(scratch);
  if (st) return st;
  b.variant = best_v;
  b.sched = best_s;
  b.tuned_ms = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[b.signature] = TuneRec{best_v, best_s, best};
  return MXG_OK;
}

// Time a tensor-core bucket's contraction (three runs, best of the last two) into
// scratch copies of C, so the problems' C are not touched; recorded as tuned_ms.
int time_tc_bucket(mxg_group_s* g, Bucket& b) {
  size_t bytes = 0;
  std::vector<size_t> off(b.tcprobs.size());
  for (size_t i = 0; i < b.tcprobs.size(); ++i) {
    const TcGroupProb& p = b.tcprobs[i];
    off[i] = bytes;
    bytes += al256(static_cast<size_t>(p.e.m) * p.e.n * dt_bytes(p.cdt));
  }
  const size_t probs_bytes = al256(b.tcprobs.size() * sizeof(TcGroupProb));
  char* scratch = nullptr;
  cudaError_t e = cudaMalloc(&scratch, bytes + probs_bytes);
  if (e != cudaSuccess) return cstat(e);
  std::vector<TcGroupProb> sp = b.tcprobs;
  for (size_t i = 0; i < sp.size(); ++i) {
    sp[i].e.C = scratch + probs_bytes + off[i];
    sp[i].e.rs = 1;
    sp[i].e.cs = sp[i].e.m;
  }
  TcGroupProb* d_sp = reinterpret_cast<TcGroupProb*>(scratch);
  cudaStream_t s = g->cap_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = MXG_OK;
  if ((e = cudaMemsetAsync(scratch + probs_bytes, 0, bytes, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_sp, sp.data(), sp.size() * sizeof(TcGroupProb), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
    st = cstat(e);
  double best = 1e30;
  for (int rep = 0; rep < 3 && !st; ++rep) {
    cudaEventRecord(e0, s);
    e = launch_gemm_tc_grouped(b.tc_split, d_sp, b.d_tiles, b.ntiles, g->h->dev_err, s);
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { st = cstat(e); break; }
    if (rep > 0) best = std::min(best, static_cast<double>(ms));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(scratch);
  if (st) return st;
  b.tuned_ms = best;
  return MXG_OK;
}

void free_group(mxg_group_s* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  if (g->arena) cudaFree(g->arena);
  delete g;
}

// The four K-major planes of a planned tensor-core problem whose packs start at pa
// (A hi, A lo, B hi, B lo; the one-plane formats repeat hi), and its two pack tasks.
void tc_describe_problem(const Plan& P, char* pa, const void* planes[4], PackArgs* ta, PackArgs* tb, int* dbg) {
  const Call& w = P.work;
  const bool one = (P.method == MXG_METHOD_TC16);
  char* pb = pa + P.bytes_a;
  planes[0] = pa;
  planes[1] = one ? pa : pa + P.plane_a;
  planes[2] = pb;
  planes[3] = one ? pb : pb + P.plane_b;
  *ta = PackArgs{};
  ta->src = w.A; ta->src_dt = w.dtA;
  if (w.transa == MXG_TRANS || w.transa == MXG_CONJTRANS) { ta->smn = w.csA; ta->sk = w.rsA; }
  else { ta->smn = w.rsA; ta->sk = w.csA; }
  ta->MN = w.m; ta->K = w.k; ta->pattern = P.pat_a; ta->conj = P.conj_a;
  ta->dst = pa; ta->dst_lo = one ? nullptr : pa + P.plane_a;
  ta->ld = P.Kp; ta->MNp = P.Mp; ta->Kp = P.Kp; ta->layout = LAYOUT_K_MAJOR; ta->split = P.split;
  *tb = PackArgs{};
  tb->src = w.B; tb->src_dt = w.dtB;
  if (w.transb == MXG_TRANS || w.transb == MXG_CONJTRANS) { tb->smn = w.rsB; tb->sk = w.csB; }
  else { tb->smn = w.csB; tb->sk = w.rsB; }
  tb->MN = w.n; tb->K = w.k; tb->pattern = P.pat_b; tb->conj = P.conj_b;
  tb->dst = pb; tb->dst_lo = one ? nullptr : pb + P.plane_b;
  tb->ld = P.Kp; tb->MNp = P.Np; tb->Kp = P.Kp; tb->layout = LAYOUT_K_MAJOR; tb->split = P.split;
  ta->dbg = tb->dbg = dbg;
}

int build_group(mxg_handle h, int64_t count, const mxg_problem* probs, int method_s, int method_d, int flags,
                mxg_group_s* g, int64_t* first_bad) {
  if (method_s != MXG_METHOD_AUTO && method_s != MXG_METHOD_FFMA && method_s != MXG_METHOD_TF32X3 &&
      method_s != MXG_METHOD_BF16X3)
    return MXG_EINVAL;
  if (method_d != MXG_METHOD_AUTO && method_d != MXG_METHOD_DMMA && method_d != MXG_METHOD_DFMA) return MXG_EINVAL;
  cudaError_t e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) return cstat(e);
  Bucket& bs = g->buckets[BK_S];
  Bucket& bd = g->buckets[BK_D];
  bs.comp_double = 0;
  bs.plan_method = MXG_METHOD_FFMA;
  bs.candidates = {VAR_FFMA_128, VAR_FFMA_64, VAR_FFMA_32};
  bd.comp_double = 1;
  // AUTO means DFMA for double precision, as in a single call (faster than DMMA on this
  // chip); planning with the DFMA tile pads K' to 8 instead of the DMMA kernel's 16
  bd.plan_method = (method_d == MXG_METHOD_DMMA) ? MXG_METHOD_DMMA : MXG_METHOD_DFMA;
  bd.candidates = (method_d == MXG_METHOD_DMMA) ? std::vector<int>{VAR_DMMA_64}
                                                : std::vector<int>{VAR_DFMA_32, VAR_DFMA_64, VAR_DFMA_16};
  const bool split_s = (method_s == MXG_METHOD_TF32X3 || method_s == MXG_METHOD_BF16X3);
  g->buckets[BK_S_TC].plan_method = method_s;
  g->buckets[BK_S_TC].tc_split = (method_s == MXG_METHOD_BF16X3) ? SPLIT_BF16 : SPLIT_TF32;
  g->buckets[BK_H].plan_method = MXG_METHOD_TC16;
  g->buckets[BK_H].tc_split = SPLIT_F16_ONE;
  g->buckets[BK_B].plan_method = MXG_METHOD_TC16;
  g->buckets[BK_B].tc_split = SPLIT_BF16_ONE;
  g->plans.resize(static_cast<size_t>(count));
  g->bucket_of.assign(static_cast<size_t>(count), BK_S);
  for (int64_t i = 0; i < count; ++i) {
    const mxg_problem& q = probs[i];
    Call c{};
    c.transa = q.transa; c.transb = q.transb; c.m = q.m; c.n = q.n; c.k = q.k;
    c.alpha_re = q.alpha_re; c.alpha_im = q.alpha_im; c.beta_re = q.beta_re; c.beta_im = q.beta_im;
    c.A = q.A; c.dtA = q.dtA; c.rsA = q.rsA; c.csA = q.csA;
    c.B = q.B; c.dtB = q.dtB; c.rsB = q.rsB; c.csB = q.csB;
    c.C = q.C; c.dtC = q.dtC; c.rsC = q.rsC; c.csC = q.csC; c.comp = q.comp_prec;
    // resolve the precision first, then plan with the bucket's padding method
    Plan probe;
    int st = make_plan(c, MXG_METHOD_AUTO, &probe);
    int bi = BK_S;
    if (st == MXG_OK) {
      bi = (probe.comp == MXG_PREC_H) ? BK_H : (probe.comp == MXG_PREC_B) ? BK_B
           : probe.comp_double ? BK_D : (split_s ? BK_S_TC : BK_S);
      st = make_plan(c, g->buckets[bi].plan_method, &g->plans[i]);
      // below a split method's smallest k (MXG_EACCURACY) the problem runs on FFMA
      if (st == MXG_EACCURACY && bi == BK_S_TC) {
        bi = BK_S;
        st = make_plan(c, bs.plan_method, &g->plans[i]);
      }
    }
    g->bucket_of[i] = bi;
    if (st == MXG_OK) {
      const Plan& P = g->plans[i];
      if (P.kind != PLAN_NOOP && !c.C) st = MXG_EINVAL;
      if (P.kind == PLAN_GEMM && (!c.A || !c.B)) st = MXG_EINVAL;
    }
    if (st != MXG_OK) {
      if (first_bad) *first_bad = i;
      return st;
    }
  }
  // arena layout: packed operands, then per-bucket arrays, then counters
  size_t off = 0;
  std::vector<size_t> pack_off(g->plans.size(), 0);
  for (size_t i = 0; i < g->plans.size(); ++i) {
    const Plan& P = g->plans[i];
    if (P.kind == PLAN_SCALE) g->scale_list.push_back(static_cast<int>(i));
    if (P.kind != PLAN_GEMM) continue;
    pack_off[i] = off;
    off += al256(P.workspace);
    g->buckets[g->bucket_of[i]].members.push_back(static_cast<int>(i));
  }
  for (Bucket& b : g->buckets) {
    if (b.tc_split != SPLIT_NONE) {
      b.tctiles = tc_tiles(g->plans, b.members);
      b.max_tiles = static_cast<int>(b.tctiles.size());
      b.signature = bucket_signature(b, g->plans);
      continue;
    }
    for (int i : b.members) {
      const Plan& P = g->plans[i];
      GroupProb gp{};
      gp.lda = P.Mp; gp.ldb = P.Np; gp.Kp = P.Kp;
      gp.e = plan_epilogue(P);
      gp.cdt = P.work.dtC;
      gp.mode = P.mode;
      b.probs.push_back(gp);
    }
    b.max_tiles = 0;
    for (int v : b.candidates) b.max_tiles = std::max(b.max_tiles, static_cast<int>(make_tiles(b, v).size()));
    b.signature = bucket_signature(b, g->plans);
  }
  size_t arr_off[NBUCKETS][4];
  for (int bi = 0; bi < NBUCKETS; ++bi) {
    Bucket& b = g->buckets[bi];
    const size_t prob_bytes = (b.tc_split != SPLIT_NONE) ? sizeof(TcGroupProb) : sizeof(GroupProb);
    arr_off[bi][0] = off; off += al256(b.members.size() * prob_bytes);
    arr_off[bi][1] = off; off += al256(static_cast<size_t>(b.max_tiles) * sizeof(GroupTile));
    arr_off[bi][2] = off; off += al256(2 * b.members.size() * sizeof(PackArgs));
    arr_off[bi][3] = off; off += al256((2 * b.members.size() + 1) * sizeof(int64_t));
  }
  g->counters_off = off;
  off += NBUCKETS * 64;
  g->arena_bytes = off;
  e = cudaMalloc(&g->arena, g->arena_bytes);
  if (e != cudaSuccess) return cstat(e);
  char* base = static_cast<char*>(g->arena);
  e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cstat(e);
  // pack tasks (two per problem) and the problems' packed operand pointers
  for (int bi = 0; bi < NBUCKETS; ++bi) {
    Bucket& b = g->buckets[bi];
    const bool tc = (b.tc_split != SPLIT_NONE);
    b.d_probs = tc ? nullptr : reinterpret_cast<GroupProb*>(base + arr_off[bi][0]);
    b.d_tcprobs = tc ? reinterpret_cast<TcGroupProb*>(base + arr_off[bi][0]) : nullptr;
    b.d_tiles = reinterpret_cast<GroupTile*>(base + arr_off[bi][1]);
    b.d_tasks = reinterpret_cast<PackArgs*>(base + arr_off[bi][2]);
    b.d_tile_start = reinterpret_cast<int64_t*>(base + arr_off[bi][3]);
    b.d_counter = reinterpret_cast<int*>(base + g->counters_off + 64 * bi);
    b.tile_start.assign(1, 0);
    if (tc) b.tcprobs.resize(b.members.size());
    for (size_t j = 0; j < b.members.size(); ++j) {
      const Plan& P = g->plans[b.members[j]];
      PackArgs ta{}, tb{};
      if (tc) {
        const void* planes[4];
        tc_describe_problem(P, base + pack_off[b.members[j]], planes, &ta, &tb, h->dev_err);
        EpiArgs ep = plan_epilogue(P);
        ep.dbg = h->dev_err;
        if (!tc_group_problem(&b.tcprobs[j], P.split, planes, P.Mp, P.Np, P.Kp, ep, P.work.dtC, P.mode))
          return MXG_ENOTSUP;
      } else {
        group_describe_problem(P, base + pack_off[b.members[j]], &b.probs[j], &ta, &tb, h->dev_err);
      }
      for (const PackArgs& t : {ta, tb}) {
        b.tasks.push_back(t);
        b.tile_start.push_back(b.tile_start.back() + pack_tiles(t));
      }
    }
    if (!b.members.empty()) {
      e = tc ? cudaMemcpyAsync(b.d_tcprobs, b.tcprobs.data(), b.tcprobs.size() * sizeof(TcGroupProb),
                               cudaMemcpyHostToDevice, g->cap_stream)
             : cudaMemcpyAsync(b.d_probs, b.probs.data(), b.probs.size() * sizeof(GroupProb), cudaMemcpyHostToDevice,
                               g->cap_stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.d_tasks, b.tasks.data(), b.tasks.size() * sizeof(PackArgs), cudaMemcpyHostToDevice, g->cap_stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.d_tile_start, b.tile_start.data(), b.tile_start.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice, g->cap_stream);
      if (e != cudaSuccess) return cstat(e);
    }
  }
  // choose each bucket's kernel and schedule
  for (Bucket& b : g->buckets) {
    if (b.members.empty()) continue;
    if (b.tc_split != SPLIT_NONE) {   // one kernel, static schedule over the longest-first list
      b.ntiles = static_cast<int>(b.tctiles.size());
      e = cudaMemcpyAsync(b.d_tiles, b.tctiles.data(), b.tctiles.size() * sizeof(GroupTile), cudaMemcpyHostToDevice,
                          g->cap_stream);
      if (e != cudaSuccess) return cstat(e);
      if (flags & MXG_GROUP_TUNE) {   // time it like the other buckets, for the description
        int st = enqueue_run(g, g->cap_stream, true, false, &b);
        if (st) return st;
        st = time_tc_bucket(g, b);
        if (st) return st;
      }
      continue;
    }
    if (flags & MXG_GROUP_TUNE) {
      // the packs must exist before the contraction candidates are timed
      int st = enqueue_run(g, g->cap_stream, true, false, &b);
      if (st) return st;
      st = tune_bucket(g, b);
      if (st) return st;
    } else {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(b.signature);
      if (it != g_tune.end() &&
          std::find(b.candidates.begin(), b.candidates.end(), it->second.variant) != b.candidates.end()) {
        b.variant = it->second.variant;
        b.sched = it->second.sched;
        b.tuned_ms = it->second.ms;
        b.from_cache = true;
      } else {
        b.variant = b.candidates[0];
        b.sched = SCHED_DYNAMIC;
      }
    }
    std::vector<GroupTile> tl = make_tiles(b, b.variant);
    b.ntiles = static_cast<int>(tl.size());
    e = cudaMemcpyAsync(b.d_tiles, tl.data(), tl.size() * sizeof(GroupTile), cudaMemcpyHostToDevice, g->cap_stream);
    if (e != cudaSuccess) return cstat(e);
    e = cudaStreamSynchronize(g->cap_stream);   // host vectors stay alive, but keep it simple
    if (e != cudaSuccess) return cstat(e);
  }
  e = cudaStreamSynchronize(g->cap_stream);
  if (e != cudaSuccess) return cstat(e);
  if (flags & MXG_GROUP_GRAPH) {
    e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cstat(e);
    const int st = enqueue_run(g, g->cap_stream, true, true);
    e = cudaStreamEndCapture(g->cap_stream, &g->graph);
    if (st) return st;
    if (e != cudaSuccess) return cstat(e);
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) return cstat(e);
  }
  return MXG_OK;
}

}  // namespace

extern "C" {

int mxg_group_create(mxg_handle h, int64_t count, const mxg_problem* probs, int method_s, int method_d, int flags,
                     mxg_group* out, int64_t* first_bad) {
  if (!h || !out || count < 0 || (count > 0 && !probs)) return MXG_EINVAL;
  if (count > (1 << 24)) return MXG_EINVAL;
  mxg_group_s* g = new (std::nothrow) mxg_group_s();
  if (!g) return MXG_ENOMEM;
  g->h = h;
  const int st = build_group(h, count, probs, method_s, method_d, flags, g, first_bad);
  if (st != MXG_OK) {
    if (g->cap_stream) cudaStreamSynchronize(g->cap_stream);
    free_group(g);
    return st;
  }
  *out = g;
  return MXG_OK;
}

int mxg_group_run(mxg_group g) {
  if (!g) return MXG_EINVAL;
  if (g->exec) return cstat(cudaGraphLaunch(g->exec, g->h->stream));
  return enqueue_run(g, g->h->stream, true, true);
}

int mxg_group_describe(mxg_group g, char* buf, size_t len) {
  if (!g || !buf || len == 0) return MXG_EINVAL;
  static const char* vnames[VAR_COUNT] = {"ffma_128", "ffma_64", "dfma_64", "dfma_32", "dmma_64", "ffma_32",
                                          "dfma_16"};
  static const char* pnames[NBUCKETS] = {"s", "d", "s", "h", "b"};
  std::string s = "{\"problems\": " + std::to_string(g->plans.size()) + ", \"graph\": " +
                  (g->exec ? "true" : "false") + ", \"arena_bytes\": " + std::to_string(g->arena_bytes) +
                  ", \"scale_only\": " + std::to_string(g->scale_list.size()) + ", \"buckets\": [";
  bool first = true;
  for (int bi = 0; bi < NBUCKETS; ++bi) {
    const Bucket& b = g->buckets[bi];
    if (b.members.empty()) continue;
    const char* kname = b.variant >= 0 ? vnames[b.variant] : "none";
    if (b.tc_split == SPLIT_BF16) kname = "tc_bf16x3";
    else if (b.tc_split == SPLIT_TF32) kname = "tc_tf32x3";
    else if (b.tc_split == SPLIT_F16_ONE) kname = "tc16_f16";
    else if (b.tc_split == SPLIT_BF16_ONE) kname = "tc16_bf16";
    char tmp[512];
    std::snprintf(tmp, sizeof(tmp),
                  "%s{\"precision\": \"%s\", \"problems\": %zu, \"kernel\": \"%s\", \"schedule\": \"%s\", "
                  "\"tiles\": %d, \"pack_tiles\": %lld, \"tuned_ms\": %.4f, \"from_cache\": %s, \"signature\": \"%s\"}",
                  first ? "" : ", ", pnames[bi], b.members.size(), kname,
                  (b.sched == SCHED_STATIC || b.tc_split != SPLIT_NONE) ? "static" : "dynamic",
                  b.ntiles, static_cast<long long>(b.tile_start.empty() ? 0 : b.tile_start.back()), b.tuned_ms,
                  b.from_cache ? "true" : "false", b.signature.c_str());
    s += tmp;
    first = false;
  }
  s += "]}";
  std::strncpy(buf, s.c_str(), len - 1);
  buf[len - 1] = '\0';
  return MXG_OK;
}

int mxg_group_destroy(mxg_group g) {
  if (!g) return MXG_EINVAL;
  cudaStreamSynchronize(g->h->stream);
  if (g->cap_stream) cudaStreamSynchronize(g->cap_stream);
  free_group(g);
  return MXG_OK;
}

int mxgemm_grouped(mxg_handle h, int64_t count, const mxg_problem* probs) {
  mxg_group g = nullptr;
  int st = mxg_group_create(h, count, probs, MXG_METHOD_AUTO, MXG_METHOD_AUTO, 0, &g, nullptr);
  if (st != MXG_OK) return st;
  st = mxg_group_run(g);
  const int st2 = mxg_group_destroy(g);
  return st != MXG_OK ? st : st2;
}

int mxg_tune_save(const char* path) {
  if (!path) return MXG_EINVAL;
  FILE* f = std::fopen(path, "w");
  if (!f) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : g_tune) std::fprintf(f, "%s %d %d %.6f\n", kv.first.c_str(), kv.second.variant, kv.second.sched, kv.second.ms);
  std::fclose(f);
  return MXG_OK;
}

int mxg_tune_load(const char* path) {
  if (!path) return MXG_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return MXG_EINVAL;
  char sig[160];
  int v = 0, s = 0;
  double ms = 0.0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (std::fscanf(f, "%159s %d %d %lf", sig, &v, &s, &ms) == 4) {
    if (v >= 0 && v < VAR_COUNT && (s == SCHED_DYNAMIC || s == SCHED_STATIC))
      g_tune[sig] = TuneRec{v, s, ms};
  }
  std::fclose(f);
  return MXG_OK;
}

}  // extern "C"
