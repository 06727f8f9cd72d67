// Host side of the library: argument validation, the planner that reduces a
// mixed-datatype gemm to one real gemm (Fig. "mixeddom", Secs. 4.1-4.2, 5.1, 7),
// workspace management, and the exported C ABI (include/mxgemm.h).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mxg_internal.h"
#include "context.h"
#include "plan.h"
#include "../../include/mxgemm.h"

namespace mxg {

thread_local int g_last_cuda_error = 0;

static int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MXG_OK;
  g_last_cuda_error = static_cast<int>(e);
  return e == cudaErrorMemoryAllocation ? MXG_ENOMEM : MXG_ECUDA;
}

static bool dt_ok(int dt) { return dt >= MXG_S && dt <= MXG_W; }
static bool trans_ok(int t) { return t >= MXG_NOTRANS && t <= MXG_CONJTRANS; }
static bool is_cplx(int dt) { return dt == MXG_C || dt == MXG_Z || dt == MXG_K || dt == MXG_W; }
// storage precision of a datatype as an MXG_PREC_* code
static int prec_of_dt(int dt) {
  switch (dt) {
    case MXG_D: case MXG_Z: return MXG_PREC_D;
    case MXG_H: case MXG_K: return MXG_PREC_H;
    case MXG_B: case MXG_W: return MXG_PREC_B;
    default: return MXG_PREC_S;
  }
}
static bool is_t(int t) { return t == MXG_TRANS || t == MXG_CONJTRANS; }
static bool is_conj(int t) { return t == MXG_CONJ || t == MXG_CONJTRANS; }
static int flip_t(int t) {  // op(X)^T expressed as a trans value on the same storage
  switch (t) {
    case MXG_NOTRANS: return MXG_TRANS;
    case MXG_TRANS: return MXG_NOTRANS;
    case MXG_CONJ: return MXG_CONJTRANS;
    default: return MXG_CONJ;
  }
}
// Round (RN-even) to an MXG_PREC_* precision, with CUDA's host conversions for 16 bits.
static double rnd_p(double x, int prec) {
  switch (prec) {
    case MXG_PREC_D: return x;
    case MXG_PREC_H: return static_cast<double>(__half2float(__double2half(x)));
    case MXG_PREC_B: return static_cast<double>(__bfloat162float(__double2bfloat16(x)));
    default: return static_cast<double>(static_cast<float>(x));
  }
}
static int64_t round_up(int64_t x, int64_t t) { return (x + t - 1) / t * t; }
static size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Strides of a stored rows x cols matrix must be >= 1 on every dimension longer than 1
// (a matrix with no elements is never read, so its strides do not matter).
static bool strides_ok(int64_t rows, int64_t cols, int64_t rs, int64_t cs) {
  if (rows == 0 || cols == 0) return true;
  if (rows > 1 && rs < 1) return false;
  if (cols > 1 && cs < 1) return false;
  if (rs < 0 || cs < 0) return false;
  return true;
}

// C must not overlap itself: with the smaller stride's dimension spanning less than
// the larger stride (the usual sufficient condition for a strided 2-D view).
static bool no_self_overlap(int64_t m, int64_t n, int64_t rs, int64_t cs) {
  if (m == 0 || n == 0) return true;
  if (m <= 1 && n <= 1) return true;
  if (m <= 1) return cs >= 1;
  if (n <= 1) return rs >= 1;
  int64_t s1 = rs, e1 = m, s2 = cs;
  if (rs > cs) { s1 = cs; e1 = n; s2 = rs; }
  return s1 >= 1 && s1 * (e1 - 1) < s2;
}

static size_t esz_of(const Plan& P) { return P.comp_double ? 8 : 4; }

int make_plan(const Call& c, int method, Plan* p) {
  if (!trans_ok(c.transa) || !trans_ok(c.transb)) return MXG_EINVAL;
  if (!dt_ok(c.dtA) || !dt_ok(c.dtB) || !dt_ok(c.dtC)) return MXG_EINVAL;
  if (c.comp < MXG_PREC_S || c.comp > MXG_PREC_B) return MXG_EINVAL;
  if (method < MXG_METHOD_AUTO || method > MXG_METHOD_TC16) return MXG_EINVAL;
  if (c.m < 0 || c.n < 0 || c.k < 0) return MXG_EINVAL;
  const int64_t a_rows = is_t(c.transa) ? c.k : c.m, a_cols = is_t(c.transa) ? c.m : c.k;
  const int64_t b_rows = is_t(c.transb) ? c.n : c.k, b_cols = is_t(c.transb) ? c.k : c.n;
  if (!strides_ok(a_rows, a_cols, c.rsA, c.csA)) return MXG_EINVAL;
  if (!strides_ok(b_rows, b_cols, c.rsB, c.csB)) return MXG_EINVAL;
  if (!strides_ok(c.m, c.n, c.rsC, c.csC)) return MXG_EINVAL;
  if (!no_self_overlap(c.m, c.n, c.rsC, c.csC)) return MXG_EINVAL;

  Plan& P = *p;
  P = Plan();
  P.call = c;
  P.domain_case = (is_cplx(c.dtC) << 2) | (is_cplx(c.dtA) << 1) | (is_cplx(c.dtB) ? 1 : 0);
  // Sec. 7.2: non-zero Im(alpha) is an error outside cases 0 and 3 (unless the caller
  // asked for the literal reading, which takes every operand's domain at face value).
  if (!c.literal_alpha && c.alpha_im != 0.0 && P.domain_case != MXG_CASE_0 && P.domain_case != MXG_CASE_3)
    return MXG_ECOMPLEX_ALPHA;
  // Sec. 5.1.1: the computation precision defaults to C's storage precision.
  P.comp = (c.comp == MXG_PREC_OF_C) ? prec_of_dt(c.dtC) : c.comp;
  P.comp_double = (P.comp == MXG_PREC_D);
  const bool comp16 = (P.comp == MXG_PREC_H || P.comp == MXG_PREC_B);
  // AUTO: the faster plain form of each precision on GB300 (measured: DFMA 1.25 vs
  // DMMA 1.10 TF/s, both on the FP64 pipe); the 16-bit precisions run on the tensor
  // cores.
  if (method == MXG_METHOD_AUTO)
    method = comp16 ? MXG_METHOD_TC16 : (P.comp_double ? MXG_METHOD_DFMA : MXG_METHOD_FFMA);
  const bool m_double = (method == MXG_METHOD_DMMA || method == MXG_METHOD_DFMA);
  const bool m_16 = (method == MXG_METHOD_TC16);
  if (m_double != P.comp_double || m_16 != comp16) return MXG_EINVAL;
  P.method = method;

  // Sec. 7.1: alpha in the computation precision, beta in C's storage precision.
  P.ar = rnd_p(c.alpha_re, P.comp);
  P.ai = (P.domain_case == MXG_CASE_3 || (c.literal_alpha && P.domain_case != MXG_CASE_0))
             ? rnd_p(c.alpha_im, P.comp) : 0.0;                                 // case 0 projects
  P.br = rnd_p(c.beta_re, prec_of_dt(c.dtC));
  P.bi = is_cplx(c.dtC) ? rnd_p(c.beta_im, prec_of_dt(c.dtC)) : 0.0;            // real C projects
  P.beta_zero = (P.br == 0.0 && P.bi == 0.0);
  P.alpha_zero = (P.ar == 0.0 && P.ai == 0.0);
  P.real_products = 1;
  if (c.m == 0 || c.n == 0) { P.kind = PLAN_NOOP; return MXG_OK; }
  if (c.k == 0 || P.alpha_zero) { P.kind = PLAN_SCALE; return MXG_OK; }
  // The split products' error floor (3 u_p^2 per product, independent of k) must fit
  // the accuracy 4 k u_s with the accumulation and the epilogue (include/mxgemm.h).
  if ((method == MXG_METHOD_BF16X3 && c.k < MXG_SPLIT_MIN_K_BF16X3) ||
      (method == MXG_METHOD_TF32X3 && c.k < MXG_SPLIT_MIN_K_TF32X3))
    return MXG_EACCURACY;
  P.kind = PLAN_GEMM;

  // Sec. 2.2.5: compute C^T := op(B)^T op(A)^T when C is row-stored, so the epilogue
  // writes along C's unit stride. The domain case follows the operands (2ac <-> 2bc,
  // 1a <-> 1b), as in the paper's logical transposition of case 2ac.
  Call w = c;
  P.swapped = (c.n > 1 && c.m > 1 && c.csC == 1 && c.rsC != 1) || (c.m == 1 && c.n > 1 && c.csC == 1);
  if (P.swapped) {
    w.m = c.n; w.n = c.m;
    w.A = c.B; w.dtA = c.dtB; w.rsA = c.rsB; w.csA = c.csB; w.transa = flip_t(c.transb);
    w.B = c.A; w.dtB = c.dtA; w.rsB = c.rsA; w.csB = c.csA; w.transb = flip_t(c.transa);
    w.rsC = c.csC; w.csC = c.rsC;
  }
  P.work = w;
  const int wcase = (is_cplx(w.dtC) << 2) | (is_cplx(w.dtA) << 1) | (is_cplx(w.dtB) ? 1 : 0);

  int pa = PAT_RE, pb = PAT_RE, mode = OUT_REAL, conj_b_extra = 0;
  switch (wcase) {
    case MXG_CASE_0: case MXG_CASE_1B: case MXG_CASE_1A:
      break;                                       // real gemm on Re of complex operands
    case MXG_CASE_2AB:                             // Re(AB): A in 1r, B in 1r conjugated
      pa = PAT_SPLIT_K; pb = PAT_SPLIT_K; conj_b_extra = 1; P.real_products = 2; break;
    case MXG_CASE_1C:
      mode = OUT_RE_ONLY; break;
    case MXG_CASE_2BC:                             // B viewed as real k x 2n, C as m x 2n
      pb = PAT_SPLIT_MN; mode = OUT_COLPAIR; P.real_products = 2; break;
    case MXG_CASE_2AC:                             // A viewed as real 2m x k, C as 2m x n
      pa = PAT_SPLIT_MN; mode = OUT_ROWPAIR; P.real_products = 2; break;
    case MXG_CASE_3:                               // 1m, Eq. (1): A in 1e, B in 1r
      pa = PAT_ONE_E; pb = PAT_SPLIT_K; mode = OUT_ROWPAIR; P.real_products = 4; break;
  }
  P.pat_a = pa; P.pat_b = pb; P.mode = mode;
  // Literal complex alpha with C real (cases 1a, 1b, 2ab): Re(alpha A B) = Re((alpha A) B),
  // so alpha is folded into the pack of a complex operand and the epilogue uses 1.
  if (c.literal_alpha && P.ai != 0.0 && !is_cplx(w.dtC)) {
    if (is_cplx(w.dtA)) P.fold_a = 1; else P.fold_b = 1;
  }
  P.conj_a = is_conj(w.transa) ? 1 : 0;
  P.conj_b = (is_conj(w.transb) ? 1 : 0) ^ conj_b_extra;
  P.Mr = w.m * pat_fm(pa);
  P.Nr = w.n * pat_fm(pb);
  P.Kr = w.k * pat_fk(pa);
  const TileCfg t = tile_cfg(method);
  P.Mp = round_up(P.Mr, t.tm);
  P.Np = round_up(P.Nr, t.tn);
  P.Kp = round_up(P.Kr, t.tk);
  if (method == MXG_METHOD_TF32X3 || method == MXG_METHOD_BF16X3 || method == MXG_METHOD_TC16) {
    // K-major planes for TMA: hi and lo for the split forms, one plane for TC16
    P.split = (method == MXG_METHOD_BF16X3) ? SPLIT_BF16
              : (method == MXG_METHOD_TF32X3) ? SPLIT_TF32
              : (P.comp == MXG_PREC_H) ? SPLIT_F16_ONE : SPLIT_BF16_ONE;
    const size_t esz = (P.split == SPLIT_TF32) ? 4 : 2;
    const int planes = (method == MXG_METHOD_TC16) ? 1 : 2;
    P.plane_a = align256(static_cast<size_t>(P.Kp) * P.Mp * esz);
    P.plane_b = align256(static_cast<size_t>(P.Kp) * P.Np * esz);
    P.bytes_a = planes * P.plane_a;
    P.bytes_b = planes * P.plane_b;
    // CTA pairs by default: half the operand rows per CTA per flop, 128-byte k rows
    P.pairs = (c.cta_pairs != 2);
  } else {
    const size_t esz = P.comp_double ? 8 : 4;
    P.bytes_a = align256(static_cast<size_t>(P.Kp) * P.Mp * esz);
    P.bytes_b = align256(static_cast<size_t>(P.Kp) * P.Np * esz);
  }
  // Split-K (Secs. 6.2-6.4: a workspace in the computation precision), only on request.
  if (c.split_k && P.split == SPLIT_NONE) {
    const int64_t tiles = (P.Mp / t.tm) * (P.Np / t.tn);
    const int64_t ktiles = P.Kp / t.tk;
    const int64_t min_ktiles = std::max<int64_t>(1, 512 / t.tk);   // at least 512 k per slice
    int64_t S = c.split_k;
    if (c.split_k == 1) {
      const int64_t sms = c.sm_count > 0 ? c.sm_count : 152;
      S = tiles >= sms ? 1 : (2 * sms + tiles - 1) / tiles;
      S = std::min<int64_t>(S, std::max<int64_t>(1, ktiles / min_ktiles));
    }
    S = std::max<int64_t>(1, std::min<int64_t>({S, ktiles, 65535}));
    if (S > 1) {
      const int64_t per = (ktiles + S - 1) / S;       // k-tiles per slice
      P.kslice = per * t.tk;
      P.splits = static_cast<int>((P.Kp + P.kslice - 1) / P.kslice);
      P.bytes_ws = align256(static_cast<size_t>(P.splits) * P.Mp * P.Np * esz_of(P));
    }
  }
  // Stream-K tail of the pair kernel: partial accumulators and tile counters.
  if (P.pairs && c.stream_k) {
    P.stream_k = c.stream_k;
    P.bytes_sk = tc_pair_stream_k_workspace(P.split, P.Mp, P.Np, P.Kp, c.sm_count, c.stream_k);
  }
  P.workspace = P.bytes_a + P.bytes_b + P.bytes_ws + P.bytes_sk;
  return MXG_OK;
}

// Operand (mn, p) strides of the logical operand of the real gemm. For A: (i, p) of
// op(A); for B: (j, p) of op(B), i.e. op(B)(p, j).
static void operand_strides_a(const Call& w, int64_t* smn, int64_t* sk) {
  if (is_t(w.transa)) { *smn = w.csA; *sk = w.rsA; } else { *smn = w.rsA; *sk = w.csA; }
}
static void operand_strides_b(const Call& w, int64_t* smn, int64_t* sk) {
  if (is_t(w.transb)) { *smn = w.rsB; *sk = w.csB; } else { *smn = w.csB; *sk = w.rsB; }
}

EpiArgs plan_epilogue(const Plan& P) {
  EpiArgs e{};
  const Call& w = (P.kind == PLAN_GEMM) ? P.work : P.call;
  e.C = w.C; e.rs = w.rsC; e.cs = w.csC; e.m = w.m; e.n = w.n;
  e.ar = P.ar; e.ai = P.ai; e.br = P.br; e.bi = P.bi; e.beta_zero = P.beta_zero;
  if (P.fold_a || P.fold_b) { e.ar = 1.0; e.ai = 0.0; }   // alpha already applied by the pack
  return e;
}

int enqueue_plan(const Plan& P, void* ws, cudaStream_t s, cudaEvent_t ev_mid, int* dev_err) {
  if (P.kind == PLAN_NOOP) return MXG_OK;
  if (P.kind == PLAN_SCALE) {
    EpiArgs e = plan_epilogue(P);
    e.ar = 0.0; e.ai = 0.0;
    e.dbg = dev_err;
    return cuda_status(launch_scale_c(e, P.call.dtC, s));
  }
  const Call& w = P.work;
  char* base = static_cast<char*>(ws);
  PackArgs pa{};
  pa.src = w.A; pa.src_dt = w.dtA;
  operand_strides_a(w, &pa.smn, &pa.sk);
  pa.MN = w.m; pa.K = w.k; pa.pattern = P.pat_a; pa.conj = P.conj_a;
  pa.dst = base; pa.dst_lo = nullptr; pa.ld = P.Mp; pa.MNp = P.Mp; pa.Kp = P.Kp;
  pa.layout = LAYOUT_MN_MAJOR; pa.split = SPLIT_NONE;
  pa.fold = P.fold_a; pa.fold_re = P.ar; pa.fold_im = P.ai;
  pa.dbg = dev_err;
  if (P.split != SPLIT_NONE) {
    pa.dst_lo = (P.method == MXG_METHOD_TC16) ? nullptr : base + P.plane_a;
    pa.ld = P.Kp; pa.layout = LAYOUT_K_MAJOR; pa.split = P.split;
  }
  int st = cuda_status(launch_pack(pa, P.comp_double, s));
  if (st) return st;
  PackArgs pb{};
  pb.src = w.B; pb.src_dt = w.dtB;
  operand_strides_b(w, &pb.smn, &pb.sk);
  pb.MN = w.n; pb.K = w.k; pb.pattern = P.pat_b; pb.conj = P.conj_b;
  pb.dst = base + P.bytes_a; pb.dst_lo = nullptr; pb.ld = P.Np; pb.MNp = P.Np; pb.Kp = P.Kp;
  pb.layout = LAYOUT_MN_MAJOR; pb.split = SPLIT_NONE;
  pb.fold = P.fold_b; pb.fold_re = P.ar; pb.fold_im = P.ai;
  pb.dbg = dev_err;
  if (P.split != SPLIT_NONE) {
    pb.dst_lo = (P.method == MXG_METHOD_TC16) ? nullptr : base + P.bytes_a + P.plane_b;
    pb.ld = P.Kp; pb.layout = LAYOUT_K_MAJOR; pb.split = P.split;
  }
  st = cuda_status(launch_pack(pb, P.comp_double, s));
  if (st) return st;
  if (ev_mid) cudaEventRecord(ev_mid, s);
  EpiArgs ep = plan_epilogue(P);
  ep.dbg = dev_err;
  if (P.split != SPLIT_NONE) {
    const bool one = (P.method == MXG_METHOD_TC16);
    const void* planes[4] = {base, one ? base : base + P.plane_a, base + P.bytes_a,
                             one ? base + P.bytes_a : base + P.bytes_a + P.plane_b};
    const cudaError_t e =
        P.pairs ? launch_gemm_tc_pair(P.split, w.dtC, P.mode, planes, P.Mp, P.Np, P.Kp, ep, dev_err,
                                      P.bytes_sk ? base + P.bytes_a + P.bytes_b + P.bytes_ws : nullptr,
                                      P.bytes_sk, P.stream_k, s)
                : launch_gemm_tc(P.method, P.split, w.dtC, P.mode, planes, P.Mp, P.Np, P.Kp, ep, dev_err,
                                 s);
    return e == cudaErrorNotSupported ? MXG_ENOTSUP : cuda_status(e);
  }
  GemmArgs g;
  g.A = base; g.B = base + P.bytes_a; g.lda = P.Mp; g.ldb = P.Np; g.Kp = P.Kp;
  g.Mp = P.Mp; g.Np = P.Np; g.e = ep;
  if (P.splits > 1)
    return cuda_status(launch_gemm_splitk(P.method, w.dtC, P.mode, g, P.splits, P.kslice,
                                          base + P.bytes_a + P.bytes_b, s));
  return cuda_status(launch_gemm_simt(P.method, w.dtC, P.mode, g, s));
}

}  // namespace mxg

using namespace mxg;

static int ensure_workspace(mxg_context* h, size_t need, void** out) {
  *out = h->ws;
  if (need == 0) return MXG_OK;
  if (need <= h->ws_bytes) return MXG_OK;
  if (!h->ws_owned) return MXG_ENOMEM;
  // The old buffer may still be in use by enqueued work: wait for the stream first.
  if (h->ws) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  size_t sz = std::max(need, static_cast<size_t>(1) << 20);
  sz = align256(sz + sz / 8);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  h->ws = p;
  h->ws_bytes = sz;
  *out = p;
  return MXG_OK;
}

static std::mutex g_default_mu;
static std::vector<mxg_context*> g_default;  // one per device, never freed

static int default_handle(mxg_context** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  std::lock_guard<std::mutex> lk(g_default_mu);
  if (static_cast<int>(g_default.size()) <= dev) g_default.resize(dev + 1, nullptr);
  if (!g_default[dev]) {
    mxg_context* h = nullptr;
    int st = mxg_create(&h);
    if (st) return st;
    g_default[dev] = h;
  }
  *out = g_default[dev];
  return MXG_OK;
}

extern "C" {

int mxg_version(void) { return 10000; }

int mxg_debug_bounds(void) {
#ifdef MXG_DEBUG_BOUNDS
  return 1;
#else
  return 0;
#endif
}

int mxg_last_cuda_error(void) { return g_last_cuda_error; }

const char* mxg_strerror(int status) {
  switch (status) {
    case MXG_OK: return "success";
    case MXG_EINVAL: return "invalid argument";
    case MXG_ECOMPLEX_ALPHA: return "imaginary alpha is not supported in mixed-domain cases 1a, 1b, 1c, 2ab, 2ac, 2bc";
    case MXG_ENOMEM: return "device workspace allocation failed or caller workspace too small";
    case MXG_ECUDA: return "CUDA runtime error";
    case MXG_ETIMEOUT: return "device-side wait ran out of its iteration limit";
    case MXG_ENOTSUP: return "method not supported on this device";
    case MXG_ESCRATCH: return "problem needs more scratch than the fixed no-allocation buffer (MXG_NOALLOC_SCRATCH_BYTES) holds";
    case MXG_EACCURACY: return "split-precision method cannot meet the accuracy 4*k*u_s at this k (BF16X3 needs k >= 320, TF32X3 k >= 32)";
  }
  return "unknown status";
}

int mxg_plan(int method, int transa, int transb, int64_t m, int64_t n, int64_t k,
             double alpha_re, double alpha_im, int dtA, int64_t rsA, int64_t csA,
             int dtB, int64_t rsB, int64_t csB, int dtC, int64_t rsC, int64_t csC,
             int comp_prec, mxg_plan_info* info) {
  Call c{};
  c.transa = transa; c.transb = transb; c.m = m; c.n = n; c.k = k;
  c.alpha_re = alpha_re; c.alpha_im = alpha_im; c.beta_re = 1.0; c.beta_im = 0.0;
  c.dtA = dtA; c.rsA = rsA; c.csA = csA; c.dtB = dtB; c.rsB = rsB; c.csB = csB;
  c.dtC = dtC; c.rsC = rsC; c.csC = csC; c.comp = comp_prec;
  c.stream_k = 1;   // a handle's default
  Plan P;
  const int st = make_plan(c, method, &P);
  if (st != MXG_OK) return st;
  if (info) {
    info->domain_case = P.domain_case;
    info->comp_prec = P.comp;
    info->method = P.method;
    info->whole_op_transposed = P.swapped ? 1 : 0;
    info->Mr = P.Mr; info->Nr = P.Nr; info->Kr = P.Kr;
    info->real_products = P.real_products;
    info->flops = 2.0 * static_cast<double>(m) * static_cast<double>(n) * static_cast<double>(k) * P.real_products;
    info->workspace_bytes = P.workspace;
    info->k_splits = P.splits;
  }
  return MXG_OK;
}

int mxg_create(mxg_handle* out) {
  if (!out) return MXG_EINVAL;
  mxg_context* h = new (std::nothrow) mxg_context();
  if (!h) return MXG_ENOMEM;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->dev_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->dev_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    if (h->dev_err) cudaFree(h->dev_err);
    delete h;
    return cuda_status(e);
  }
  *out = h;
  return MXG_OK;
}

int mxg_destroy(mxg_handle h) {
  if (!h) return MXG_EINVAL;
  cudaStreamSynchronize(h->stream);
  if (h->ws && h->ws_owned) cudaFree(h->ws);
  if (h->dev_err) cudaFree(h->dev_err);
  recycle_events(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return MXG_OK;
}

int mxg_set_split_k(mxg_handle h, int mode) {
  if (!h || mode < 0 || mode > 65535) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  h->split_k = mode;
  return MXG_OK;
}

int mxg_set_cta_pairs(mxg_handle h, int mode) {
  if (!h || mode < 0 || mode > 2) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  h->cta_pairs = mode;
  return MXG_OK;
}

int mxg_set_stream_k(mxg_handle h, int mode) {
  if (!h || mode < 0 || mode > 2) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  h->stream_k = mode;
  return MXG_OK;
}

int mxg_set_literal_alpha(mxg_handle h, int on) {
  if (!h) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  h->literal_alpha = (on != 0);
  return MXG_OK;
}

int mxg_set_stream(mxg_handle h, void* stream) {
  if (!h) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  h->stream = static_cast<cudaStream_t>(stream);
  return MXG_OK;
}

int mxg_set_workspace(mxg_handle h, void* ptr, size_t bytes) {
  if (!h) return MXG_EINVAL;
  if (ptr && (reinterpret_cast<uintptr_t>(ptr) & 255)) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  if (h->ws && h->ws_owned) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
  }
  if (ptr) {
    h->ws = ptr; h->ws_bytes = bytes; h->ws_owned = false;
  } else {
    h->ws = nullptr; h->ws_bytes = 0; h->ws_owned = true;
  }
  return MXG_OK;
}

int mxg_set_phase_timing(mxg_handle h, int on) {
  if (!h) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  if (!on) {
    cudaStreamSynchronize(h->stream);
    recycle_events(h);
  }
  h->timing = (on != 0);
  return MXG_OK;
}

int mxg_phase_times(mxg_handle h, double* pack_ms, double* contraction_ms, int64_t* launches) {
  if (!h || !pack_ms || !contraction_ms || !launches) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  double pk = 0.0, ct = 0.0;
  for (size_t i = 0; i + 2 < h->ev_rec.size(); i += 3) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, h->ev_rec[i], h->ev_rec[i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&b, h->ev_rec[i + 1], h->ev_rec[i + 2]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    pk += a;
    ct += b;
  }
  *pack_ms = pk;
  *contraction_ms = ct;
  *launches = static_cast<int64_t>(h->ev_rec.size() / 3);
  recycle_events(h);
  return MXG_OK;
}

int mxg_selftest_wait_timeout(mxg_handle h, double seconds) {
  if (!h || !(seconds > 0.0) || seconds > 10.0) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaError_t e = launch_wait_timeout_probe(h->dev_err, seconds, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int v = 0;
  e = cudaMemcpyAsync(&v, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  return v ? MXG_ETIMEOUT : MXG_OK;
}

int mxg_check_device_error(mxg_handle h, int* flag) {
  if (!h || !flag) return MXG_EINVAL;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && v) e = cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  *flag = v;
  return MXG_OK;
}

int mxgemm_ex(mxg_handle h, int method, int transa, int transb, int64_t m, int64_t n, int64_t k,
              double alpha_re, double alpha_im,
              const void* A, int dtA, int64_t rsA, int64_t csA,
              const void* B, int dtB, int64_t rsB, int64_t csB,
              double beta_re, double beta_im,
              void* C, int dtC, int64_t rsC, int64_t csC, int comp_prec) {
  if (!h) return MXG_EINVAL;
  Call c{};
  c.transa = transa; c.transb = transb; c.m = m; c.n = n; c.k = k;
  c.alpha_re = alpha_re; c.alpha_im = alpha_im; c.beta_re = beta_re; c.beta_im = beta_im;
  c.A = A; c.dtA = dtA; c.rsA = rsA; c.csA = csA;
  c.B = B; c.dtB = dtB; c.rsB = rsB; c.csB = csB;
  c.C = C; c.dtC = dtC; c.rsC = rsC; c.csC = csC; c.comp = comp_prec;
  c.literal_alpha = h->literal_alpha ? 1 : 0;
  c.split_k = h->split_k;
  c.sm_count = h->sm_count;
  c.cta_pairs = h->cta_pairs;
  c.stream_k = h->stream_k;
  Plan P;
  int st = make_plan(c, method, &P);
  if (st != MXG_OK) return st;
  if (P.kind == PLAN_NOOP) return MXG_OK;
  if (!C) return MXG_EINVAL;
  if (P.kind == PLAN_GEMM && (!A || !B)) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  // a caller workspace that holds everything but the stream-K tail runs without the tail
  if (!h->ws_owned && P.bytes_sk && P.workspace > h->ws_bytes && P.workspace - P.bytes_sk <= h->ws_bytes) {
    P.workspace -= P.bytes_sk;
    P.bytes_sk = 0;
  }
  void* ws = nullptr;
  st = ensure_workspace(h, P.kind == PLAN_GEMM ? P.workspace : 0, &ws);
  if (st != MXG_OK) return st;
  if (h->timing && P.kind == PLAN_GEMM) {
    cudaEvent_t e0 = take_event(h), e1 = take_event(h), e2 = take_event(h);
    if (e0 && e1 && e2) {
      cudaEventRecord(e0, h->stream);
      st = enqueue_plan(P, ws, h->stream, e1, h->dev_err);
      cudaEventRecord(e2, h->stream);
      h->ev_rec.push_back(e0); h->ev_rec.push_back(e1); h->ev_rec.push_back(e2);
      return st;
    }
    for (cudaEvent_t e : {e0, e1, e2}) if (e) h->ev_pool.push_back(e);
  }
  return enqueue_plan(P, ws, h->stream, nullptr, h->dev_err);
}

int mxgemm(int transa, int transb, int64_t m, int64_t n, int64_t k,
           double alpha_re, double alpha_im,
           const void* A, int dtA, int64_t rsA, int64_t csA,
           const void* B, int dtB, int64_t rsB, int64_t csB,
           double beta_re, double beta_im,
           void* C, int dtC, int64_t rsC, int64_t csC, int comp_prec) {
  // Validate before touching the device, so argument errors never depend on CUDA.
  Call c{};
  c.transa = transa; c.transb = transb; c.m = m; c.n = n; c.k = k;
  c.alpha_re = alpha_re; c.alpha_im = alpha_im; c.beta_re = beta_re; c.beta_im = beta_im;
  c.dtA = dtA; c.rsA = rsA; c.csA = csA; c.dtB = dtB; c.rsB = rsB; c.csB = csB;
  c.dtC = dtC; c.rsC = rsC; c.csC = csC; c.comp = comp_prec;
  Plan P;
  int st = make_plan(c, MXG_METHOD_AUTO, &P);
  if (st != MXG_OK) return st;
  if (P.kind == PLAN_NOOP) return MXG_OK;
  mxg_context* h = nullptr;
  st = default_handle(&h);
  if (st != MXG_OK) return st;
  return mxgemm_ex(h, MXG_METHOD_AUTO, transa, transb, m, n, k, alpha_re, alpha_im,
                   A, dtA, rsA, csA, B, dtB, rsB, csB, beta_re, beta_im, C, dtC, rsC, csC, comp_prec);
}

}  // extern "C"
