// Planner types: a validated call and the real gemm it reduces to.
#pragma once

#include <cstddef>
#include <cstdint>

#include "mxg_internal.h"

namespace mxg {

struct Call {
  int transa, transb;
  int64_t m, n, k;
  double alpha_re, alpha_im, beta_re, beta_im;
  const void* A; int dtA; int64_t rsA, csA;
  const void* B; int dtB; int64_t rsB, csB;
  void* C; int dtC; int64_t rsC, csC;
  int comp;
  int literal_alpha;   // Sec. 7.2's literal reading: complex alpha honoured in every case
  int split_k;         // 0 off, 1 automatic, >= 2 that many K slices (SIMT and DMMA methods)
  int sm_count;        // SMs of the device (0: assume 152) for the automatic split
  int cta_pairs;       // tensor-core methods: 0 automatic, 1 CTA pairs, 2 single CTAs
  int stream_k;        // CTA-pair kernel's stream-K tail: 0 off, 1 automatic, 2 always
};

enum PlanKind : int { PLAN_NOOP = 0, PLAN_SCALE = 1, PLAN_GEMM = 2 };

struct Plan {
  Call call{};            // as given
  Call work{};            // after the optional whole-op transpose
  int kind = PLAN_NOOP;
  int domain_case = 0;    // of the call as given (Fig. "mixeddom")
  int comp = 0;                     // resolved MXG_PREC_* (S, D, H or B)
  bool comp_double = false;
  int method = 0;
  bool swapped = false;
  double ar = 0, ai = 0, br = 0, bi = 0;
  bool beta_zero = false, alpha_zero = false;
  int pat_a = PAT_RE, pat_b = PAT_RE, mode = OUT_REAL;
  int conj_a = 0, conj_b = 0;
  int fold_a = 0, fold_b = 0;       // alpha folded into this operand's pack (literal alpha, C real)
  int real_products = 1;
  int64_t Mr = 0, Nr = 0, Kr = 0;   // real gemm
  int64_t Mp = 0, Np = 0, Kp = 0;   // padded to the kernel's tiles
  int split = SPLIT_NONE;           // hi/lo planes for the tensor-core methods
  bool pairs = false;               // tensor-core contraction on CTA pairs
  size_t plane_a = 0, plane_b = 0;  // bytes of one plane (split methods)
  int splits = 1;                   // split-K slices
  int64_t kslice = 0;               // k elements per slice
  size_t bytes_ws = 0;              // split-K partial sums
  size_t bytes_sk = 0;              // stream-K tail of the CTA-pair kernel (after the rest)
  int stream_k = 0;                 // its mode
  size_t bytes_a = 0, bytes_b = 0, workspace = 0;
};

int make_plan(const Call& c, int method, Plan* p);
EpiArgs plan_epilogue(const Plan& P);
int enqueue_plan(const Plan& P, void* ws, cudaStream_t s, cudaEvent_t ev_mid, int* dev_err = nullptr);

}  // namespace mxg
