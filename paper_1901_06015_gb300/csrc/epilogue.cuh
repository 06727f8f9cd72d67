// Fused epilogue of the contraction kernels: alpha, the cast to C's storage precision,
// beta*C in C's storage precision, the store (Sec. 5.1.3, Sec. 7.1 option 1 for both
// scalars: alpha in the computation precision, beta in C's storage precision, and
// alpha*AB cast to C's precision before it is accumulated).
#pragma once

#include "mxg_internal.h"
#include "../../include/mxgemm.h"

namespace mxg {

template <int CDT> struct CStore { using T = float; static constexpr bool cplx = false; };
template <> struct CStore<MXG_D> { using T = double; static constexpr bool cplx = false; };
template <> struct CStore<MXG_C> { using T = float; static constexpr bool cplx = true; };
template <> struct CStore<MXG_Z> { using T = double; static constexpr bool cplx = true; };

// Explicitly rounded products and sums (round-to-nearest-even). The compiler never
// fuses these into FMAs, so every rounding the paper's order prescribes happens, and
// the result does not depend on the kernel the epilogue is inlined into.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Update C(i, j) with the product value (pr, pi), both in the computation precision
// AccT. pi is ignored unless MODE pairs two real results into one complex value.
// Order of operations (Sec. 7.1): t = alpha*P rounded in AccT, cast to C's precision;
// beta*C formed in C's precision; their sum rounded in C's precision.
template <typename AccT, int CDT, int MODE>
__device__ __forceinline__ void epi_store(const EpiArgs& e, int64_t i, int64_t j, AccT pr, AccT pi) {
  using CT = typename CStore<CDT>::T;
  if (i >= e.m || j >= e.n) return;
  const AccT ar = static_cast<AccT>(e.ar);
  CT* c = static_cast<CT*>(e.C) + (i * e.rs + j * e.cs) * (CStore<CDT>::cplx ? 2 : 1);
  if constexpr (!CStore<CDT>::cplx) {
    // C real: alpha and beta projected onto the real line (Sec. 7.2).
    const CT t = static_cast<CT>(mul_rn(ar, pr));
    c[0] = e.beta_zero ? t : add_rn(mul_rn(static_cast<CT>(e.br), c[0]), t);
  } else {
    AccT tr, ti;
    const AccT ai_ = static_cast<AccT>(e.ai);
    if constexpr (MODE == OUT_RE_ONLY) {
      tr = mul_rn(ar, pr);     // case 1c: the product is real; with a real alpha it reaches Re(C) only
      ti = mul_rn(ai_, pr);    // (a complex alpha only under the literal reading)
    } else {
      const AccT ai = static_cast<AccT>(e.ai);
      tr = sub_rn(mul_rn(ar, pr), mul_rn(ai, pi));  // complex alpha honoured (case 3)
      ti = add_rn(mul_rn(ar, pi), mul_rn(ai, pr));  // ai == 0 otherwise
    }
    const CT tcr = static_cast<CT>(tr), tci = static_cast<CT>(ti);
    if (e.beta_zero) {
      c[0] = tcr;
      c[1] = (MODE == OUT_RE_ONLY && e.ai == 0.0) ? CT(0) : tci;
    } else {
      const CT br = static_cast<CT>(e.br), bi = static_cast<CT>(e.bi);
      const CT cr = c[0], ci = c[1];
      const CT bcr = sub_rn(mul_rn(br, cr), mul_rn(bi, ci));
      const CT bci = add_rn(mul_rn(br, ci), mul_rn(bi, cr));
      c[0] = add_rn(bcr, tcr);
      c[1] = (MODE == OUT_RE_ONLY && e.ai == 0.0) ? bci : add_rn(bci, tci);
    }
  }
}

}  // namespace mxg
