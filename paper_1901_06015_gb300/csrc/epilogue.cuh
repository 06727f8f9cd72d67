// Fused epilogue of the contraction kernels: alpha, the cast to C's storage precision,
// beta*C in C's storage precision, the store (Sec. 5.1.3, Sec. 7.1 option 1 for both
// scalars: alpha in the computation precision, beta in C's storage precision, and
// alpha*AB cast to C's precision before it is accumulated).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "mxg_internal.h"
#include "../../include/mxgemm.h"

namespace mxg {

template <int CDT> struct CStore { using T = float; static constexpr bool cplx = false; };
template <> struct CStore<MXG_D> { using T = double; static constexpr bool cplx = false; };
template <> struct CStore<MXG_C> { using T = float; static constexpr bool cplx = true; };
template <> struct CStore<MXG_Z> { using T = double; static constexpr bool cplx = true; };
template <> struct CStore<MXG_H> { using T = __half; static constexpr bool cplx = false; };
template <> struct CStore<MXG_K> { using T = __half; static constexpr bool cplx = true; };
template <> struct CStore<MXG_B> { using T = __nv_bfloat16; static constexpr bool cplx = false; };
template <> struct CStore<MXG_W> { using T = __nv_bfloat16; static constexpr bool cplx = true; };

template <int V> using IC = std::integral_constant<int, V>;

// Call f(IC<C datatype>, IC<output mode>) for the 16 valid pairs: a real C takes
// OUT_REAL, a complex C one of OUT_RE_ONLY / OUT_ROWPAIR / OUT_COLPAIR. Returns false
// for any other pair.
template <class F>
__host__ __device__ __forceinline__ bool with_c_mode(int cdt, int mode, F&& f) {
  switch (cdt * 4 + mode) {
#define MXG_CM(C, M) \
    case C * 4 + M: f(IC<C>{}, IC<M>{}); return true;
    MXG_CM(MXG_S, OUT_REAL) MXG_CM(MXG_D, OUT_REAL) MXG_CM(MXG_H, OUT_REAL) MXG_CM(MXG_B, OUT_REAL)
    MXG_CM(MXG_C, OUT_RE_ONLY) MXG_CM(MXG_C, OUT_ROWPAIR) MXG_CM(MXG_C, OUT_COLPAIR)
    MXG_CM(MXG_Z, OUT_RE_ONLY) MXG_CM(MXG_Z, OUT_ROWPAIR) MXG_CM(MXG_Z, OUT_COLPAIR)
    MXG_CM(MXG_K, OUT_RE_ONLY) MXG_CM(MXG_K, OUT_ROWPAIR) MXG_CM(MXG_K, OUT_COLPAIR)
    MXG_CM(MXG_W, OUT_RE_ONLY) MXG_CM(MXG_W, OUT_ROWPAIR) MXG_CM(MXG_W, OUT_COLPAIR)
#undef MXG_CM
    default: return false;
  }
}

// Explicitly rounded products and sums (round-to-nearest-even). The compiler never
// fuses these into FMAs, so every rounding the paper's order prescribes happens, and
// the result does not depend on the kernel the epilogue is inlined into.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ __half mul_rn(__half a, __half b) { return __hmul_rn(a, b); }
__device__ __forceinline__ __half add_rn(__half a, __half b) { return __hadd_rn(a, b); }
__device__ __forceinline__ __half sub_rn(__half a, __half b) { return __hsub_rn(a, b); }
__device__ __forceinline__ __nv_bfloat16 mul_rn(__nv_bfloat16 a, __nv_bfloat16 b) { return __hmul_rn(a, b); }
__device__ __forceinline__ __nv_bfloat16 add_rn(__nv_bfloat16 a, __nv_bfloat16 b) { return __hadd_rn(a, b); }
__device__ __forceinline__ __nv_bfloat16 sub_rn(__nv_bfloat16 a, __nv_bfloat16 b) { return __hsub_rn(a, b); }

// Conversion (RN-even) to C's storage type.
template <typename CT> __device__ __forceinline__ CT to_ct(float x);
template <typename CT> __device__ __forceinline__ CT to_ct(double x);
template <> __device__ __forceinline__ float to_ct<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_ct<float>(double x) { return static_cast<float>(x); }
template <> __device__ __forceinline__ double to_ct<double>(float x) { return x; }
template <> __device__ __forceinline__ double to_ct<double>(double x) { return x; }
template <> __device__ __forceinline__ __half to_ct<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __half to_ct<__half>(double x) { return __double2half(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_ct<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_ct<__nv_bfloat16>(double x) { return __double2bfloat16(x); }


// Debug builds: does the element at c lie inside the storage that (m, n, rs, cs)
// describe for C (first element to the last one, both parts of a complex element)?
template <int CDT>
__device__ __forceinline__ bool c_in_extent(const EpiArgs& e, const void* c) {
  using CT = typename CStore<CDT>::T;
  const int64_t w = CStore<CDT>::cplx ? 2 : 1;
  const int64_t off = static_cast<const CT*>(c) - static_cast<const CT*>(e.C);
  const int64_t last = ((e.m - 1) * e.rs + (e.n - 1) * e.cs) * w + (w - 1);
  return off >= 0 && off + (w - 1) <= last;
}

// C's value at (i, j) before the update, in C's storage type (im = 0 for a real C);
// zero, and not read, where beta == 0 or (i, j) lies outside C. The kernels read a
// thread's group of C elements with epi_load first and then update them with
// epi_update, so that the group's loads are in flight together rather than one
// load-update-store after another.
template <int CDT> struct COld { typename CStore<CDT>::T re, im; };

template <int CDT>
__device__ __forceinline__ COld<CDT> epi_load(const EpiArgs& e, int64_t i, int64_t j) {
  using CT = typename CStore<CDT>::T;
  COld<CDT> o{to_ct<CT>(0.0f), to_ct<CT>(0.0f)};
  if (e.beta_zero || i >= e.m || j >= e.n) return o;
  const CT* c = static_cast<const CT*>(e.C) + (i * e.rs + j * e.cs) * (CStore<CDT>::cplx ? 2 : 1);
  if (!MXG_DBG_OK(c_in_extent<CDT>(e, c), e.dbg)) return o;
  o.re = c[0];
  if constexpr (CStore<CDT>::cplx) o.im = c[1];
  return o;
}

// alpha in the computation precision and beta in C's storage precision, converted
// from the double-precision arguments once per tile: a conversion from double runs on
// the FP64 pipe, which on this chip is slow enough to stall an epilogue that converted
// per element.
template <typename AccT, int CDT>
struct EpiScalars {
  using CT = typename CStore<CDT>::T;
  AccT ar, ai;
  CT br, bi;
  bool ai_zero;
};

template <typename AccT, int CDT>
__device__ __forceinline__ EpiScalars<AccT, CDT> epi_scalars(const EpiArgs& e) {
  using CT = typename CStore<CDT>::T;
  return {static_cast<AccT>(e.ar), static_cast<AccT>(e.ai), to_ct<CT>(e.br), to_ct<CT>(e.bi), e.ai == 0.0};
}

// The new value of a C element from the product value (pr, pi), both in the computation
// precision AccT, C's old value from epi_load and the converted scalars. pi is ignored
// unless MODE pairs two real results into one complex value. Order of operations
// (Sec. 7.1): t = alpha*P rounded in AccT, cast to C's precision; beta*C formed in C's
// precision; their sum rounded in C's precision.
template <typename AccT, int CDT, int MODE>
__device__ __forceinline__ COld<CDT> epi_value(const EpiArgs& e, const EpiScalars<AccT, CDT>& sc, AccT pr, AccT pi,
                                               const COld<CDT>& old) {
  using CT = typename CStore<CDT>::T;
  COld<CDT> r;
  if constexpr (!CStore<CDT>::cplx) {
    // C real: alpha and beta projected onto the real line (Sec. 7.2).
    const CT t = to_ct<CT>(mul_rn(sc.ar, pr));
    r.re = e.beta_zero ? t : add_rn(mul_rn(sc.br, old.re), t);
    r.im = r.re;
  } else {
    AccT tr, ti;
    if constexpr (MODE == OUT_RE_ONLY) {
      tr = mul_rn(sc.ar, pr);     // case 1c: the product is real; with a real alpha it reaches Re(C) only
      ti = mul_rn(sc.ai, pr);     // (a complex alpha only under the literal reading)
    } else {
      tr = sub_rn(mul_rn(sc.ar, pr), mul_rn(sc.ai, pi));  // complex alpha honoured (case 3)
      ti = add_rn(mul_rn(sc.ar, pi), mul_rn(sc.ai, pr));  // ai == 0 otherwise
    }
    const CT tcr = to_ct<CT>(tr), tci = to_ct<CT>(ti);
    if (e.beta_zero) {
      r.re = tcr;
      r.im = (MODE == OUT_RE_ONLY && sc.ai_zero) ? to_ct<CT>(0.0f) : tci;
    } else {
      const CT cr = old.re, ci = old.im;
      const CT bcr = sub_rn(mul_rn(sc.br, cr), mul_rn(sc.bi, ci));
      const CT bci = add_rn(mul_rn(sc.br, ci), mul_rn(sc.bi, cr));
      r.re = add_rn(bcr, tcr);
      r.im = (MODE == OUT_RE_ONLY && sc.ai_zero) ? bci : add_rn(bci, tci);
    }
  }
  return r;
}

// The same update, stored to C(i, j) when (i, j) lies inside C.
template <typename AccT, int CDT, int MODE>
__device__ __forceinline__ void epi_update(const EpiArgs& e, const EpiScalars<AccT, CDT>& sc, int64_t i, int64_t j,
                                           AccT pr, AccT pi, const COld<CDT>& old) {
  using CT = typename CStore<CDT>::T;
  if (i >= e.m || j >= e.n) return;
  CT* c = static_cast<CT*>(e.C) + (i * e.rs + j * e.cs) * (CStore<CDT>::cplx ? 2 : 1);
  if (!MXG_DBG_OK(c_in_extent<CDT>(e, c), e.dbg)) return;
  const COld<CDT> r = epi_value<AccT, CDT, MODE>(e, sc, pr, pi, old);
  c[0] = r.re;
  if constexpr (CStore<CDT>::cplx) c[1] = r.im;
}

// Load, update and store one element of C.
template <typename AccT, int CDT, int MODE>
__device__ __forceinline__ void epi_store(const EpiArgs& e, const EpiScalars<AccT, CDT>& sc, int64_t i, int64_t j,
                                          AccT pr, AccT pi) {
  epi_update<AccT, CDT, MODE>(e, sc, i, j, pr, pi, epi_load<CDT>(e, i, j));
}

}  // namespace mxg
