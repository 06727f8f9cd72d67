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

// Update C(i, j) with the product value (pr, pi), both in the computation precision
// AccT. pi is ignored unless MODE pairs two real results into one complex value.
template <typename AccT, int CDT, int MODE>
__device__ __forceinline__ void epi_store(const EpiArgs& e, int64_t i, int64_t j, AccT pr, AccT pi) {
  using CT = typename CStore<CDT>::T;
  if (i >= e.m || j >= e.n) return;
  const AccT ar = static_cast<AccT>(e.ar);
  CT* c = static_cast<CT*>(e.C) + (i * e.rs + j * e.cs) * (CStore<CDT>::cplx ? 2 : 1);
  if constexpr (!CStore<CDT>::cplx) {
    // C real: alpha and beta projected onto the real line (Sec. 7.2).
    const CT t = static_cast<CT>(ar * pr);
    c[0] = e.beta_zero ? t : static_cast<CT>(e.br) * c[0] + t;
  } else {
    AccT tr, ti;
    if constexpr (MODE == OUT_RE_ONLY) {
      tr = ar * pr;            // case 1c: alpha is real; the product reaches Re(C) only
      ti = AccT(0);
    } else {
      const AccT ai = static_cast<AccT>(e.ai);
      tr = ar * pr - ai * pi;  // complex alpha honoured (case 3); ai == 0 otherwise
      ti = ar * pi + ai * pr;
    }
    const CT tcr = static_cast<CT>(tr), tci = static_cast<CT>(ti);
    if (e.beta_zero) {
      c[0] = tcr;
      c[1] = tci;
    } else {
      const CT br = static_cast<CT>(e.br), bi = static_cast<CT>(e.bi);
      const CT cr = c[0], ci = c[1];
      const CT bcr = br * cr - bi * ci;
      const CT bci = br * ci + bi * cr;
      c[0] = bcr + tcr;
      c[1] = (MODE == OUT_RE_ONLY) ? bci : bci + tci;
    }
  }
}

}  // namespace mxg
