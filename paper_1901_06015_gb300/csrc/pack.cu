// Pack kernels: one HBM pass that reads op(X) in its storage datatype through any
// strides, casts it to the computation precision (Sec. 5.1.2: the target datatype is
// the operand's own domain with the computation precision; typecasting happens while
// packing), applies conjugation (Sec. 2.2.3), projects it by domain and lays it out
// as a real operand (the patterns of mxg_internal.h), and writes the padded packed
// operand in full (zeros outside the logical extent), so the contraction kernels run
// without bounds checks.
//
// A block handles a 64 (mn) x 32 (p) tile of logical elements: it reads the tile with
// the lanes along whichever source dimension has unit stride, keeps it in shared
// memory, and writes the packed sub-block in 16-byte vectors along the packed
// operand's contiguous dimension, so both sides are coalesced for row-, column- and
// (as far as possible) general storage.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "mxg_internal.h"
#include "../../include/mxgemm.h"

namespace mxg {
namespace {

template <int DT> struct SrcT { using T = float; static constexpr bool cplx = false; };
template <> struct SrcT<MXG_D> { using T = double; static constexpr bool cplx = false; };
template <> struct SrcT<MXG_C> { using T = float; static constexpr bool cplx = true; };
template <> struct SrcT<MXG_Z> { using T = double; static constexpr bool cplx = true; };
template <> struct SrcT<MXG_H> { using T = __half; static constexpr bool cplx = false; };
template <> struct SrcT<MXG_K> { using T = __half; static constexpr bool cplx = true; };
template <> struct SrcT<MXG_B> { using T = __nv_bfloat16; static constexpr bool cplx = false; };
template <> struct SrcT<MXG_W> { using T = __nv_bfloat16; static constexpr bool cplx = true; };

// Exact widening of a stored component to the working type.
template <typename DT> __device__ __forceinline__ DT widen(float x) { return static_cast<DT>(x); }
template <typename DT> __device__ __forceinline__ DT widen(double x) { return static_cast<DT>(x); }
template <typename DT> __device__ __forceinline__ DT widen(__half x) { return static_cast<DT>(__half2float(x)); }
template <typename DT> __device__ __forceinline__ DT widen(__nv_bfloat16 x) { return static_cast<DT>(__bfloat162float(x)); }

// One rounding (RN-even) from the working type to binary16 / bfloat16.
__device__ __forceinline__ __half to_f16(float x) { return __float2half_rn(x); }
__device__ __forceinline__ __half to_f16(double x) { return __double2half(x); }
__device__ __forceinline__ __nv_bfloat16 to_bf16(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ __nv_bfloat16 to_bf16(double x) { return __double2bfloat16(x); }

// Round-to-nearest-even of an FP32 value to TF32 (10 explicit mantissa bits), done on
// the bit pattern; infinities and NaNs pass through.
__device__ __forceinline__ float tf32_rne(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0xfffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  return __uint_as_float(u);
}

// a*b - c*d and a*b + c*d with each product and the sum rounded (no FMA contraction)
__device__ __forceinline__ float mul_sub(float a, float b, float c, float d) {
  return __fsub_rn(__fmul_rn(a, b), __fmul_rn(c, d));
}
__device__ __forceinline__ double mul_sub(double a, double b, double c, double d) {
  return __dsub_rn(__dmul_rn(a, b), __dmul_rn(c, d));
}
__device__ __forceinline__ float mul_add(float a, float b, float c, float d) {
  return __fadd_rn(__fmul_rn(a, b), __fmul_rn(c, d));
}
__device__ __forceinline__ double mul_add(double a, double b, double c, double d) {
  return __dadd_rn(__dmul_rn(a, b), __dmul_rn(c, d));
}

// Value of packed element (k-row sub-index s, mn-column sub-index t) of logical element
// (xr, xi) under pattern PAT (a real source only ever uses PAT_RE, so xi is not read
// there).
template <int PAT, typename DT>
__device__ __forceinline__ DT pattern_value(int s, int t, DT xr, DT xi) {
  if constexpr (PAT == PAT_SPLIT_MN) return t ? xi : xr;
  else if constexpr (PAT == PAT_SPLIT_K) return s ? xi : xr;
  else if constexpr (PAT == PAT_ONE_E) return s == 0 ? (t ? xi : xr) : (t ? xr : -xi);
  else return xr;
}
// Packed rows per logical k (FK) and packed columns per logical mn (FM) of a pattern.
template <int PAT> struct PatDim {
  static constexpr int FK = (PAT == PAT_SPLIT_K || PAT == PAT_ONE_E) ? 2 : 1;
  static constexpr int FM = (PAT == PAT_SPLIT_MN || PAT == PAT_ONE_E) ? 2 : 1;
};

constexpr int PK_MN = 64, PK_P = 32;   // logical tile: 64 (mn) x 32 (p) elements

template <typename DT>
struct PackSmem {
  DT re[PK_P][PK_MN + 1];
  DT im[PK_P][PK_MN + 1];
};

template <int SPLIT, typename DT> struct OutVec;
template <> struct OutVec<SPLIT_NONE, float> { static constexpr int n = 4; };
template <> struct OutVec<SPLIT_NONE, double> { static constexpr int n = 2; };
template <> struct OutVec<SPLIT_TF32, float> { static constexpr int n = 4; };
template <> struct OutVec<SPLIT_BF16, float> { static constexpr int n = 8; };
template <typename DT> struct OutVec<SPLIT_F16_ONE, DT> { static constexpr int n = 8; };
template <typename DT> struct OutVec<SPLIT_BF16_ONE, DT> { static constexpr int n = 8; };

// One 64 (mn) x 32 (p) tile of logical elements starting at (mn0, p0): read it with
// the lanes along the source's smaller-stride dimension (8 independent loads per
// thread, addressed from one base pointer and a fixed step; bounds checked only in
// tiles that cross the logical extent), keep it in shared memory, and write the
// 32*FK x 64*FM packed sub-block as 16-byte vectors along the packed operand's
// contiguous dimension (MN for the SIMT layout, K for the tensor-core planes). The
// pattern is a template parameter, so the index arithmetic of the write-out is
// shifts and masks. Padded extents are multiples of the vector width, so a vector is
// either wholly inside or wholly outside them. Ends with the block synchronised.
template <int SDT, typename DT, int LAYOUT, int SPLIT, int PAT>
__device__ __forceinline__ void pack_tile(const PackArgs& a, int64_t mn0, int64_t p0, PackSmem<DT>& sm) {
  using ST = typename SrcT<SDT>::T;
  constexpr bool SC = SrcT<SDT>::cplx;
  constexpr int V = OutVec<SPLIT, DT>::n;
  constexpr int FK = PatDim<PAT>::FK, FM = PatDim<PAT>::FM;
  constexpr int64_t CM = SC ? 2 : 1;   // stored components per element
  const int t = threadIdx.x;
  // lanes along the dimension with the smaller stride (the unit-stride one for column-
  // or row-stored operands; for general storage the closer-packed one)
  const bool unit_mn = (a.smn <= a.sk);
  // element i of this thread: (lm0 + i*dm, lp0 + i*dp)
  const int lm0 = unit_mn ? (t & 63) : (t >> 5), lp0 = unit_mn ? (t >> 6) : (t & 31);
  const int dm = unit_mn ? 0 : 8, dp = unit_mn ? 4 : 0;
  ST vr[8], vi[8];
  const ST* src = static_cast<const ST*>(a.src);
#ifdef MXG_DEBUG_BOUNDS
  // last stored component of the source operand: (MN-1, K-1), imaginary part included
  const int64_t src_last = ((a.MN - 1) * a.smn + (a.K - 1) * a.sk) * CM + (CM - 1);
#endif
  if (mn0 + PK_MN <= a.MN && p0 + PK_P <= a.K) {
    const ST* sp = src + ((mn0 + lm0) * a.smn + (p0 + lp0) * a.sk) * CM;
    const int64_t step = (dm * a.smn + dp * a.sk) * CM;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const ST* q = sp + i * step;
      if (!MXG_DBG_OK(q >= src && q + (CM - 1) - src <= src_last, a.dbg)) {
        vr[i] = ST(0.0f);
        vi[i] = ST(0.0f);
        continue;
      }
      vr[i] = __ldg(q);
      if constexpr (SC) vi[i] = __ldg(q + 1);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t mn = mn0 + lm0 + i * dm, p = p0 + lp0 + i * dp;
      vr[i] = ST(0.0f);
      vi[i] = ST(0.0f);
      if (mn < a.MN && p < a.K) {
        const ST* sp = src + (mn * a.smn + p * a.sk) * CM;
        if (!MXG_DBG_OK(sp >= src && sp + (CM - 1) - src <= src_last, a.dbg)) continue;
        vr[i] = __ldg(sp);
        if constexpr (SC) vi[i] = __ldg(sp + 1);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int lm = lm0 + i * dm, lp = lp0 + i * dp;
    DT re = widen<DT>(vr[i]);
    if constexpr (SC) {
      DT im = widen<DT>(vi[i]);
      if (a.conj) im = -im;
      if (a.fold) {       // alpha * x in the computation precision (literal complex alpha)
        const DT fr = static_cast<DT>(a.fold_re), fi = static_cast<DT>(a.fold_im);
        const DT nr = mul_sub(fr, re, fi, im), ni = mul_add(fr, im, fi, re);
        re = nr;
        im = ni;
      }
      sm.im[lp][lm] = im;
    }
    sm.re[lp][lm] = re;
  }
  __syncthreads();
  constexpr int NK = PK_P * FK, NM = PK_MN * FM;
  auto value = [&](int r, int c) -> DT {   // packed element (row r of k, column c of mn) of the tile
    const int lp = r / FK, sk = r % FK, lm = c / FM, tt = c % FM;
    if constexpr (SC) return pattern_value<PAT, DT>(sk, tt, sm.re[lp][lm], sm.im[lp][lm]);
    else return sm.re[lp][lm];
  };
  if constexpr (LAYOUT == LAYOUT_MN_MAJOR) {
    constexpr int VPR = NM / V, TOTAL = NK * VPR;
#pragma unroll 1
    for (int idx = t; idx < TOTAL; idx += 256) {
      const int r = idx / VPR, c0 = (idx % VPR) * V;
      const int64_t kk = p0 * FK + r, mm = mn0 * FM + c0;
      if (kk >= a.Kp || mm >= a.MNp) continue;
      // the packed operand is Kp rows of ld elements; a vector lies inside it
      if (!MXG_DBG_OK(mm + V <= a.ld && kk * a.ld + mm + V <= a.Kp * a.ld, a.dbg)) continue;
      DT v[V];
#pragma unroll
      for (int u = 0; u < V; ++u) v[u] = value(r, c0 + u);
      DT* dst = static_cast<DT*>(a.dst) + kk * a.ld + mm;
      if constexpr (V == 4) *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      else *reinterpret_cast<double2*>(dst) = make_double2(v[0], v[1]);
    }
  } else {
    constexpr int VPR = NK / V, TOTAL = NM * VPR;
#pragma unroll 1
    for (int idx = t; idx < TOTAL; idx += 256) {
      const int c = idx / VPR, r0 = (idx % VPR) * V;
      const int64_t kk = p0 * FK + r0, mm = mn0 * FM + c;
      if (kk >= a.Kp || mm >= a.MNp) continue;
      const int64_t off = mm * a.ld + kk;
      // the packed planes are MNp rows of ld elements; a vector lies inside them
      if (!MXG_DBG_OK(kk + V <= a.ld && off + V <= a.MNp * a.ld, a.dbg)) continue;
      if constexpr (SPLIT == SPLIT_F16_ONE || SPLIT == SPLIT_BF16_ONE) {
        // one plane rounded once from the working type (TC16)
        uint4 pk;
        uint16_t* p16 = reinterpret_cast<uint16_t*>(&pk);
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const DT x = value(r0 + u, c);
          if constexpr (SPLIT == SPLIT_F16_ONE) {
            const __half hv = to_f16(x);
            p16[u] = *reinterpret_cast<const uint16_t*>(&hv);
          } else {
            const __nv_bfloat16 bv = to_bf16(x);
            p16[u] = *reinterpret_cast<const uint16_t*>(&bv);
          }
        }
        *reinterpret_cast<uint4*>(static_cast<uint16_t*>(a.dst) + off) = pk;
      } else {
        float hi[V], lo[V];
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const float x = static_cast<float>(value(r0 + u, c));
          if constexpr (SPLIT == SPLIT_TF32) {
            hi[u] = tf32_rne(x);
            lo[u] = tf32_rne(x - hi[u]);
          } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            hi[u] = __bfloat162float(h);
            lo[u] = x - hi[u];
          }
        }
        if constexpr (SPLIT == SPLIT_TF32) {
          *reinterpret_cast<float4*>(static_cast<float*>(a.dst) + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<float4*>(static_cast<float*>(a.dst_lo) + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        } else {
          uint4 ph, pl;
          uint32_t* h32 = reinterpret_cast<uint32_t*>(&ph);
          uint32_t* l32 = reinterpret_cast<uint32_t*>(&pl);
#pragma unroll
          for (int u = 0; u < V; u += 2) {
            const __nv_bfloat162 hh = __floats2bfloat162_rn(hi[u], hi[u + 1]);   // exact: already bf16
            const __nv_bfloat162 ll = __floats2bfloat162_rn(lo[u], lo[u + 1]);   // RN of x - hi
            h32[u / 2] = *reinterpret_cast<const uint32_t*>(&hh);
            l32[u / 2] = *reinterpret_cast<const uint32_t*>(&ll);
          }
          *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.dst) + off) = ph;
          *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.dst_lo) + off) = pl;
        }
      }
    }
  }
  __syncthreads();
}

// Call f(IC<pattern>) for the pattern of a (a real source only ever has PAT_RE).
template <int SDT, class F>
__device__ __host__ __forceinline__ bool with_pattern(int pattern, F&& f) {
  if constexpr (!SrcT<SDT>::cplx) {
    if (pattern != PAT_RE) return false;
    f(std::integral_constant<int, PAT_RE>{});
    return true;
  } else {
    switch (pattern) {
      case PAT_RE: f(std::integral_constant<int, PAT_RE>{}); return true;
      case PAT_SPLIT_MN: f(std::integral_constant<int, PAT_SPLIT_MN>{}); return true;
      case PAT_SPLIT_K: f(std::integral_constant<int, PAT_SPLIT_K>{}); return true;
      case PAT_ONE_E: f(std::integral_constant<int, PAT_ONE_E>{}); return true;
    }
    return false;
  }
}

template <int SDT, typename DT, int LAYOUT, int SPLIT, int PAT>
__global__ void __launch_bounds__(256, 5) pack_kernel(PackArgs a, int64_t ntile_p) {
  __shared__ PackSmem<DT> sm;
  const int64_t mn0 = static_cast<int64_t>(blockIdx.x) * PK_MN;
  for (int64_t tp = blockIdx.y; tp < ntile_p; tp += gridDim.y)
    pack_tile<SDT, DT, LAYOUT, SPLIT, PAT>(a, mn0, tp * PK_P, sm);
}

// Grouped pack: block b packs tile (b - tile_start[t]) of task t, where t is found by a
// binary search of the tile prefix sums; the tasks' source datatypes and patterns
// differ, so both are dispatched at run time (uniformly over the block). The layout and
// plane format are the bucket's: MN-major for the SIMT / DMMA kernels, or the K-major
// planes of one tensor-core format.
template <typename DT, int LAYOUT, int SPLIT>
__global__ void __launch_bounds__(256) pack_grouped_kernel(const PackArgs* __restrict__ tasks,
                                                           const int64_t* __restrict__ tile_start, int ntasks) {
  __shared__ PackSmem<DT> sm;
  const int64_t b = blockIdx.x;
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {   // last t with tile_start[t] <= b
    const int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= b) lo = mid; else hi = mid - 1;
  }
  const PackArgs a = tasks[lo];
  const int64_t local = b - tile_start[lo];
  const int fm = pat_fm(a.pattern);
  const int64_t tiles_mn = (a.MNp / fm + PK_MN - 1) / PK_MN;
  const int64_t mn0 = (local % tiles_mn) * PK_MN, p0 = (local / tiles_mn) * PK_P;
  auto run = [&](auto S) {
    constexpr int SDT = decltype(S)::value;
    with_pattern<SDT>(a.pattern, [&](auto P) {
      pack_tile<SDT, DT, LAYOUT, SPLIT, decltype(P)::value>(a, mn0, p0, sm);
    });
  };
  switch (a.src_dt) {
    case MXG_S: run(std::integral_constant<int, MXG_S>{}); break;
    case MXG_D: run(std::integral_constant<int, MXG_D>{}); break;
    case MXG_C: run(std::integral_constant<int, MXG_C>{}); break;
    case MXG_Z: run(std::integral_constant<int, MXG_Z>{}); break;
    case MXG_H: run(std::integral_constant<int, MXG_H>{}); break;
    case MXG_K: run(std::integral_constant<int, MXG_K>{}); break;
    case MXG_B: run(std::integral_constant<int, MXG_B>{}); break;
    case MXG_W: run(std::integral_constant<int, MXG_W>{}); break;
  }
}

template <int SDT, typename DT, int LAYOUT, int SPLIT>
cudaError_t launch_pattern(const PackArgs& a, dim3 grid, int64_t ntp, cudaStream_t s) {
  const bool ok = with_pattern<SDT>(a.pattern, [&](auto P) {
    pack_kernel<SDT, DT, LAYOUT, SPLIT, decltype(P)::value><<<grid, 256, 0, s>>>(a, ntp);
  });
  return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

template <int SDT>
cudaError_t launch_src(const PackArgs& a, int comp_double, cudaStream_t s) {
  const int fk = pat_fk(a.pattern), fm = pat_fm(a.pattern);
  const int64_t ntm = (a.MNp / fm + PK_MN - 1) / PK_MN, ntp = (a.Kp / fk + PK_P - 1) / PK_P;
  if (ntm <= 0 || ntp <= 0) return cudaSuccess;
  if (ntm > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(ntm), static_cast<unsigned>(ntp < 65535 ? ntp : 65535));
  if (a.split == SPLIT_NONE && a.layout == LAYOUT_MN_MAJOR) {
    if (comp_double) return launch_pattern<SDT, double, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, grid, ntp, s);
    return launch_pattern<SDT, float, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, grid, ntp, s);
  } else if (a.split == SPLIT_TF32 && a.layout == LAYOUT_K_MAJOR && !comp_double) {
    return launch_pattern<SDT, float, LAYOUT_K_MAJOR, SPLIT_TF32>(a, grid, ntp, s);
  } else if (a.split == SPLIT_BF16 && a.layout == LAYOUT_K_MAJOR && !comp_double) {
    return launch_pattern<SDT, float, LAYOUT_K_MAJOR, SPLIT_BF16>(a, grid, ntp, s);
  } else if ((a.split == SPLIT_F16_ONE || a.split == SPLIT_BF16_ONE) && a.layout == LAYOUT_K_MAJOR) {
    // working type: the source's own precision, so the 16-bit rounding happens once
    constexpr bool src_double = (SDT == MXG_D || SDT == MXG_Z);
    using WT = typename std::conditional<src_double, double, float>::type;
    if (a.split == SPLIT_F16_ONE) return launch_pattern<SDT, WT, LAYOUT_K_MAJOR, SPLIT_F16_ONE>(a, grid, ntp, s);
    return launch_pattern<SDT, WT, LAYOUT_K_MAJOR, SPLIT_BF16_ONE>(a, grid, ntp, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int64_t pack_tiles(const PackArgs& a) {
  const int fk = pat_fk(a.pattern), fm = pat_fm(a.pattern);
  return ((a.MNp / fm + PK_MN - 1) / PK_MN) * ((a.Kp / fk + PK_P - 1) / PK_P);
}

cudaError_t launch_pack_grouped(const PackArgs* tasks, const int64_t* tile_start, int ntasks, int64_t ntiles,
                                int comp_double, cudaStream_t s) {
  if (ntasks <= 0 || ntiles <= 0) return cudaSuccess;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const unsigned grid = static_cast<unsigned>(ntiles);
  if (comp_double)
    pack_grouped_kernel<double, LAYOUT_MN_MAJOR, SPLIT_NONE><<<grid, 256, 0, s>>>(tasks, tile_start, ntasks);
  else
    pack_grouped_kernel<float, LAYOUT_MN_MAJOR, SPLIT_NONE><<<grid, 256, 0, s>>>(tasks, tile_start, ntasks);
  return cudaGetLastError();
}

cudaError_t launch_pack_grouped_tc(const PackArgs* tasks, const int64_t* tile_start, int ntasks, int64_t ntiles,
                                   int split, cudaStream_t s) {
  if (ntasks <= 0 || ntiles <= 0) return cudaSuccess;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const unsigned grid = static_cast<unsigned>(ntiles);
  // the split forms cast to single precision first; the one-plane 16-bit formats round
  // once from a double working type (exact for every source, so the same rounding as
  // the single-problem pack's source-precision working type)
  switch (split) {
    case SPLIT_TF32:
      pack_grouped_kernel<float, LAYOUT_K_MAJOR, SPLIT_TF32><<<grid, 256, 0, s>>>(tasks, tile_start, ntasks);
      break;
    case SPLIT_BF16:
      pack_grouped_kernel<float, LAYOUT_K_MAJOR, SPLIT_BF16><<<grid, 256, 0, s>>>(tasks, tile_start, ntasks);
      break;
    case SPLIT_F16_ONE:
      pack_grouped_kernel<double, LAYOUT_K_MAJOR, SPLIT_F16_ONE><<<grid, 256, 0, s>>>(tasks, tile_start, ntasks);
      break;
    case SPLIT_BF16_ONE:
      pack_grouped_kernel<double, LAYOUT_K_MAJOR, SPLIT_BF16_ONE><<<grid, 256, 0, s>>>(tasks, tile_start, ntasks);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pack(const PackArgs& a, int comp_double, cudaStream_t s) {
  switch (a.src_dt) {
    case MXG_S: return launch_src<MXG_S>(a, comp_double, s);
    case MXG_D: return launch_src<MXG_D>(a, comp_double, s);
    case MXG_C: return launch_src<MXG_C>(a, comp_double, s);
    case MXG_Z: return launch_src<MXG_Z>(a, comp_double, s);
    case MXG_H: return launch_src<MXG_H>(a, comp_double, s);
    case MXG_K: return launch_src<MXG_K>(a, comp_double, s);
    case MXG_B: return launch_src<MXG_B>(a, comp_double, s);
    case MXG_W: return launch_src<MXG_W>(a, comp_double, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mxg
