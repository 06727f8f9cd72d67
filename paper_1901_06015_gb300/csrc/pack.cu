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

template <typename DT>
__device__ __forceinline__ DT pattern_value(int pattern, int s, int t, DT xr, DT xi) {
  // (for a real source the planner only uses PAT_RE, so xi is never read there)
  switch (pattern) {
    case PAT_SPLIT_MN: return t ? xi : xr;
    case PAT_SPLIT_K: return s ? xi : xr;
    case PAT_ONE_E: return s == 0 ? (t ? xi : xr) : (t ? xr : -xi);
    default: return xr;
  }
}

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
// the lanes along the source's unit-stride dimension (8 independent loads per
// thread), keep it in shared memory, and write the 32*fk x 64*fm packed sub-block as
// 16-byte vectors along the packed operand's contiguous dimension (MN for the SIMT
// layout, K for the tensor-core planes). Padded extents are multiples of the vector
// width, so a vector is either wholly inside or wholly outside them. Ends with the
// block synchronised.
template <int SDT, typename DT, int LAYOUT, int SPLIT>
__device__ __forceinline__ void pack_tile(const PackArgs& a, int64_t mn0, int64_t p0, PackSmem<DT>& sm) {
  using ST = typename SrcT<SDT>::T;
  constexpr bool SC = SrcT<SDT>::cplx;
  constexpr int V = OutVec<SPLIT, DT>::n;
  const int t = threadIdx.x;
  const bool unit_mn = (a.smn == 1);
  const int fk = (a.pattern == PAT_SPLIT_K || a.pattern == PAT_ONE_E) ? 2 : 1;
  const int fm = (a.pattern == PAT_SPLIT_MN || a.pattern == PAT_ONE_E) ? 2 : 1;
  ST vr_[8], vi_[8];
  int lm_[8], lp_[8];
  bool in_[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int lm = unit_mn ? (t & 63) : ((t >> 5) + 8 * i);
    const int lp = unit_mn ? ((t >> 6) + 4 * i) : (t & 31);
    const int64_t mn = mn0 + lm, p = p0 + lp;
    lm_[i] = lm; lp_[i] = lp;
    in_[i] = (mn < a.MN && p < a.K);
    vr_[i] = ST(0.0f); vi_[i] = ST(0.0f);
    if (in_[i]) {
      const ST* sp = static_cast<const ST*>(a.src) + (mn * a.smn + p * a.sk) * (SC ? 2 : 1);
      vr_[i] = __ldg(sp);
      if constexpr (SC) vi_[i] = __ldg(sp + 1);
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    DT re = widen<DT>(vr_[i]);
    if constexpr (SC) {   // a real source only ever uses the RE pattern
      DT im = widen<DT>(vi_[i]);
      if (a.conj) im = -im;
      if (a.fold) {       // alpha * x in the computation precision (literal complex alpha)
        const DT fr = static_cast<DT>(a.fold_re), fi = static_cast<DT>(a.fold_im);
        const DT nr = mul_sub(fr, re, fi, im), ni = mul_add(fr, im, fi, re);
        re = nr;
        im = ni;
      }
      sm.im[lp_[i]][lm_[i]] = im;
    }
    sm.re[lp_[i]][lm_[i]] = re;
  }
  __syncthreads();
  const int nk_out = PK_P * fk, nm_out = PK_MN * fm;
  if constexpr (LAYOUT == LAYOUT_MN_MAJOR) {
    const int vec_per_row = nm_out / V, total = nk_out * vec_per_row;
    for (int idx = t; idx < total; idx += 256) {
      const int r = idx / vec_per_row, c0 = (idx - r * vec_per_row) * V;
      const int64_t kk = p0 * fk + r, mm = mn0 * fm + c0;
      if (kk >= a.Kp || mm >= a.MNp) continue;
      const int lp = r / fk, s = r - lp * fk;
      DT v[V];
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int c = c0 + u, lm = c / fm, tt = c - lm * fm;
        v[u] = SC ? pattern_value<DT>(a.pattern, s, tt, sm.re[lp][lm], sm.im[lp][lm]) : sm.re[lp][lm];
      }
      DT* dst = static_cast<DT*>(a.dst) + kk * a.ld + mm;
      if constexpr (V == 4) *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      else *reinterpret_cast<double2*>(dst) = make_double2(v[0], v[1]);
    }
  } else {
    const int vec_per_row = nk_out / V, total = nm_out * vec_per_row;
    for (int idx = t; idx < total; idx += 256) {
      const int c = idx / vec_per_row, r0 = (idx - c * vec_per_row) * V;
      const int64_t kk = p0 * fk + r0, mm = mn0 * fm + c;
      if (kk >= a.Kp || mm >= a.MNp) continue;
      const int lm = c / fm, tt = c - lm * fm;
      const int64_t off = mm * a.ld + kk;
      if constexpr (SPLIT == SPLIT_F16_ONE || SPLIT == SPLIT_BF16_ONE) {
        // one plane rounded once from the working type (TC16)
        uint4 pk;
        uint16_t* p16 = reinterpret_cast<uint16_t*>(&pk);
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const int r = r0 + u, lp = r / fk, s = r - lp * fk;
          const DT x = SC ? pattern_value<DT>(a.pattern, s, tt, sm.re[lp][lm], sm.im[lp][lm]) : sm.re[lp][lm];
          if constexpr (SPLIT == SPLIT_F16_ONE) {
            const __half hv = to_f16(x);
            p16[u] = *reinterpret_cast<const uint16_t*>(&hv);
          } else {
            const __nv_bfloat16 bv = to_bf16(x);
            p16[u] = *reinterpret_cast<const uint16_t*>(&bv);
          }
        }
        *reinterpret_cast<uint4*>(static_cast<uint16_t*>(a.dst) + off) = pk;
        continue;
      } else {
      float hi[V], lo[V];
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int r = r0 + u, lp = r / fk, s = r - lp * fk;
        const float x = static_cast<float>(SC ? pattern_value<DT>(a.pattern, s, tt, sm.re[lp][lm], sm.im[lp][lm])
                                              : sm.re[lp][lm]);
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

template <int SDT, typename DT, int LAYOUT, int SPLIT>
__global__ void __launch_bounds__(256) pack_kernel(PackArgs a, int64_t ntile_p) {
  __shared__ PackSmem<DT> sm;
  const int64_t mn0 = static_cast<int64_t>(blockIdx.x) * PK_MN;
  for (int64_t tp = blockIdx.y; tp < ntile_p; tp += gridDim.y) pack_tile<SDT, DT, LAYOUT, SPLIT>(a, mn0, tp * PK_P, sm);
}

// Grouped pack: block b packs tile (b - tile_start[t]) of task t, where t is found by a
// binary search of the tile prefix sums; the tasks' source datatypes differ, so the
// source type is dispatched at run time (uniformly over the block).
template <typename DT>
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
  switch (a.src_dt) {
    case MXG_S: pack_tile<MXG_S, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_D: pack_tile<MXG_D, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_C: pack_tile<MXG_C, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_Z: pack_tile<MXG_Z, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_H: pack_tile<MXG_H, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_K: pack_tile<MXG_K, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_B: pack_tile<MXG_B, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_W: pack_tile<MXG_W, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
  }
}

template <int SDT>
cudaError_t launch_src(const PackArgs& a, int comp_double, cudaStream_t s) {
  const int fk = pat_fk(a.pattern), fm = pat_fm(a.pattern);
  const int64_t ntm = (a.MNp / fm + PK_MN - 1) / PK_MN, ntp = (a.Kp / fk + PK_P - 1) / PK_P;
  if (ntm <= 0 || ntp <= 0) return cudaSuccess;
  if (ntm > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(ntm), static_cast<unsigned>(ntp < 65535 ? ntp : 65535));
  if (a.split == SPLIT_NONE && a.layout == LAYOUT_MN_MAJOR) {
    if (comp_double) pack_kernel<SDT, double, LAYOUT_MN_MAJOR, SPLIT_NONE><<<grid, 256, 0, s>>>(a, ntp);
    else pack_kernel<SDT, float, LAYOUT_MN_MAJOR, SPLIT_NONE><<<grid, 256, 0, s>>>(a, ntp);
  } else if (a.split == SPLIT_TF32 && a.layout == LAYOUT_K_MAJOR && !comp_double) {
    pack_kernel<SDT, float, LAYOUT_K_MAJOR, SPLIT_TF32><<<grid, 256, 0, s>>>(a, ntp);
  } else if (a.split == SPLIT_BF16 && a.layout == LAYOUT_K_MAJOR && !comp_double) {
    pack_kernel<SDT, float, LAYOUT_K_MAJOR, SPLIT_BF16><<<grid, 256, 0, s>>>(a, ntp);
  } else if ((a.split == SPLIT_F16_ONE || a.split == SPLIT_BF16_ONE) && a.layout == LAYOUT_K_MAJOR) {
    // working type: the source's own precision, so the 16-bit rounding happens once
    constexpr bool src_double = (SDT == MXG_D || SDT == MXG_Z);
    using WT = typename std::conditional<src_double, double, float>::type;
    if (a.split == SPLIT_F16_ONE) pack_kernel<SDT, WT, LAYOUT_K_MAJOR, SPLIT_F16_ONE><<<grid, 256, 0, s>>>(a, ntp);
    else pack_kernel<SDT, WT, LAYOUT_K_MAJOR, SPLIT_BF16_ONE><<<grid, 256, 0, s>>>(a, ntp);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
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
  if (comp_double) pack_grouped_kernel<double><<<static_cast<unsigned>(ntiles), 256, 0, s>>>(tasks, tile_start, ntasks);
  else pack_grouped_kernel<float><<<static_cast<unsigned>(ntiles), 256, 0, s>>>(tasks, tile_start, ntasks);
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
