// Pack kernels: one HBM pass that reads op(X) in its storage datatype through any
// strides, casts it to the computation precision (Sec. 5.1.2: the target datatype is
// the operand's own domain with the computation precision; typecasting happens while
// packing), applies conjugation (Sec. 2.2.3), projects it by domain and lays it out
// as a real operand (the patterns of mxg_internal.h), and writes the padded packed
// operand in full (zeros outside the logical extent), so the contraction kernels run
// without bounds checks.
//
// A block handles a 32 (mn) x 32 (p) tile of logical elements: it reads the tile with
// the lanes along whichever source dimension has unit stride, keeps it in shared
// memory, and writes the 32*fk x 32*fm packed sub-block with the lanes along the
// packed operand's contiguous dimension, so both sides are coalesced for row-,
// column- and (as far as possible) general storage.
#include <cuda_bf16.h>

#include "mxg_internal.h"
#include "../../include/mxgemm.h"

namespace mxg {
namespace {

template <int DT> struct SrcT { using T = float; static constexpr bool cplx = false; };
template <> struct SrcT<MXG_D> { using T = double; static constexpr bool cplx = false; };
template <> struct SrcT<MXG_C> { using T = float; static constexpr bool cplx = true; };
template <> struct SrcT<MXG_Z> { using T = double; static constexpr bool cplx = true; };

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

template <typename DT>
__device__ __forceinline__ DT pattern_value(int pattern, int s, int t, DT xr, DT xi) {
  switch (pattern) {
    case PAT_SPLIT_MN: return t ? xi : xr;
    case PAT_SPLIT_K: return s ? xi : xr;
    case PAT_ONE_E: return s == 0 ? (t ? xi : xr) : (t ? xr : -xi);
    default: return xr;
  }
}

template <typename DT>
struct PackSmem {
  DT re[32][33];
  DT im[32][33];
};

// One 32 (mn) x 32 (p) tile of logical elements starting at (mn0, p0): read it with
// the lanes along the source's unit-stride dimension, keep it in shared memory, and
// write the 32*fk x 32*fm packed sub-block with the lanes along the packed operand's
// contiguous dimension. Ends with the block synchronised.
template <int SDT, typename DT, int LAYOUT, int SPLIT>
__device__ __forceinline__ void pack_tile(const PackArgs& a, int64_t mn0, int64_t p0, PackSmem<DT>& sm) {
  using ST = typename SrcT<SDT>::T;
  constexpr bool SC = SrcT<SDT>::cplx;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const bool unit_mn = (a.smn == 1);
  const int fk = (a.pattern == PAT_SPLIT_K || a.pattern == PAT_ONE_E) ? 2 : 1;
  const int fm = (a.pattern == PAT_SPLIT_MN || a.pattern == PAT_ONE_E) ? 2 : 1;
  for (int r = ty; r < 32; r += 8) {
    const int lm = unit_mn ? tx : r;
    const int lp = unit_mn ? r : tx;
    const int64_t mn = mn0 + lm, p = p0 + lp;
    DT vr = DT(0), vi = DT(0);
    if (mn < a.MN && p < a.K) {
      const ST* s = static_cast<const ST*>(a.src) + (mn * a.smn + p * a.sk) * (SC ? 2 : 1);
      vr = static_cast<DT>(s[0]);
      if constexpr (SC) vi = static_cast<DT>(a.conj ? -s[1] : s[1]);
    }
    sm.re[lp][lm] = vr;
    sm.im[lp][lm] = vi;
  }
  __syncthreads();
  const int nk_out = 32 * fk, nm_out = 32 * fm, total = nk_out * nm_out;
  for (int idx = threadIdx.x; idx < total; idx += 256) {
    int r, c;  // r: packed K index in the tile, c: packed MN index in the tile
    if constexpr (LAYOUT == LAYOUT_MN_MAJOR) {
      r = idx / nm_out;
      c = idx - r * nm_out;
    } else {
      c = idx / nk_out;
      r = idx - c * nk_out;
    }
    const int64_t kk = p0 * fk + r, mm = mn0 * fm + c;
    if (kk >= a.Kp || mm >= a.MNp) continue;
    const int lp = r / fk, s = r - lp * fk, lm = c / fm, t = c - lm * fm;
    const DT v = pattern_value<DT>(a.pattern, s, t, sm.re[lp][lm], sm.im[lp][lm]);
    const int64_t off = (LAYOUT == LAYOUT_MN_MAJOR) ? kk * a.ld + mm : mm * a.ld + kk;
    if constexpr (SPLIT == SPLIT_NONE) {
      static_cast<DT*>(a.dst)[off] = v;
    } else if constexpr (SPLIT == SPLIT_TF32) {
      const float hi = tf32_rne(static_cast<float>(v));
      const float lo = tf32_rne(static_cast<float>(v) - hi);
      static_cast<float*>(a.dst)[off] = hi;
      static_cast<float*>(a.dst_lo)[off] = lo;
    } else {
      const __nv_bfloat16 hi = __float2bfloat16_rn(static_cast<float>(v));
      const __nv_bfloat16 lo = __float2bfloat16_rn(static_cast<float>(v) - __bfloat162float(hi));
      static_cast<__nv_bfloat16*>(a.dst)[off] = hi;
      static_cast<__nv_bfloat16*>(a.dst_lo)[off] = lo;
    }
  }
  __syncthreads();
}

template <int SDT, typename DT, int LAYOUT, int SPLIT>
__global__ void __launch_bounds__(256) pack_kernel(PackArgs a, int64_t ntile_p) {
  __shared__ PackSmem<DT> sm;
  const int64_t mn0 = static_cast<int64_t>(blockIdx.x) * 32;
  for (int64_t tp = blockIdx.y; tp < ntile_p; tp += gridDim.y) pack_tile<SDT, DT, LAYOUT, SPLIT>(a, mn0, tp * 32, sm);
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
  const int64_t tiles_mn = (a.MNp / fm + 31) / 32;
  const int64_t mn0 = (local % tiles_mn) * 32, p0 = (local / tiles_mn) * 32;
  switch (a.src_dt) {
    case MXG_S: pack_tile<MXG_S, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_D: pack_tile<MXG_D, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_C: pack_tile<MXG_C, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
    case MXG_Z: pack_tile<MXG_Z, DT, LAYOUT_MN_MAJOR, SPLIT_NONE>(a, mn0, p0, sm); break;
  }
}

template <int SDT>
cudaError_t launch_src(const PackArgs& a, int comp_double, cudaStream_t s) {
  const int fk = pat_fk(a.pattern), fm = pat_fm(a.pattern);
  const int64_t ntm = (a.MNp / fm + 31) / 32, ntp = (a.Kp / fk + 31) / 32;
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
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

int64_t pack_tiles(const PackArgs& a) {
  const int fk = pat_fk(a.pattern), fm = pat_fm(a.pattern);
  return ((a.MNp / fm + 31) / 32) * ((a.Kp / fk + 31) / 32);
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
  }
  return cudaErrorInvalidValue;
}

}  // namespace mxg
