// Internal declarations shared by the host planner (api.cpp) and the CUDA kernels.
// Not part of the public C ABI (include/mxgemm.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace mxg {

// How one logical operand element x = xr + i*xi (already cast to the computation
// precision and conjugated if requested) is laid out in the packed real operand.
// The packed operand is a real (K' x MN') matrix; fk/fm are the factors by which a
// pattern expands K and MN.
//   RE        1x1: xr                     (real operand, or Re of a complex one:
//                                           cases 0, 1a, 1b, 1c, and the real side
//                                           of 2ac / 2bc)
//   SPLIT_MN  1x2: [xr, xi] along MN       (complex side of 2ac and 2bc: C and the
//                                           operand viewed as real 2m x n / k x 2n,
//                                           Sec. 4.2.5)
//   SPLIT_K   2x1: [xr; xi] along K        (the 1r format of the 1m method, Sec. 4.1;
//                                           with conj toggled on B it gives case 2ab,
//                                           Sec. 4.2.3)
//   ONE_E     2x2: K-row 0 [xr, xi], K-row 1 [-xi, xr]
//                                          (the 1e format of the 1m method, Eq. (1)
//                                           for A, Eq. (2) for B)
enum PackPattern : int { PAT_RE = 0, PAT_SPLIT_MN = 1, PAT_SPLIT_K = 2, PAT_ONE_E = 3 };

// Bytes of one element of a storage datatype (MXG_S .. MXG_W).
inline size_t dt_bytes(int dt) {
  static const size_t b[8] = {4, 8, 8, 16, 2, 4, 2, 4};
  return (dt >= 0 && dt < 8) ? b[dt] : 0;
}

__host__ __device__ inline int pat_fk(int p) { return (p == PAT_SPLIT_K || p == PAT_ONE_E) ? 2 : 1; }
__host__ __device__ inline int pat_fm(int p) { return (p == PAT_SPLIT_MN || p == PAT_ONE_E) ? 2 : 1; }

// How the real product P (M' x N') maps onto C.
//   OUT_REAL    C real: C(i,j) <- P(i,j)                  (cases 0, 1a, 1b, 2ab)
//   OUT_RE_ONLY C complex, P real: Re C(i,j) <- P(i,j);   (case 1c)
//               Im C(i,j) only scaled by beta
//   OUT_ROWPAIR C complex: C(i,j) <- P(2i,j) + i P(2i+1,j) (case 2ac; case 3 by Eq. (1))
//   OUT_COLPAIR C complex: C(i,j) <- P(i,2j) + i P(i,2j+1) (case 2bc; case 3 by Eq. (2))
enum OutMode : int { OUT_REAL = 0, OUT_RE_ONLY = 1, OUT_ROWPAIR = 2, OUT_COLPAIR = 3 };

// Layout of a packed operand: MN-major (element (kk, mm) at kk*ld + mm) for the SIMT
// kernels, K-major (element (kk, mm) at mm*ld + kk) for the tensor-core kernels.
enum PackLayout : int { LAYOUT_MN_MAJOR = 0, LAYOUT_K_MAJOR = 1 };

// Formats of the K-major planes written for the tensor-core methods: hi and lo planes
// of the split forms, or one plane rounded to binary16 / bfloat16 (TC16).
enum SplitKind : int { SPLIT_NONE = 0, SPLIT_TF32 = 1, SPLIT_BF16 = 2, SPLIT_F16_ONE = 3, SPLIT_BF16_ONE = 4 };

struct PackArgs {
  const void* src;   // source operand, storage datatype src_dt
  int src_dt;        // MXG_S..MXG_Z
  int64_t smn, sk;   // strides (elements) of logical element (mn, p) of op(X): src + mn*smn + p*sk
  int64_t MN, K;     // logical extent
  int pattern;       // PackPattern
  int conj;          // negate the imaginary part before applying the pattern
  void* dst;         // packed operand (hi plane for split formats)
  void* dst_lo;      // lo plane for split formats (else unused)
  int64_t ld;        // leading dimension of dst (elements)
  int64_t MNp, Kp;   // padded extent of the packed operand (written in full, zero padding)
  int layout;        // PackLayout
  int split;         // SplitKind
  int fold;          // multiply each element by (fold_re + i fold_im) before the pattern
  double fold_re, fold_im;
  int* dbg;          // debug builds (MXG_DEBUG_BOUNDS): error word for out-of-extent accesses
};

struct EpiArgs {
  void* C;           // C after the optional whole-op transpose
  int64_t rs, cs;    // strides of C (elements)
  int64_t m, n;      // extent of C
  double ar, ai;     // alpha, already rounded to the computation precision
  double br, bi;     // beta, already rounded to C's storage precision
  int beta_zero;     // C is not read
  int* dbg;          // debug builds (MXG_DEBUG_BOUNDS): error word for out-of-extent accesses
};

// Debug builds (compiled with -DMXG_DEBUG_BOUNDS, see build.py) check every element
// address the pack kernels read and write and every C address the epilogues read and
// write against the extent its arguments describe, and OR MXG_DEBUG_BOUNDS_FLAG into
// the error word when one falls outside (the access is then skipped). No trap: the
// host reads the word (mxg_check_device_error). Normal builds compile the checks out.
constexpr int MXG_DEBUG_BOUNDS_FLAG = 2;
#if defined(MXG_DEBUG_BOUNDS) && defined(__CUDACC__)
#define MXG_DBG_OK(cond, word) (((cond)) ? true : (((word) ? atomicOr((word), MXG_DEBUG_BOUNDS_FLAG) : 0), false))
#else
#define MXG_DBG_OK(cond, word) true
#endif

struct GemmArgs {
  const void* A;     // packed A' (comp precision), MN-major, Kp x lda
  const void* B;     // packed B', MN-major, Kp x ldb
  int64_t lda, ldb;  // = padded M', N'
  int64_t Kp;        // padded K' (multiple of the kernel's k tile)
  int64_t Mp, Np;    // padded M', N' (multiples of the kernel's tile)
  EpiArgs e;
};

// Tile sizes the planner pads to, per method.
struct TileCfg { int tm, tn, tk; };
TileCfg tile_cfg(int method);

// Launchers (return cudaError_t of the launch).
cudaError_t launch_pack(const PackArgs& a, int comp_double, cudaStream_t s);
cudaError_t launch_gemm_simt(int method, int c_dt, int mode, const GemmArgs& g, cudaStream_t s);
cudaError_t launch_scale_c(const EpiArgs& e, int c_dt, cudaStream_t s);
// Split-K: `splits` slices of kslice k elements accumulate into ws (splits x Np x Mp in
// the computation precision), then an ordered reduction applies the epilogue.
cudaError_t launch_gemm_splitk(int method, int c_dt, int mode, const GemmArgs& g, int splits, int64_t kslice,
                               void* ws, cudaStream_t s);
// Bounded-wait self-test: a wait nothing will satisfy, limited to `seconds`.
cudaError_t launch_wait_timeout_probe(int* err, double seconds, cudaStream_t s);
// Tensor-core contraction: planes = {A_hi, A_lo, B_hi, B_lo}, K-major (one plane per
// operand for the TC16 formats: the lo entries are ignored).
cudaError_t launch_gemm_tc(int method, int split, int c_dt, int mode, const void* const planes[4], int64_t Mp,
                           int64_t Np, int64_t Kp, const EpiArgs& e, int* err, cudaStream_t s);
// The same contraction on CTA pairs (tcgen05 cta_group::2, 256 x 256 pair tiles; Mp a
// multiple of 128, Np of 256). sk_ws / sk_bytes: workspace for the stream-K tail (null:
// none); sk_mode 0 off, 1 automatic, 2 whenever the last wave is partial. The tail runs
// only when the workspace holds tc_pair_stream_k_bytes(resident pairs).
cudaError_t launch_gemm_tc_pair(int split, int c_dt, int mode, const void* const planes[4], int64_t Mp, int64_t Np,
                                int64_t Kp, const EpiArgs& e, int* err, void* sk_ws, size_t sk_bytes, int sk_mode,
                                cudaStream_t s);
// Stream-K tail decision for `tiles` pair tiles of nkb k-blocks on `pairs` resident pairs.
bool tc_pair_stream_k(int64_t tiles, int64_t nkb, int64_t pairs, int mode);
// Workspace of the tail for `pairs` resident pairs (partial slots and tile counters).
size_t tc_pair_stream_k_bytes(int64_t pairs);
// Workspace a pair-kernel plan reserves for the tail (0 when the tail would not run),
// assuming sm_count / 2 resident pairs (152 SMs when sm_count is 0).
size_t tc_pair_stream_k_workspace(int split, int64_t Mp, int64_t Np, int64_t Kp, int sm_count, int mode);

}  // namespace mxg
