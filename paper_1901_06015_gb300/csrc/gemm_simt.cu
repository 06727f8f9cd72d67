// Plain contraction kernels with the fused epilogue: the real gemm P = A' B' over the
// packed operands (M' x N' x K' from the domain case, Fig. "mixeddom"), accumulated
// over the whole K' in the computation precision (Sec. 6.3: one cast per element of
// C, no intermediate round-off in C's precision), then alpha / beta / store.
//
//  * simt_gemm<float>  : FP32 FFMA, 128 x 128 CTA tile, 8 x 8 outputs per thread.
//  * simt_gemm<double> : FP64 DFMA,  64 x 64 CTA tile, 4 x 4 outputs per thread.
//  * dmma_gemm         : FP64 tensor-core mma.sync.m8n8k4, 64 x 64 CTA tile, 4 warps.
//
// Packed operands are MN-major (element (kk, mm) at kk*ld + mm) and padded to whole
// tiles with zeros, so the main loops have no bounds checks. Each thread owns pairs of
// adjacent rows and adjacent columns, so the complex pairings of the 1m layouts
// (rows 2i, 2i+1 or columns 2j, 2j+1) are formed in registers.
#include "epilogue.cuh"

namespace mxg {
namespace {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using V = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using V = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void unpack16(const typename Vec16<T>::V& v, T* out);
template <>
__device__ __forceinline__ void unpack16<float>(const float4& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
template <>
__device__ __forceinline__ void unpack16<double>(const double2& v, double* o) { o[0] = v.x; o[1] = v.y; }

// Generic SIMT tile: 256 threads as 16 x 16; thread (tm, tn) owns rows
// {tm*H + i, TM/2 + tm*H + i} and columns {tn*H + j, TN/2 + tn*H + j}, i, j < H,
// where H = 16 bytes / sizeof(T) (one vector load per half).
template <typename T, int CDT, int MODE>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 2 : 3)) simt_gemm(GemmArgs g) {
  using V = typename Vec16<T>::V;
  constexpr int H = Vec16<T>::n;      // elements per 16-byte vector
  constexpr int TM = 32 * H, TN = 32 * H, TK = 8;
  constexpr int R = 2 * H;            // outputs per thread per dimension
  __shared__ __align__(16) T As[2][TK][TM];
  __shared__ __align__(16) T Bs[2][TK][TN];

  const int tid = threadIdx.x;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * TM;
  const int64_t n0 = static_cast<int64_t>(blockIdx.y) * TN;
  // global -> shared: TK rows x TM elements = 256 vectors, one per thread
  const int lrow = tid / (TM / H), lcol = (tid % (TM / H)) * H;
  const T* Ag = static_cast<const T*>(g.A) + lrow * g.lda + m0 + lcol;
  const T* Bg = static_cast<const T*>(g.B) + lrow * g.ldb + n0 + lcol;
  V ra = __ldg(reinterpret_cast<const V*>(Ag));
  V rb = __ldg(reinterpret_cast<const V*>(Bg));
  *reinterpret_cast<V*>(&As[0][lrow][lcol]) = ra;
  *reinterpret_cast<V*>(&Bs[0][lrow][lcol]) = rb;
  __syncthreads();

  T acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = T(0);

  const int tm = tid & 15, tn = tid >> 4;
  const int64_t nk = g.Kp / TK;
  int buf = 0;
  for (int64_t kt = 0; kt < nk; ++kt) {
    const bool more = (kt + 1 < nk);
    if (more) {
      Ag += TK * g.lda;
      Bg += TK * g.ldb;
      ra = __ldg(reinterpret_cast<const V*>(Ag));
      rb = __ldg(reinterpret_cast<const V*>(Bg));
    }
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T a[R], b[R];
      unpack16<T>(*reinterpret_cast<const V*>(&As[buf][kk][tm * H]), a);
      unpack16<T>(*reinterpret_cast<const V*>(&As[buf][kk][TM / 2 + tm * H]), a + H);
      unpack16<T>(*reinterpret_cast<const V*>(&Bs[buf][kk][tn * H]), b);
      unpack16<T>(*reinterpret_cast<const V*>(&Bs[buf][kk][TN / 2 + tn * H]), b + H);
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) {
      *reinterpret_cast<V*>(&As[buf ^ 1][lrow][lcol]) = ra;
      *reinterpret_cast<V*>(&Bs[buf ^ 1][lrow][lcol]) = rb;
      __syncthreads();
      buf ^= 1;
    }
  }

  // Fused epilogue.
  auto row_of = [&](int i) -> int64_t { return m0 + (i < H ? tm * H + i : TM / 2 + tm * H + (i - H)); };
  auto col_of = [&](int j) -> int64_t { return n0 + (j < H ? tn * H + j : TN / 2 + tn * H + (j - H)); };
  if constexpr (MODE == OUT_ROWPAIR) {
#pragma unroll
    for (int i = 0; i < R; i += 2)
#pragma unroll
      for (int j = 0; j < R; ++j)
        epi_store<T, CDT, MODE>(g.e, row_of(i) >> 1, col_of(j), acc[i][j], acc[i + 1][j]);
  } else if constexpr (MODE == OUT_COLPAIR) {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; j += 2)
        epi_store<T, CDT, MODE>(g.e, row_of(i), col_of(j) >> 1, acc[i][j], acc[i][j + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j)
        epi_store<T, CDT, MODE>(g.e, row_of(i), col_of(j), acc[i][j], T(0));
  }
}

// FP64 tensor-core kernel (mma.sync.aligned.m8n8k4 .f64). 128 threads = 2 x 2 warps,
// each warp a 32 x 32 sub-tile of 4 x 4 mma blocks. Shared rows are padded to 68
// doubles so the fragment loads (4 k-rows x 8 m-columns per half warp) hit 16
// distinct 8-byte banks. The accumulator tile is staged through shared memory for the
// epilogue, which then pairs rows or columns for the complex layouts.
constexpr int DM_T = 64, DM_TK = 16, DM_LD = DM_T + 4;

template <int CDT, int MODE>
__global__ void __launch_bounds__(128) dmma_gemm(GemmArgs g) {
  __shared__ __align__(16) double smem[2 * 2 * DM_TK * DM_LD];
  double* As = smem;                       // [2][TK][LD]
  double* Bs = smem + 2 * DM_TK * DM_LD;   // [2][TK][LD]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * DM_T;
  const int64_t n0 = static_cast<int64_t>(blockIdx.y) * DM_T;
  const double* A = static_cast<const double*>(g.A);
  const double* B = static_cast<const double*>(g.B);

  // global -> shared: TK x 64 doubles = 512 double2 per operand, 4 per thread.
  double2 ra[4], rb[4];
  auto gload = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + r * 128, row = idx >> 5, col = (idx & 31) * 2;
      ra[r] = __ldg(reinterpret_cast<const double2*>(A + (k0 + row) * g.lda + m0 + col));
      rb[r] = __ldg(reinterpret_cast<const double2*>(B + (k0 + row) * g.ldb + n0 + col));
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + r * 128, row = idx >> 5, col = (idx & 31) * 2;
      *reinterpret_cast<double2*>(&As[(buf * DM_TK + row) * DM_LD + col]) = ra[r];
      *reinterpret_cast<double2*>(&Bs[(buf * DM_TK + row) * DM_LD + col]) = rb[r];
    }
  };
  gload(0);
  sstore(0);
  __syncthreads();

  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  const int fr = lane & 3, fc = lane >> 2;
  const int64_t nk = g.Kp / DM_TK;
  int buf = 0;
  for (int64_t kt = 0; kt < nk; ++kt) {
    const bool more = (kt + 1 < nk);
    if (more) gload((kt + 1) * DM_TK);
#pragma unroll
    for (int kk = 0; kk < DM_TK; kk += 4) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[(buf * DM_TK + kk + fr) * DM_LD + wm * 32 + i * 8 + fc];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[(buf * DM_TK + kk + fr) * DM_LD + wn * 32 + j * 8 + fc];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                       : "+d"(acc[i][j][0]), "+d"(acc[i][j][1])
                       : "d"(a[i]), "d"(b[j]));
    }
    if (more) {
      sstore(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

  // Stage the 64 x 64 accumulator tile as Cs[col][row] (row contiguous).
  constexpr int CLD = DM_T + 1;
  static_assert(DM_T * CLD <= 2 * 2 * DM_TK * DM_LD, "staging tile must fit");
  __syncthreads();
  double* Cs = smem;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = wm * 32 + i * 8 + fc;
      const int col = wn * 32 + j * 8 + fr * 2;
      Cs[col * CLD + row] = acc[i][j][0];
      Cs[(col + 1) * CLD + row] = acc[i][j][1];
    }
  __syncthreads();
  if constexpr (MODE == OUT_ROWPAIR) {
    for (int idx = tid; idx < (DM_T / 2) * DM_T; idx += 128) {
      const int rp = idx % (DM_T / 2), col = idx / (DM_T / 2);
      epi_store<double, CDT, MODE>(g.e, (m0 >> 1) + rp, n0 + col, Cs[col * CLD + 2 * rp], Cs[col * CLD + 2 * rp + 1]);
    }
  } else if constexpr (MODE == OUT_COLPAIR) {
    for (int idx = tid; idx < DM_T * (DM_T / 2); idx += 128) {
      const int row = idx % DM_T, cp = idx / DM_T;
      epi_store<double, CDT, MODE>(g.e, m0 + row, (n0 >> 1) + cp, Cs[2 * cp * CLD + row], Cs[(2 * cp + 1) * CLD + row]);
    }
  } else {
    for (int idx = tid; idx < DM_T * DM_T; idx += 128) {
      const int row = idx % DM_T, col = idx / DM_T;
      epi_store<double, CDT, MODE>(g.e, m0 + row, n0 + col, Cs[col * CLD + row], 0.0);
    }
  }
}

// C := beta * C (k == 0 or alpha == 0: A and B are not read).
template <int CDT>
__global__ void scale_c_kernel(EpiArgs e) {
  const int64_t total = e.m * e.n;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx % e.m, j = idx / e.m;
    if constexpr (CStore<CDT>::cplx) {
      epi_store<double, CDT, OUT_ROWPAIR>(e, i, j, 0.0, 0.0);
    } else {
      epi_store<double, CDT, OUT_REAL>(e, i, j, 0.0, 0.0);
    }
  }
}

template <typename T, int CDT>
cudaError_t launch_simt_mode(int mode, const GemmArgs& g, cudaStream_t s, dim3 grid) {
  switch (mode) {
    case OUT_REAL: simt_gemm<T, CDT, OUT_REAL><<<grid, 256, 0, s>>>(g); break;
    case OUT_RE_ONLY: simt_gemm<T, CDT, OUT_RE_ONLY><<<grid, 256, 0, s>>>(g); break;
    case OUT_ROWPAIR: simt_gemm<T, CDT, OUT_ROWPAIR><<<grid, 256, 0, s>>>(g); break;
    case OUT_COLPAIR: simt_gemm<T, CDT, OUT_COLPAIR><<<grid, 256, 0, s>>>(g); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int CDT>
cudaError_t launch_dmma_mode(int mode, const GemmArgs& g, cudaStream_t s, dim3 grid) {
  switch (mode) {
    case OUT_REAL: dmma_gemm<CDT, OUT_REAL><<<grid, 128, 0, s>>>(g); break;
    case OUT_RE_ONLY: dmma_gemm<CDT, OUT_RE_ONLY><<<grid, 128, 0, s>>>(g); break;
    case OUT_ROWPAIR: dmma_gemm<CDT, OUT_ROWPAIR><<<grid, 128, 0, s>>>(g); break;
    case OUT_COLPAIR: dmma_gemm<CDT, OUT_COLPAIR><<<grid, 128, 0, s>>>(g); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int CDT>
cudaError_t launch_for_c(int method, int mode, const GemmArgs& g, cudaStream_t s) {
  const TileCfg t = tile_cfg(method);
  const int64_t gx = g.Mp / t.tm, gy = g.Np / t.tn;
  if (gx <= 0 || gy <= 0) return cudaSuccess;
  if (gx > 0x7fffffffLL || gy > 65535) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  // Real C only takes OUT_REAL; complex C never does.
  if (!CStore<CDT>::cplx && mode != OUT_REAL) return cudaErrorInvalidValue;
  if (CStore<CDT>::cplx && mode == OUT_REAL) return cudaErrorInvalidValue;
  switch (method) {
    case MXG_METHOD_FFMA: return launch_simt_mode<float, CDT>(mode, g, s, grid);
    case MXG_METHOD_DFMA: return launch_simt_mode<double, CDT>(mode, g, s, grid);
    case MXG_METHOD_DMMA: return launch_dmma_mode<CDT>(mode, g, s, grid);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

TileCfg tile_cfg(int method) {
  switch (method) {
    case MXG_METHOD_FFMA: return {128, 128, 8};
    case MXG_METHOD_DFMA: return {64, 64, 8};
    case MXG_METHOD_DMMA: return {DM_T, DM_T, DM_TK};
    case MXG_METHOD_TF32X3: return {128, 128, 32};
    case MXG_METHOD_BF16X3: return {128, 128, 64};
  }
  return {128, 128, 8};
}

cudaError_t launch_gemm_simt(int method, int c_dt, int mode, const GemmArgs& g, cudaStream_t s) {
  switch (c_dt) {
    case MXG_S: return launch_for_c<MXG_S>(method, mode, g, s);
    case MXG_D: return launch_for_c<MXG_D>(method, mode, g, s);
    case MXG_C: return launch_for_c<MXG_C>(method, mode, g, s);
    case MXG_Z: return launch_for_c<MXG_Z>(method, mode, g, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_scale_c(const EpiArgs& e, int c_dt, cudaStream_t s) {
  const int64_t total = e.m * e.n;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  switch (c_dt) {
    case MXG_S: scale_c_kernel<MXG_S><<<static_cast<unsigned>(blocks), 256, 0, s>>>(e); break;
    case MXG_D: scale_c_kernel<MXG_D><<<static_cast<unsigned>(blocks), 256, 0, s>>>(e); break;
    case MXG_C: scale_c_kernel<MXG_C><<<static_cast<unsigned>(blocks), 256, 0, s>>>(e); break;
    case MXG_Z: scale_c_kernel<MXG_Z><<<static_cast<unsigned>(blocks), 256, 0, s>>>(e); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mxg
