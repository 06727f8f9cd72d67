// FP64 tensor-core contraction (mma.sync.aligned.m8n8k4 .f64) with the fused
// epilogue: the real gemm P = A' B' over the packed operands, accumulated over the
// whole K' in FP64 (Sec. 6.3), then alpha / beta / store. On GB300 the FP64 mma runs
// on the FP64 pipe (the same pipe as DFMA), so this kernel is bound by that pipe.
#include "epilogue.cuh"
#include "grouped.h"

namespace mxg {
namespace {

// ---------------------------------------------------------------- FP64 tensor core
// 128 threads = 2 x 2 warps, each warp a 32 x 32 sub-tile of 4 x 4 mma blocks. Shared
// rows are padded to 68 doubles so the fragment loads (4 k-rows x 8 m-columns per half
// warp) hit 16 distinct 8-byte banks. The accumulator tile is staged through shared
// memory for the epilogue, which then pairs rows or columns for the complex layouts.
constexpr int DM_T = 64, DM_TK = 16, DM_LD = DM_T + 4, DM_CLD = DM_T + 1;
constexpr int DM_SMEM = 2 * 2 * DM_TK * DM_LD;   // doubles
static_assert(DM_T * DM_CLD <= DM_SMEM, "staging tile must fit");

__device__ __forceinline__ void dmma_mainloop(const double* __restrict__ A, const double* __restrict__ B,
                                              int64_t lda, int64_t ldb, int64_t Kp, int64_t m0, int64_t n0,
                                              double* smem, double (&acc)[4][4][2]) {
  double* As = smem;                       // [2][TK][LD]
  double* Bs = smem + 2 * DM_TK * DM_LD;   // [2][TK][LD]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  double2 ra[4], rb[4];
  auto gload = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + r * 128, row = idx >> 5, col = (idx & 31) * 2;
      ra[r] = __ldg(reinterpret_cast<const double2*>(A + (k0 + row) * lda + m0 + col));
      rb[r] = __ldg(reinterpret_cast<const double2*>(B + (k0 + row) * ldb + n0 + col));
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
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  const int fr = lane & 3, fc = lane >> 2;
  const int64_t nk = Kp / DM_TK;
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
}

// Stage the 64 x 64 accumulator tile as Cs[col][row] (row contiguous); ends synced.
__device__ __forceinline__ void dmma_stage(double* smem, const double (&acc)[4][4][2]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1, fr = lane & 3, fc = lane >> 2;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = wm * 32 + i * 8 + fc;
      const int col = wn * 32 + j * 8 + fr * 2;
      smem[col * DM_CLD + row] = acc[i][j][0];
      smem[(col + 1) * DM_CLD + row] = acc[i][j][1];
    }
  __syncthreads();
}

// Each thread updates elements tid, tid + 128, ... of the tile's output grid, eight at
// a time: the eight C loads first, then the updates.
template <int CDT, int MODE>
__device__ __forceinline__ void dmma_epilogue(const EpiArgs& e, int64_t m0, int64_t n0, const double* Cs) {
  constexpr int NOUT = (MODE == OUT_ROWPAIR || MODE == OUT_COLPAIR) ? DM_T * DM_T / 2 : DM_T * DM_T;
  constexpr int B = 8;
  static_assert(NOUT % (128 * B) == 0, "whole batches per thread");
  const EpiScalars<double, CDT> sc = epi_scalars<double, CDT>(e);
  auto where = [&](int idx, int64_t* i, int64_t* j, int* o_r, int* o_i) {
    if constexpr (MODE == OUT_ROWPAIR) {
      const int rp = idx % (DM_T / 2), col = idx / (DM_T / 2);
      *i = (m0 >> 1) + rp; *j = n0 + col; *o_r = col * DM_CLD + 2 * rp; *o_i = *o_r + 1;
    } else if constexpr (MODE == OUT_COLPAIR) {
      const int row = idx % DM_T, cp = idx / DM_T;
      *i = m0 + row; *j = (n0 >> 1) + cp; *o_r = 2 * cp * DM_CLD + row; *o_i = *o_r + DM_CLD;
    } else {
      const int row = idx % DM_T, col = idx / DM_T;
      *i = m0 + row; *j = n0 + col; *o_r = col * DM_CLD + row; *o_i = -1;
    }
  };
  for (int base = threadIdx.x; base < NOUT; base += 128 * B) {
    COld<CDT> old[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      int64_t i, j;
      int o_r, o_i;
      where(base + 128 * u, &i, &j, &o_r, &o_i);
      old[u] = epi_load<CDT>(e, i, j);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      int64_t i, j;
      int o_r, o_i;
      where(base + 128 * u, &i, &j, &o_r, &o_i);
      epi_update<double, CDT, MODE>(e, sc, i, j, Cs[o_r], o_i >= 0 ? Cs[o_i] : 0.0, old[u]);
    }
  }
}

__device__ __forceinline__ void dmma_epilogue_rt(int cdt, int mode, const EpiArgs& e, int64_t m0, int64_t n0,
                                                 const double* Cs) {
  with_c_mode(cdt, mode, [&](auto C, auto M) { dmma_epilogue<decltype(C)::value, decltype(M)::value>(e, m0, n0, Cs); });
}

// Blocks are numbered in launch order (x fastest) and mapped to tiles in groups of
// DM_GM tile rows, columns of the group next: the blocks resident at one time then
// cover a few tile rows and a few tile columns, whose packed panels they share in L2.
constexpr int DM_GM = 16;

template <int CDT, int MODE>
__global__ void __launch_bounds__(128) dmma_gemm(GemmArgs g) {
  __shared__ __align__(16) double smem[DM_SMEM];
  double acc[4][4][2];
  const int64_t tiles_m = gridDim.x, tiles_n = gridDim.y;
  const int64_t bid = static_cast<int64_t>(blockIdx.y) * tiles_m + blockIdx.x;
  const int64_t per_group = DM_GM * tiles_n;
  const int64_t gm0 = (bid / per_group) * DM_GM, r = bid % per_group;
  const int64_t gsz = (tiles_m - gm0 < DM_GM) ? tiles_m - gm0 : DM_GM;
  const int64_t m0 = (gm0 + r % gsz) * DM_T, n0 = (r / gsz) * DM_T;
  dmma_mainloop(static_cast<const double*>(g.A), static_cast<const double*>(g.B), g.lda, g.ldb, g.Kp, m0, n0, smem, acc);
  dmma_stage(smem, acc);
  dmma_epilogue<CDT, MODE>(g.e, m0, n0, smem);
}

__global__ void __launch_bounds__(128)
dmma_gemm_grouped(const GroupProb* __restrict__ probs, const GroupTile* __restrict__ tiles, int ntiles,
                  int* counter, int sched) {
  __shared__ __align__(16) double smem[DM_SMEM];
  __shared__ int slot;
  double acc[4][4][2];
  for (int t = next_tile(counter, &slot, -1, sched); t < ntiles; t = next_tile(counter, &slot, t, sched)) {
    const GroupTile tl = tiles[t];
    const GroupProb& p = probs[tl.prob];
    const int64_t m0 = static_cast<int64_t>(tl.tm) * DM_T, n0 = static_cast<int64_t>(tl.tn) * DM_T;
    __syncthreads();
    dmma_mainloop(static_cast<const double*>(p.A), static_cast<const double*>(p.B), p.lda, p.ldb, p.Kp, m0, n0,
                  smem, acc);
    dmma_stage(smem, acc);
    dmma_epilogue_rt(p.cdt, p.mode, p.e, m0, n0, smem);
  }
}

// Split-K slice: k-tiles [z*kslice, ...) of one tile; raw sums to ws[z] (column-major,
// leading dimension Mp), written through the shared staging tile so stores coalesce.
__global__ void __launch_bounds__(128) dmma_gemm_partial(GemmArgs g, int64_t kslice, double* __restrict__ ws) {
  __shared__ __align__(16) double smem[DM_SMEM];
  double acc[4][4][2];
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * DM_T, n0 = static_cast<int64_t>(blockIdx.y) * DM_T;
  const int64_t k0 = static_cast<int64_t>(blockIdx.z) * kslice;
  const int64_t klen = (g.Kp - k0 < kslice) ? g.Kp - k0 : kslice;
  dmma_mainloop(static_cast<const double*>(g.A) + k0 * g.lda, static_cast<const double*>(g.B) + k0 * g.ldb, g.lda,
                g.ldb, klen, m0, n0, smem, acc);
  dmma_stage(smem, acc);
  double* out = ws + static_cast<int64_t>(blockIdx.z) * g.Mp * g.Np;
  for (int idx = threadIdx.x; idx < DM_T * DM_T; idx += 128) {
    const int row = idx % DM_T, col = idx / DM_T;
    out[(n0 + col) * g.Mp + m0 + row] = smem[col * DM_CLD + row];
  }
}

}  // namespace

cudaError_t launch_dmma_partial(const GemmArgs& g, int64_t kslice, double* ws, dim3 grid, cudaStream_t s) {
  dmma_gemm_partial<<<grid, 128, 0, s>>>(g, kslice, ws);
  return cudaGetLastError();
}

cudaError_t launch_dmma(int mode, int cdt, const GemmArgs& g, cudaStream_t s, dim3 grid) {
  const bool ok = with_c_mode(cdt, mode, [&](auto C, auto M) {
    dmma_gemm<decltype(C)::value, decltype(M)::value><<<grid, 128, 0, s>>>(g);
  });
  return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

cudaError_t launch_dmma_grouped(const GroupProb* probs, const GroupTile* tiles, int ntiles, int* counter, int sched,
                                int grid, cudaStream_t s) {
  dmma_gemm_grouped<<<grid, 128, 0, s>>>(probs, tiles, ntiles, counter, sched);
  return cudaGetLastError();
}

int dmma_grouped_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dmma_gemm_grouped, 128, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

}  // namespace mxg
