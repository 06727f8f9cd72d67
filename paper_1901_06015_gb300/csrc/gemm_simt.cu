// Plain contraction kernels with the fused epilogue: the real gemm P = A' B' over the
// packed operands (M' x N' x K' from the domain case, Fig. "mixeddom"), accumulated
// over the whole K' in the computation precision (Sec. 6.3: one cast per element of
// C, no intermediate round-off in C's precision), then alpha / beta / store.
//
//  * simt tiles (FFMA for float, DFMA for double): 256 threads as 16 x 16, tile
//    32H x 32H x 8, each thread 2H x 2H outputs, H = elements per vector load
//    (float: H = 4 -> 128 x 128, H = 2 -> 64 x 64, H = 1 -> 32 x 32; double: H = 2 ->
//    64 x 64, H = 1 -> 32 x 32). With H >= 2 a thread's rows are two runs of H at
//    t*H and 16H + t*H; with H = 1 they are the adjacent pair 2t, 2t+1. Either way a
//    thread holds whole row pairs 2i, 2i+1 (and column pairs), which the complex
//    epilogue combines.
//  (The FP64 tensor-core kernel is in gemm_dmma.cu.)
//
// Packed operands are MN-major (element (kk, mm) at kk*ld + mm) and padded with zeros
// (to a multiple of the tile in M/N as far as the tile grid reads, and of the k tile
// in K), so the main loops have no bounds checks. Each output element is accumulated
// by one thread in increasing k, so the result does not depend on the tile shape or
// on which CTA computes the tile.
//
// Each kernel exists as a single-problem launch (C datatype and output mode fixed at
// compile time) and as a grouped persistent launch that walks a device work list of
// (problem, tile) entries from many problems, dispatching the epilogue per tile.
#include <algorithm>

#include "epilogue.cuh"
#include "grouped.h"

namespace mxg {
namespace {

template <typename T, int H> struct VecT;
template <> struct VecT<float, 4> { using V = float4; };
template <> struct VecT<float, 2> { using V = float2; };
template <> struct VecT<float, 1> { using V = float; };
template <> struct VecT<double, 2> { using V = double2; };
template <> struct VecT<double, 1> { using V = double; };

// Offset within the tile of a thread's i-th accumulator row (or column), t = the
// thread's row (column) index in the 16 x 16 thread grid.
template <int H>
__device__ __forceinline__ int frag_off(int t, int i) {
  if constexpr (H == 1) return 2 * t + i;
  else return i < H ? t * H + i : 16 * H + t * H + (i - H);
}

template <typename T, int H>
__device__ __forceinline__ void unpack(const typename VecT<T, H>::V& v, T* o) {
  if constexpr (H == 4) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  else if constexpr (H == 2) { o[0] = v.x; o[1] = v.y; }
  else { o[0] = v; }
}

constexpr int SIMT_STAGES = 4;

// Shared-memory ring of S k-tiles of TK rows of A' and B' (TM = 32H columns each).
template <typename T, int H, int TK = 8, int S = SIMT_STAGES>
struct SimtSmem {
  static constexpr int TM = 32 * H;
  __align__(16) T As[S][TK][TM];
  __align__(16) T Bs[S][TK][TM];
};
// The single-problem 128 x 128 FFMA kernel takes k-tiles of 16 rows in a 3-stage ring
// (48 KB): half the barriers of 8-row k-tiles. Every other kernel: 8 rows, 4 stages.
template <typename T, int H> struct PlainTile {
  static constexpr bool big = (sizeof(T) == 4 && H == 4);
  static constexpr int TK = big ? 16 : 8, S = big ? 3 : SIMT_STAGES;
};

// Asynchronous global -> shared copy of one vector of BYTES (16, 8 or 4) bytes; both
// addresses must be BYTES-aligned.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  static_assert(BYTES == 16 || BYTES == 8 || BYTES == 4, "cp.async sizes");
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  else if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Main loop of one 32H x 32H tile at (m0, n0); leaves the accumulators in acc. The
// packed k-tiles stream global -> shared with cp.async through an S-deep ring (each
// thread copies TK/8 vectors -- H elements, 16, 8 or 4 bytes -- of A' and as many of B'
// per k-tile; each row of a k-tile is TM elements = 32 threads' vectors), so the loads
// for k-tile kt + S - 1 are in flight while k-tile kt is computed.
// ncols: columns of the tile inside the real product (the rest is padding). With H = 1
// warp w owns tile columns 4w .. 4w+3 (threads 32w .. 32w+31 have tn = 2w, 2w+1), so a
// warp whose columns all lie in the padding skips its FMAs: those outputs are never
// stored, and it still takes part in the copies and barriers.
template <typename T, int H, int TK, int S>
__device__ __forceinline__ void simt_mainloop(const T* __restrict__ A, const T* __restrict__ B, int64_t lda,
                                              int64_t ldb, int64_t Kp, int64_t m0, int64_t n0,
                                              SimtSmem<T, H, TK, S>& sm, T (&acc)[2 * H][2 * H],
                                              int64_t ncols = 32 * H) {
  using V = typename VecT<T, H>::V;
  constexpr int TM = 32 * H, R = 2 * H;
  constexpr int CP = TK / 8;                          // rows each thread copies per operand and k-tile
  static_assert(TK % 8 == 0, "k-tile rows: 8 per 256 threads");
  constexpr int VB = static_cast<int>(sizeof(V));   // bytes per copied vector
  const int tid = threadIdx.x;
  const int lrow = tid / (TM / H), lcol = (tid % (TM / H)) * H;
  const T* Ag = A + lrow * lda + m0 + lcol;
  const T* Bg = B + lrow * ldb + n0 + lcol;
  const int64_t nk = Kp / TK;
  // prologue: k-tiles 0 .. S-2
#pragma unroll
  for (int st = 0; st < S - 1; ++st) {
    if (st < nk) {
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        cp_async<VB>(&sm.As[st][lrow + 8 * c][lcol], Ag + (st * TK + 8 * c) * lda);
        cp_async<VB>(&sm.Bs[st][lrow + 8 * c][lcol], Bg + (st * TK + 8 * c) * ldb);
      }
    }
    cp_async_commit();
  }
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = T(0);
  const int tm = tid & 15, tn = tid >> 4;
  // the next k-tile's source rows and the ring positions advance incrementally (no
  // per-k-tile multiplications or modulo)
  const T* Agn = Ag + static_cast<int64_t>(S - 1) * TK * lda;
  const T* Bgn = Bg + static_cast<int64_t>(S - 1) * TK * ldb;
  const int64_t a_step = static_cast<int64_t>(TK) * lda, b_step = static_cast<int64_t>(TK) * ldb;
  const int64_t lda8 = 8 * lda, ldb8 = 8 * ldb;
  int st_w = S - 1, st_r = 0;
  for (int64_t kt = 0; kt < nk; ++kt) {
    cp_async_wait<S - 2>();      // k-tile kt has landed (for this thread) ...
    __syncthreads();             // ... and for every thread; stage (kt-1) % S is free
    if (kt + S - 1 < nk) {
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        cp_async<VB>(&sm.As[st_w][lrow + 8 * c][lcol], Agn + c * lda8);
        cp_async<VB>(&sm.Bs[st_w][lrow + 8 * c][lcol], Bgn + c * ldb8);
      }
    }
    cp_async_commit();
    Agn += a_step;
    Bgn += b_step;
    const int buf = st_r;
    st_w = (st_w + 1 == S) ? 0 : st_w + 1;
    st_r = (st_r + 1 == S) ? 0 : st_r + 1;
    if (H == 1 && 4 * static_cast<int64_t>(tid >> 5) >= ncols) continue;   // whole warp in the padding
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T a[R], b[R];
      if constexpr (H == 1) {
        unpack<T, 2>(*reinterpret_cast<const typename VecT<T, 2>::V*>(&sm.As[buf][kk][2 * tm]), a);
        unpack<T, 2>(*reinterpret_cast<const typename VecT<T, 2>::V*>(&sm.Bs[buf][kk][2 * tn]), b);
      } else {
        unpack<T, H>(*reinterpret_cast<const V*>(&sm.As[buf][kk][tm * H]), a);
        unpack<T, H>(*reinterpret_cast<const V*>(&sm.As[buf][kk][TM / 2 + tm * H]), a + H);
        unpack<T, H>(*reinterpret_cast<const V*>(&sm.Bs[buf][kk][tn * H]), b);
        unpack<T, H>(*reinterpret_cast<const V*>(&sm.Bs[buf][kk][TM / 2 + tn * H]), b + H);
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  cp_async_wait<0>();
}

// TW: threads per side of the tile's thread grid (16 x 16 threads; 8 x 8 for the 16 x 16
// DFMA tiles).
template <typename T, int H, int CDT, int MODE, int TW = 16>
__device__ __forceinline__ void simt_epilogue(const EpiArgs& e, int64_t m0, int64_t n0, const T (&acc)[2 * H][2 * H]) {
  constexpr int R = 2 * H;
  constexpr int EB = (H == 1) ? 2 : H;   // C elements loaded together
  const EpiScalars<T, CDT> sc = epi_scalars<T, CDT>(e);
  const int tm = threadIdx.x % TW, tn = threadIdx.x / TW;
  auto row_of = [&](int i) -> int64_t { return m0 + frag_off<H>(tm, i); };
  auto col_of = [&](int j) -> int64_t { return n0 + frag_off<H>(tn, j); };
  // EB elements of one row (or row pair) of the thread's block at a time: their C
  // loads first, then the updates
  if constexpr (MODE == OUT_ROWPAIR) {
#pragma unroll
    for (int i = 0; i < R; i += 2)
#pragma unroll
      for (int j0 = 0; j0 < R; j0 += EB) {
        COld<CDT> old[EB];
#pragma unroll
        for (int j = 0; j < EB; ++j) old[j] = epi_load<CDT>(e, row_of(i) >> 1, col_of(j0 + j));
#pragma unroll
        for (int j = 0; j < EB; ++j)
          epi_update<T, CDT, MODE>(e, sc, row_of(i) >> 1, col_of(j0 + j), acc[i][j0 + j], acc[i + 1][j0 + j], old[j]);
      }
  } else if constexpr (MODE == OUT_COLPAIR) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      COld<CDT> old[H];
#pragma unroll
      for (int j = 0; j < R; j += 2) old[j / 2] = epi_load<CDT>(e, row_of(i), col_of(j) >> 1);
#pragma unroll
      for (int j = 0; j < R; j += 2)
        epi_update<T, CDT, MODE>(e, sc, row_of(i), col_of(j) >> 1, acc[i][j], acc[i][j + 1], old[j / 2]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j0 = 0; j0 < R; j0 += EB) {
        COld<CDT> old[EB];
#pragma unroll
        for (int j = 0; j < EB; ++j) old[j] = epi_load<CDT>(e, row_of(i), col_of(j0 + j));
#pragma unroll
        for (int j = 0; j < EB; ++j)
          epi_update<T, CDT, MODE>(e, sc, row_of(i), col_of(j0 + j), acc[i][j0 + j], T(0), old[j]);
      }
  }
}

// Runtime dispatch over the valid (C datatype, output mode) pairs, once per tile.
template <typename T, int H>
__device__ __forceinline__ void simt_epilogue_rt(int cdt, int mode, const EpiArgs& e, int64_t m0, int64_t n0,
                                                 const T (&acc)[2 * H][2 * H]) {
  with_c_mode(cdt, mode, [&](auto C, auto M) {
    simt_epilogue<T, H, decltype(C)::value, decltype(M)::value>(e, m0, n0, acc);
  });
}

template <typename T, int H, int CDT, int MODE>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 2 : 3)) simt_gemm(GemmArgs g) {
  __shared__ SimtSmem<T, H, PlainTile<T, H>::TK, PlainTile<T, H>::S> sm;
  T acc[2 * H][2 * H];
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * 32 * H, n0 = static_cast<int64_t>(blockIdx.y) * 32 * H;
  const int64_t nreal = g.e.n * (MODE == OUT_COLPAIR ? 2 : 1);   // columns of the real product
  simt_mainloop<T, H>(static_cast<const T*>(g.A), static_cast<const T*>(g.B), g.lda, g.ldb, g.Kp, m0, n0, sm, acc,
                      nreal - n0);
  simt_epilogue<T, H, CDT, MODE>(g.e, m0, n0, acc);
}

// DFMA on 16 x 16 tiles for double-precision calls too small to fill the device with
// 32 x 32 tiles: 64 threads as 8 x 8, each the adjacent row pair 2t, 2t+1 and column
// pair of the 32 x 32 kernel's mapping, k-tiles of 8 rows in a 4-stage cp.async ring
// (one 16-byte copy per thread and operand). A problem gets 4x the CTAs, so 4x the SMs'
// share of the FP64 pipe; each output is accumulated in increasing k as in every other
// DFMA kernel, so the results are the same.
constexpr int D16_TK = 8, D16_S = 4;

struct D16Smem {
  __align__(16) double As[D16_S][D16_TK][16];
  __align__(16) double Bs[D16_S][D16_TK][16];
};

// Main loop of one 16 x 16 tile at (m0, n0); leaves the accumulators in acc.
__device__ __forceinline__ void dfma16_mainloop(const double* __restrict__ A, const double* __restrict__ B,
                                                int64_t lda, int64_t ldb, int64_t Kp, int64_t m0, int64_t n0,
                                                D16Smem& sm, double (&acc)[2][2]) {
  const int tid = threadIdx.x, tm = tid & 7, tn = tid >> 3;
  // copies: row tid / 8 of the k-tile, columns 2 * (tid % 8) .. +1 (one double2)
  const int lrow = tid >> 3, lcol = (tid & 7) * 2;
  const double* Ag = A + lrow * lda + m0 + lcol;
  const double* Bg = B + lrow * ldb + n0 + lcol;
  const int64_t nk = Kp / D16_TK;
  const int64_t a_step = D16_TK * lda, b_step = D16_TK * ldb;
#pragma unroll
  for (int st = 0; st < D16_S - 1; ++st) {
    if (st < nk) {
      cp_async<16>(&sm.As[st][lrow][lcol], Ag + st * a_step);
      cp_async<16>(&sm.Bs[st][lrow][lcol], Bg + st * b_step);
    }
    cp_async_commit();
  }
  acc[0][0] = acc[0][1] = acc[1][0] = acc[1][1] = 0.0;
  const double* Agn = Ag + (D16_S - 1) * a_step;
  const double* Bgn = Bg + (D16_S - 1) * b_step;
  int st_w = D16_S - 1, st_r = 0;
  for (int64_t kt = 0; kt < nk; ++kt) {
    cp_async_wait<D16_S - 2>();
    __syncthreads();
    if (kt + D16_S - 1 < nk) {
      cp_async<16>(&sm.As[st_w][lrow][lcol], Agn);
      cp_async<16>(&sm.Bs[st_w][lrow][lcol], Bgn);
    }
    cp_async_commit();
    Agn += a_step;
    Bgn += b_step;
    const int buf = st_r;
    st_w = (st_w + 1 == D16_S) ? 0 : st_w + 1;
    st_r = (st_r + 1 == D16_S) ? 0 : st_r + 1;
#pragma unroll
    for (int kk = 0; kk < D16_TK; ++kk) {
      const double2 x = *reinterpret_cast<const double2*>(&sm.As[buf][kk][2 * tm]);
      const double2 y = *reinterpret_cast<const double2*>(&sm.Bs[buf][kk][2 * tn]);
      acc[0][0] = fma(x.x, y.x, acc[0][0]);
      acc[0][1] = fma(x.x, y.y, acc[0][1]);
      acc[1][0] = fma(x.y, y.x, acc[1][0]);
      acc[1][1] = fma(x.y, y.y, acc[1][1]);
    }
  }
  cp_async_wait<0>();
}

template <int CDT, int MODE>
__global__ void __launch_bounds__(64) dfma16_gemm(GemmArgs g) {
  __shared__ D16Smem sm;
  double acc[2][2];
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * 16, n0 = static_cast<int64_t>(blockIdx.y) * 16;
  dfma16_mainloop(static_cast<const double*>(g.A), static_cast<const double*>(g.B), g.lda, g.ldb, g.Kp, m0, n0, sm,
                  acc);
  simt_epilogue<double, 1, CDT, MODE, 8>(g.e, m0, n0, acc);
}

// Grouped form: a persistent launch over a (problem, 16 x 16 tile) work list.
__global__ void __launch_bounds__(64)
dfma16_gemm_grouped(const GroupProb* __restrict__ probs, const GroupTile* __restrict__ tiles, int ntiles,
                    int* counter, int sched) {
  __shared__ D16Smem sm;
  __shared__ int slot;
  double acc[2][2];
  for (int t = next_tile(counter, &slot, -1, sched); t < ntiles; t = next_tile(counter, &slot, t, sched)) {
    const GroupTile tl = tiles[t];
    const GroupProb& p = probs[tl.prob];
    const int64_t m0 = static_cast<int64_t>(tl.tm) * 16, n0 = static_cast<int64_t>(tl.tn) * 16;
    __syncthreads();   // the previous tile's shared-memory reads are done
    dfma16_mainloop(static_cast<const double*>(p.A), static_cast<const double*>(p.B), p.lda, p.ldb, p.Kp, m0, n0,
                    sm, acc);
    with_c_mode(p.cdt, p.mode, [&](auto C, auto M) {
      simt_epilogue<double, 1, decltype(C)::value, decltype(M)::value, 8>(p.e, m0, n0, acc);
    });
  }
}

template <typename T, int H>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 2 : 3))
simt_gemm_grouped(const GroupProb* __restrict__ probs, const GroupTile* __restrict__ tiles, int ntiles,
                  int* counter, int sched) {
  __shared__ SimtSmem<T, H> sm;
  __shared__ int slot;
  T acc[2 * H][2 * H];
  for (int t = next_tile(counter, &slot, -1, sched); t < ntiles; t = next_tile(counter, &slot, t, sched)) {
    const GroupTile tl = tiles[t];
    const GroupProb& p = probs[tl.prob];
    const int64_t m0 = static_cast<int64_t>(tl.tm) * 32 * H, n0 = static_cast<int64_t>(tl.tn) * 32 * H;
    __syncthreads();   // the previous tile's shared-memory reads are done
    const int64_t nreal = p.e.n * (p.mode == OUT_COLPAIR ? 2 : 1);   // columns of the real product
    simt_mainloop<T, H>(static_cast<const T*>(p.A), static_cast<const T*>(p.B), p.lda, p.ldb, p.Kp, m0, n0, sm, acc,
                        nreal - n0);
    simt_epilogue_rt<T, H>(p.cdt, p.mode, p.e, m0, n0, acc);
  }
}

// Split-K (the paper's C_temp in the computation precision, Secs. 6.2-6.4, here for
// parallelism over K): slice z = blockIdx.z accumulates k-tiles [z*kslice, ...) of one
// tile and stores the raw sums to ws[z] (column-major, leading dimension Mp); a
// reduction then adds the slices in order and applies the epilogue once.
template <typename T, int H>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 2 : 3))
simt_gemm_partial(GemmArgs g, int64_t kslice, T* __restrict__ ws) {
  __shared__ SimtSmem<T, H> sm;
  T acc[2 * H][2 * H];
  constexpr int TM = 32 * H;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * TM, n0 = static_cast<int64_t>(blockIdx.y) * TM;
  const int64_t k0 = static_cast<int64_t>(blockIdx.z) * kslice;
  const int64_t klen = (g.Kp - k0 < kslice) ? g.Kp - k0 : kslice;
  simt_mainloop<T, H>(static_cast<const T*>(g.A) + k0 * g.lda, static_cast<const T*>(g.B) + k0 * g.ldb, g.lda, g.ldb,
                      klen, m0, n0, sm, acc);
  T* out = ws + static_cast<int64_t>(blockIdx.z) * g.Mp * g.Np;
  const int tm = threadIdx.x & 15, tn = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 2 * H; ++i)
#pragma unroll
    for (int j = 0; j < 2 * H; ++j) {
      const int64_t row = m0 + frag_off<H>(tm, i);
      const int64_t col = n0 + frag_off<H>(tn, j);
      out[col * g.Mp + row] = acc[i][j];
    }
}

template <typename T, int CDT, int MODE>
__global__ void splitk_reduce(const T* __restrict__ ws, int splits, int64_t Mp, int64_t Np, EpiArgs e) {
  const int64_t total = e.m * e.n, slice = Mp * Np;
  const EpiScalars<T, CDT> sc = epi_scalars<T, CDT>(e);
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx % e.m, j = idx / e.m;
    int64_t o_r, o_i = -1;   // offsets of the real and (paired) imaginary values of P
    if constexpr (MODE == OUT_ROWPAIR) { o_r = j * Mp + 2 * i; o_i = o_r + 1; }
    else if constexpr (MODE == OUT_COLPAIR) { o_r = 2 * j * Mp + i; o_i = o_r + Mp; }
    else { o_r = j * Mp + i; }
    T pr = ws[o_r], pi = (o_i >= 0) ? ws[o_i] : T(0);
    for (int z = 1; z < splits; ++z) {
      pr = add_rn(pr, ws[z * slice + o_r]);
      if (o_i >= 0) pi = add_rn(pi, ws[z * slice + o_i]);
    }
    epi_store<T, CDT, MODE>(e, sc, i, j, pr, pi);
  }
}

// C := beta * C (k == 0 or alpha == 0: A and B are not read). Block (bx, by) walks
// columns by, by + gridDim.y, ... and in each the rows 256*bx + t + 256*gridDim.x*u
// (lanes along the rows, which are unit-stride after the whole-operation transpose),
// four elements per thread at a time with their loads in flight together.
template <int CDT>
__global__ void __launch_bounds__(256) scale_c_kernel(EpiArgs e) {
  constexpr int MODE = CStore<CDT>::cplx ? OUT_ROWPAIR : OUT_REAL;
  constexpr int U = 4;
  const int64_t rstep = static_cast<int64_t>(gridDim.x) * 256;
  const EpiScalars<double, CDT> sc = epi_scalars<double, CDT>(e);
  for (int64_t j = blockIdx.y; j < e.n; j += gridDim.y) {
    for (int64_t i0 = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x; i0 < e.m; i0 += U * rstep) {
      COld<CDT> old[U];
#pragma unroll
      for (int u = 0; u < U; ++u) old[u] = epi_load<CDT>(e, i0 + u * rstep, j);
#pragma unroll
      for (int u = 0; u < U; ++u) epi_update<double, CDT, MODE>(e, sc, i0 + u * rstep, j, 0.0, 0.0, old[u]);
    }
  }
}

}  // namespace

TileCfg tile_cfg(int method) {
  switch (method) {
    case MXG_METHOD_FFMA: return {128, 128, 16};
    case MXG_METHOD_DFMA: return {64, 64, 8};
    case MXG_METHOD_DMMA: return {64, 64, 16};
    case MXG_METHOD_TF32X3: return {128, 256, 32};   // tcgen05 tiles, k padded to 128 bytes
    case MXG_METHOD_BF16X3: return {128, 256, 64};
    case MXG_METHOD_TC16: return {128, 256, 64};
  }
  return {128, 128, 8};
}

int variant_tile(int variant) {
  switch (variant) {
    case VAR_FFMA_128: return 128;
    case VAR_FFMA_64: return 64;
    case VAR_DFMA_64: return 64;
    case VAR_DMMA_64: return 64;
    case VAR_DFMA_32: return 32;
    case VAR_FFMA_32: return 32;
    case VAR_DFMA_16: return 16;
  }
  return 0;
}

cudaError_t launch_gemm_simt(int method, int c_dt, int mode, const GemmArgs& g, cudaStream_t s) {
  const TileCfg t = tile_cfg(method);
  int64_t gx = g.Mp / t.tm, gy = g.Np / t.tn;
  if (gx <= 0 || gy <= 0) return cudaSuccess;
  // FFMA problems with fewer 128 x 128 tiles than half the SMs run 32 x 32 tiles instead
  // (inside the same 128-padded packs): a small call spreads over up to 16x the CTAs,
  // with the same per-element accumulation order, so the same results
  const bool ffma_small = (method == MXG_METHOD_FFMA) && (gx * gy < 76);
  bool dfma16 = false;
  if (method == MXG_METHOD_DFMA || ffma_small) {
    // DFMA runs 32 x 32 tiles over the real product's extent inside the 64-padded packs:
    // the FP64 pipe is busy with a few warps per SM, so smaller tiles only cut padding
    const int64_t mr = g.e.m * (mode == OUT_ROWPAIR ? 2 : 1), nr = g.e.n * (mode == OUT_COLPAIR ? 2 : 1);
    gx = (mr + 31) / 32;
    gy = (nr + 31) / 32;
    if (gx <= 0 || gy <= 0) return cudaSuccess;
    // and 16 x 16 tiles when 32 x 32 ones would leave more than half the SMs idle
    if (method == MXG_METHOD_DFMA && gx * gy < 76) {
      dfma16 = true;
      gx = (mr + 15) / 16;
      gy = (nr + 15) / 16;
    }
  }
  if (gx > 0x7fffffffLL || gy > 65535) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  if (method == MXG_METHOD_DMMA) return launch_dmma(mode, c_dt, g, s, grid);
  if (method != MXG_METHOD_FFMA && method != MXG_METHOD_DFMA) return cudaErrorInvalidValue;
  const bool ok = with_c_mode(c_dt, mode, [&](auto C, auto M) {
    constexpr int CDT = decltype(C)::value, MODE = decltype(M)::value;
    if (dfma16) dfma16_gemm<CDT, MODE><<<grid, 64, 0, s>>>(g);
    else if (method == MXG_METHOD_FFMA && ffma_small) simt_gemm<float, 1, CDT, MODE><<<grid, 256, 0, s>>>(g);
    else if (method == MXG_METHOD_FFMA) simt_gemm<float, 4, CDT, MODE><<<grid, 256, 0, s>>>(g);
    else simt_gemm<double, 1, CDT, MODE><<<grid, 256, 0, s>>>(g);
  });
  return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_reduce(int c_dt, int mode, const T* ws, int splits, int64_t Mp, int64_t Np, const EpiArgs& e,
                                 cudaStream_t s) {
  const int64_t total = e.m * e.n;
  if (total <= 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 152 * 16));
  const bool ok = with_c_mode(c_dt, mode, [&](auto C, auto M) {
    splitk_reduce<T, decltype(C)::value, decltype(M)::value><<<blocks, 256, 0, s>>>(ws, splits, Mp, Np, e);
  });
  return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

cudaError_t launch_gemm_splitk(int method, int c_dt, int mode, const GemmArgs& g, int splits, int64_t kslice,
                               void* ws, cudaStream_t s) {
  const TileCfg t = tile_cfg(method);
  const int64_t gx = g.Mp / t.tm, gy = g.Np / t.tn;
  if (gx <= 0 || gy <= 0) return cudaSuccess;
  if (gx > 0x7fffffffLL || gy > 65535 || splits < 1 || splits > 65535) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy), static_cast<unsigned>(splits));
  cudaError_t e;
  switch (method) {
    case MXG_METHOD_FFMA:
      simt_gemm_partial<float, 4><<<grid, 256, 0, s>>>(g, kslice, static_cast<float*>(ws));
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      return launch_reduce<float>(c_dt, mode, static_cast<const float*>(ws), splits, g.Mp, g.Np, g.e, s);
    case MXG_METHOD_DFMA:
      simt_gemm_partial<double, 2><<<grid, 256, 0, s>>>(g, kslice, static_cast<double*>(ws));
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      return launch_reduce<double>(c_dt, mode, static_cast<const double*>(ws), splits, g.Mp, g.Np, g.e, s);
    case MXG_METHOD_DMMA:
      if ((e = launch_dmma_partial(g, kslice, static_cast<double*>(ws), grid, s)) != cudaSuccess) return e;
      return launch_reduce<double>(c_dt, mode, static_cast<const double*>(ws), splits, g.Mp, g.Np, g.e, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_gemm_grouped(int variant, const GroupProb* probs, const GroupTile* tiles, int ntiles,
                                int* counter, int sched, int grid, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (grid <= 0) return cudaErrorInvalidValue;
  switch (variant) {
    case VAR_FFMA_128: simt_gemm_grouped<float, 4><<<grid, 256, 0, s>>>(probs, tiles, ntiles, counter, sched); break;
    case VAR_FFMA_64: simt_gemm_grouped<float, 2><<<grid, 256, 0, s>>>(probs, tiles, ntiles, counter, sched); break;
    case VAR_DFMA_64: simt_gemm_grouped<double, 2><<<grid, 256, 0, s>>>(probs, tiles, ntiles, counter, sched); break;
    case VAR_DFMA_32: simt_gemm_grouped<double, 1><<<grid, 256, 0, s>>>(probs, tiles, ntiles, counter, sched); break;
    case VAR_FFMA_32: simt_gemm_grouped<float, 1><<<grid, 256, 0, s>>>(probs, tiles, ntiles, counter, sched); break;
    case VAR_DMMA_64: return launch_dmma_grouped(probs, tiles, ntiles, counter, sched, grid, s);
    case VAR_DFMA_16: dfma16_gemm_grouped<<<grid, 64, 0, s>>>(probs, tiles, ntiles, counter, sched); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int grouped_blocks_per_sm(int variant) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (variant) {
    case VAR_FFMA_128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_gemm_grouped<float, 4>, 256, 0); break;
    case VAR_FFMA_64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_gemm_grouped<float, 2>, 256, 0); break;
    case VAR_DFMA_64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_gemm_grouped<double, 2>, 256, 0); break;
    case VAR_DFMA_32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_gemm_grouped<double, 1>, 256, 0); break;
    case VAR_FFMA_32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_gemm_grouped<float, 1>, 256, 0); break;
    case VAR_DMMA_64: return dmma_grouped_blocks_per_sm();
    case VAR_DFMA_16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dfma16_gemm_grouped, 64, 0); break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_scale_c(const EpiArgs& e, int c_dt, cudaStream_t s) {
  if (e.m <= 0 || e.n <= 0) return cudaSuccess;
  // about 16 blocks of 256 threads per SM in total: rows split into at most 8 row
  // blocks of 4 x 256 rows per pass, columns over the rest
  const int64_t gx = std::min<int64_t>((e.m + 1023) / 1024, 8);
  const int64_t gy = std::min<int64_t>(e.n, std::max<int64_t>(1, (152 * 16) / gx));
  const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  const int mode = (c_dt == MXG_C || c_dt == MXG_Z || c_dt == MXG_K || c_dt == MXG_W) ? OUT_ROWPAIR : OUT_REAL;
  const bool ok = with_c_mode(c_dt, mode, [&](auto C, auto) {
    scale_c_kernel<decltype(C)::value><<<grid, 256, 0, s>>>(e);
  });
  return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

}  // namespace mxg
