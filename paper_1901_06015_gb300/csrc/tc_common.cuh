// Device helpers shared by the tcgen05 contraction kernels (sm_103a): bounded mbarrier
// waits, TMA tile loads, shared-memory and instruction descriptors, TMEM loads, and the
// 32-column epilogue chunk that pairs rows or columns for complex C. Host helpers: the
// tensor-map encoder, 2-D K-major tensor maps, and the SM count of the current device.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "epilogue.cuh"

namespace mxg {
namespace tc {

constexpr unsigned long long kWaitNs = 2000000000ull;      // 2 s per wait
constexpr uint32_t ROWB = 64;                              // bytes of K per tile row (64-byte swizzle)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on the phase of the given parity; false after kWaitNs or when another
// role of the CTA has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > kWaitNs) return false;
    }
  }
}
// Bounded wait that ignores the abort flag (used to drain the CTA's own work).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > kWaitNs) return;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor of a K-major tile written by TMA with the 64-byte
// swizzle: rows of 64 bytes, 8-row swizzle atoms 512 bytes apart (stride byte
// offset), leading byte offset unused for this layout (encoded as 1), descriptor
// version 1, layout type 4 (64-byte swizzle).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3fff);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(512 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(4) << 61;
  return d;
}
// The same for rows of RB bytes (64 or 128) written with the RB-byte swizzle: 8-row
// atoms of 8 * RB bytes, layout type 4 (64-byte) or 2 (128-byte).
template <uint32_t RB>
__device__ __forceinline__ uint64_t swz_desc(uint32_t saddr) {
  static_assert(RB == 64 || RB == 128, "swizzle width");
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3fff);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>((8 * RB) >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(RB == 128 ? 2 : 4) << 61;
  return d;
}
// Instruction descriptor (kind::f16 / kind::tf32): D in FP32, A and B of the given
// format code (1 = BF16 for kind::f16, 2 = TF32 for kind::tf32), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Epilogue of one 32-column chunk of the accumulator (C datatype and mode fixed), in
// two phases: tc_epi_load reads the thread's old C values for the chunk (all loads in
// flight together, overlapping the TMEM read), tc_epi_finish updates and stores them.
// ROWPAIR: rows 2i and 2i+1 (real and imaginary parts) sit in lanes 2l and 2l+1; the
// even lane updates the even columns of the chunk, the odd lane the odd ones. COLPAIR: columns 2j, 2j+1 form one
// complex column.
template <int MODE> struct TcChunk { static constexpr int nold = (MODE == OUT_ROWPAIR || MODE == OUT_COLPAIR) ? 16 : 32; };

// Does the warp's whole chunk lie inside C? Then its loads and stores need no bounds
// test: one address per thread and chunk, and the elements' updates form straight-line
// code (a test and branch per element left the epilogue warps stalled on branch
// resolution: measured at a short k, the fused epilogue moved C at 0.39 of HBM with the
// tests and 0.69 without). Debug builds test every address.
template <int MODE>
__device__ __forceinline__ bool tc_chunk_inside(const EpiArgs& e, int64_t row, int64_t col0) {
  bool in;
  if constexpr (MODE == OUT_ROWPAIR) in = (row >> 1) < e.m && col0 + 32 <= e.n;
  else if constexpr (MODE == OUT_COLPAIR) in = row < e.m && (col0 >> 1) + 16 <= e.n;
  else in = row < e.m && col0 + 32 <= e.n;
#ifdef MXG_DEBUG_BOUNDS
  in = false;
#endif
  return __all_sync(0xffffffffu, in);
}
// A thread's first element of the chunk in C (as tc_old_pos, t = 0) and the distance
// between its consecutive elements, in elements of C's storage type.
template <int CDT, int MODE>
__device__ __forceinline__ typename CStore<CDT>::T* tc_chunk_ptr(const EpiArgs& e, int64_t row, int64_t col0,
                                                                 int lane, int64_t* step) {
  using CT = typename CStore<CDT>::T;
  constexpr int W = CStore<CDT>::cplx ? 2 : 1;
  int64_t i, j;
  if constexpr (MODE == OUT_ROWPAIR) { i = row >> 1; j = col0 + (lane & 1); *step = 2 * e.cs * W; }
  else if constexpr (MODE == OUT_COLPAIR) { i = row; j = col0 >> 1; *step = e.cs * W; }
  else { i = row; j = col0; *step = e.cs * W; }
  return static_cast<CT*>(e.C) + (i * e.rs + j * e.cs) * W;
}

template <int CDT, int MODE>
__device__ __forceinline__ void tc_epi_load(const EpiArgs& e, int64_t row, int64_t col0, int lane,
                                            COld<CDT> (&old)[TcChunk<MODE>::nold]) {
  if (!e.beta_zero && tc_chunk_inside<MODE>(e, row, col0)) {
    int64_t step;
    const typename CStore<CDT>::T* p = tc_chunk_ptr<CDT, MODE>(e, row, col0, lane, &step);
#pragma unroll
    for (int t = 0; t < TcChunk<MODE>::nold; ++t) {
      old[t].re = p[t * step];
      if constexpr (CStore<CDT>::cplx) old[t].im = p[t * step + 1];
      else old[t].im = old[t].re;
    }
    return;
  }
  if constexpr (MODE == OUT_ROWPAIR) {
#pragma unroll
    for (int t = 0; t < 16; ++t) old[t] = epi_load<CDT>(e, row >> 1, col0 + 2 * t + (lane & 1));
  } else if constexpr (MODE == OUT_COLPAIR) {
#pragma unroll
    for (int t = 0; t < 16; ++t) old[t] = epi_load<CDT>(e, row, (col0 >> 1) + t);
  } else {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) old[jj] = epi_load<CDT>(e, row, col0 + jj);
  }
}

template <int CDT, int MODE>
__device__ __forceinline__ void tc_epi_finish(const EpiArgs& e, const EpiScalars<float, CDT>& sc, int64_t row,
                                              int64_t col0, const uint32_t (&v)[32], int lane,
                                              const COld<CDT> (&old)[TcChunk<MODE>::nold]) {
  if (tc_chunk_inside<MODE>(e, row, col0)) {
    int64_t step;
    typename CStore<CDT>::T* p = tc_chunk_ptr<CDT, MODE>(e, row, col0, lane, &step);
    if constexpr (MODE == OUT_ROWPAIR) {
      const bool odd = (lane & 1) != 0;
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const float ve = __uint_as_float(v[2 * t]), vo = __uint_as_float(v[2 * t + 1]);
        const float got = __shfl_xor_sync(0xffffffffu, odd ? ve : vo, 1);
        const float pr = odd ? got : ve, pi = odd ? vo : got;
        const COld<CDT> r = epi_value<float, CDT, MODE>(e, sc, pr, pi, old[t]);
        p[t * step] = r.re;
        p[t * step + 1] = r.im;
      }
    } else if constexpr (MODE == OUT_COLPAIR) {
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const COld<CDT> r =
            epi_value<float, CDT, MODE>(e, sc, __uint_as_float(v[2 * t]), __uint_as_float(v[2 * t + 1]), old[t]);
        p[t * step] = r.re;
        p[t * step + 1] = r.im;
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const COld<CDT> r = epi_value<float, CDT, MODE>(e, sc, __uint_as_float(v[jj]), 0.0f, old[jj]);
        p[jj * step] = r.re;
        if constexpr (CStore<CDT>::cplx) p[jj * step + 1] = r.im;
      }
    }
    return;
  }
  if constexpr (MODE == OUT_ROWPAIR) {
    // per column pair (2t, 2t+1) one exchange: the even lane sends its value of column
    // 2t+1 and receives the odd lane's value of column 2t, so both lanes of the pair
    // update one element (no divergence)
    const bool odd = (lane & 1) != 0;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const float ve = __uint_as_float(v[2 * t]), vo = __uint_as_float(v[2 * t + 1]);
      const float got = __shfl_xor_sync(0xffffffffu, odd ? ve : vo, 1);
      const float pr = odd ? got : ve, pi = odd ? vo : got;
      epi_update<float, CDT, MODE>(e, sc, row >> 1, col0 + 2 * t + (odd ? 1 : 0), pr, pi, old[t]);
    }
  } else if constexpr (MODE == OUT_COLPAIR) {
#pragma unroll
    for (int t = 0; t < 16; ++t)
      epi_update<float, CDT, MODE>(e, sc, row, (col0 >> 1) + t, __uint_as_float(v[2 * t]), __uint_as_float(v[2 * t + 1]),
                                   old[t]);
  } else {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj)
      epi_update<float, CDT, MODE>(e, sc, row, col0 + jj, __uint_as_float(v[jj]), 0.0f, old[jj]);
  }
}

// Position in C of element t of a thread's old values for a chunk (as tc_epi_load).
template <int MODE>
__device__ __forceinline__ void tc_old_pos(int64_t row, int64_t col0, int lane, int t, int64_t* i, int64_t* j) {
  if constexpr (MODE == OUT_ROWPAIR) { *i = row >> 1; *j = col0 + 2 * t + (lane & 1); }
  else if constexpr (MODE == OUT_COLPAIR) { *i = row; *j = (col0 >> 1) + t; }
  else { *i = row; *j = col0 + t; }
}

// Staging of old C values through shared memory: the (C datatype, mode) pairs whose
// element is 8 bytes and whose chunk is at most 128 bytes per thread (complex single C
// with row or column pairs) copy the next chunk's old values with cp.async into a
// per-warp double buffer (2 x 4 KB, element t of lane l at (t * 32 + l) * 8) while the
// current chunk is finished. The copies hold no registers, so the next chunk's loads are
// in flight during the current chunk's work without adding to the kernel's register
// pressure. Measured on GB300 at 8192^2 with a short k: +7-19% C bandwidth for complex
// single C; 4-byte elements (s, and complex 16-bit) were 26-28% slower this way and load
// into registers, as do the rest.
template <int CDT, int MODE> struct TcStage {
  static constexpr int esz = static_cast<int>(sizeof(typename CStore<CDT>::T)) * (CStore<CDT>::cplx ? 2 : 1);
  static constexpr int nold = TcChunk<MODE>::nold;
  static constexpr bool on = (esz == 8) && nold * esz <= 128;
};
constexpr uint32_t TC_STAGE_WARP_BYTES = 2 * 32 * 128;   // two chunk buffers per epilogue warp
constexpr uint32_t TC_STAGE_BYTES = 4 * TC_STAGE_WARP_BYTES;

template <int BYTES>
__device__ __forceinline__ void cp_async_ca(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int CDT, int MODE>
__device__ __forceinline__ void tc_stage_issue(const EpiArgs& e, int64_t row, int64_t col0, int lane, uint32_t sbuf) {
  using S = TcStage<CDT, MODE>;
  using CT = typename CStore<CDT>::T;
  if (e.beta_zero) return;
#pragma unroll
  for (int t = 0; t < S::nold; ++t) {
    int64_t i, j;
    tc_old_pos<MODE>(row, col0, lane, t, &i, &j);
    if (i >= e.m || j >= e.n) continue;
    const CT* c = static_cast<const CT*>(e.C) + (i * e.rs + j * e.cs) * (CStore<CDT>::cplx ? 2 : 1);
    if (!MXG_DBG_OK(c_in_extent<CDT>(e, c), e.dbg)) continue;
    cp_async_ca<S::esz>(sbuf + static_cast<uint32_t>((t * 32 + lane) * S::esz), c);
  }
}

template <int CDT, int MODE>
__device__ __forceinline__ void tc_stage_read(const EpiArgs& e, int64_t row, int64_t col0, int lane,
                                              const uint8_t* sbuf, COld<CDT> (&old)[TcChunk<MODE>::nold]) {
  using S = TcStage<CDT, MODE>;
  using CT = typename CStore<CDT>::T;
#pragma unroll
  for (int t = 0; t < S::nold; ++t) {
    int64_t i, j;
    tc_old_pos<MODE>(row, col0, lane, t, &i, &j);
    old[t].re = to_ct<CT>(0.0f);
    old[t].im = to_ct<CT>(0.0f);
    if (e.beta_zero || i >= e.m || j >= e.n) continue;
    const CT* p = reinterpret_cast<const CT*>(sbuf + (t * 32 + lane) * S::esz);
    old[t].re = p[0];
    if constexpr (CStore<CDT>::cplx) old[t].im = p[1];
  }
}

// The epilogue of one thread's row of a BN-column accumulator (TMEM address tbase) in
// 32-column chunks; stage: this warp's 8 KB staging area (shared-memory address).
template <int CDT, int MODE, int BN>
__device__ __forceinline__ void tc_epi_row(const EpiArgs& e, const EpiScalars<float, CDT>& sc, int64_t row,
                                           int64_t n0, uint32_t tbase, int lane, uint32_t stage,
                                           const uint8_t* stage_gen) {
  constexpr int NO = TcChunk<MODE>::nold;
  if constexpr (TcStage<CDT, MODE>::on) {
    constexpr uint32_t HALF = TC_STAGE_WARP_BYTES / 2;
    tc_stage_issue<CDT, MODE>(e, row, n0, lane, stage);
    cp_async_commit_group();
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      const uint32_t cur = static_cast<uint32_t>((c0 >> 5) & 1);
      if (c0 + 32 < BN) tc_stage_issue<CDT, MODE>(e, row, n0 + c0 + 32, lane, stage + (cur ^ 1u) * HALF);
      cp_async_commit_group();
      cp_async_wait_group<1>();   // this thread's copies of chunk c0 have landed
      COld<CDT> old[NO];
      tc_stage_read<CDT, MODE>(e, row, n0 + c0, lane, stage_gen + cur * HALF, old);
      uint32_t v[32];
      tmem_ld32(tbase + static_cast<uint32_t>(c0), v);
      tc_epi_finish<CDT, MODE>(e, sc, row, n0 + c0, v, lane, old);
    }
    cp_async_wait_group<0>();
  } else {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      COld<CDT> old[NO];
      tc_epi_load<CDT, MODE>(e, row, n0 + c0, lane, old);
      uint32_t v[32];
      tmem_ld32(tbase + static_cast<uint32_t>(c0), v);
      tc_epi_finish<CDT, MODE>(e, sc, row, n0 + c0, v, lane, old);
    }
  }
}

}  // namespace tc

// Host side (defined in gemm_tc.cu).
bool tc_get_encoder();
// 2-D map over a K-major plane (rows x Kp elements, row pitch Kp elements), box
// (rows_box x rowb bytes), rowb-byte swizzle (rowb = 64 or 128); rows past the plane
// read as zero.
bool tc_make_map(CUtensorMap* map, const void* ptr, int split, int64_t rows, int64_t Kp, uint32_t rows_box,
                 uint32_t rowb);
cudaError_t tc_current_sm_count(int* out);
// 2-D map over C stored with unit row stride (rows x cols elements of esz = 2, 4 or 8
// bytes, a complex element counted as one; column pitch ld_bytes), box (box_rows x
// box_cols), no swizzle; elements past the edges read as zero. False when C, its pitch
// or the box break a TMA alignment rule.
bool tc_make_c_map(CUtensorMap* map, const void* C, int esz, int64_t rows, int64_t cols, int64_t ld_bytes,
                   uint32_t box_rows, uint32_t box_cols);

}  // namespace mxg
