// Split-precision tensor-core contraction for computation precision single (tcgen05,
// sm_103a): P = A' B' with each packed operand split as X = X_hi + X_lo (TF32 or
// BF16 planes written by the pack) and
//     P ~= A_hi B_hi + A_hi B_lo + A_lo B_hi,
// accumulated in FP32 in tensor memory over the whole K' (Sec. 6.3: one cast per
// element of C), followed by the same fused epilogue as the other contractions.
//
// Persistent kernel, one CTA per SM, tiles of 128 x 256 of P walked in a grouped order
// (GM m-tiles at a time) so that concurrently running CTAs share operand panels in L2:
//   warp 0      TMA producer: per k-block of 64 bytes loads A_hi, A_lo (128 rows) and
//               B_hi, B_lo (256 rows) with the 64-byte swizzle into a 4-stage ring;
//   warp 1      owns the TMEM allocation (two 128 x 256 FP32 accumulators, 512
//               columns); one lane issues tcgen05.mma (M = 128, N = 256) for the three
//               products, frees each stage with tcgen05.commit and hands a finished
//               accumulator to the epilogue;
//   warps 2..5  epilogue: tcgen05.ld the accumulator (warp w reads TMEM lanes
//               32*(w%4)..), pair rows or columns for complex C, alpha/beta, store,
//               then release the accumulator -- overlapping the next tile's main loop.
// Every mbarrier wait is bounded in time (%globaltimer). On expiry the CTA sets the
// error word and an abort flag, skips its stores, waits (bounded) for its own TMA
// copies and MMAs in flight, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "grouped.h"
#include "tc_common.cuh"

namespace mxg {

struct TcArgs {
  int64_t Mp, Np, Kp;   // padded real problem (multiples of 128, 256, BK)
  EpiArgs e;
  int cdt, mode;        // C datatype and output mode (epilogue dispatched at run time)
  int* err;             // device error word set on a wait timeout (may be null)
};

using namespace tc;

namespace tcs {

constexpr int TC_BM = 128, TC_BN = 256, TC_GM = 16;
constexpr uint32_t TILE_A = TC_BM * ROWB;                  // 8 KB
constexpr uint32_t TILE_B = TC_BN * ROWB;                  // 16 KB
constexpr uint32_t RING_BYTES = 192 * 1024;                // shared-memory ring
constexpr uint32_t TC_SMEM = RING_BYTES + 1024 + 256 + TC_STAGE_BYTES;   // ring, barriers, epilogue staging
constexpr uint32_t TMEM_COLS = 2 * TC_BN;                  // two accumulators

// Operand formats: the split forms load hi and lo planes of A and B and issue three
// MMAs per k-step; TC16 loads one plane each and issues one.
template <int SPLIT> struct TcFmt {
  static constexpr int planes = (SPLIT == SPLIT_F16_ONE || SPLIT == SPLIT_BF16_ONE) ? 1 : 2;
  static constexpr int elem = (SPLIT == SPLIT_TF32) ? 4 : 2;
  // instruction-descriptor format code: 0 F16, 1 BF16 (kind::f16), 2 TF32 (kind::tf32)
  static constexpr uint32_t fmt = (SPLIT == SPLIT_TF32) ? 2u : (SPLIT == SPLIT_F16_ONE ? 0u : 1u);
  static_assert(fmt <= 2u, "format code");
  static constexpr uint32_t stage_bytes = planes * (TILE_A + TILE_B);
  static constexpr int stages = static_cast<int>(RING_BYTES / stage_bytes);   // 4 split, 8 TC16
};
constexpr uint32_t NBARS_MAX = 2 * 8 + 2 + 2 + 1;          // full, empty, acc_full, acc_empty, drain

template <int SPLIT>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  if constexpr (SPLIT != SPLIT_TF32) {
    constexpr uint32_t idesc = make_idesc(TcFmt<SPLIT>::fmt, TC_BM, TC_BN);
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  } else {
    constexpr uint32_t idesc = make_idesc(2, TC_BM, TC_BN);
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Tile t of the grouped order -> (m tile, n tile): groups of TC_GM m-tiles, n fastest
// within a group column.
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int* tm, int* tn) {
  const int per_group = TC_GM * tiles_n;
  const int g = t / per_group, r = t - g * per_group;
  const int gm0 = g * TC_GM;
  const int gsz = min(TC_GM, tiles_m - gm0);
  *tm = gm0 + r % gsz;
  *tn = r / gsz;
}

// One tile of work for the tcgen05 body: the tensor maps of its operand planes, its
// first rows of A' and B' (= its position in P), its number of k-blocks and the
// epilogue it ends with.
struct TcJob {
  const CUtensorMap *ah, *al, *bh, *bl;
  int32_t ym, yn;
  int nkb;
  const EpiArgs* e;
  int cdt, mode;
};

// The tiles of one problem in the grouped order; maps and arguments are kernel
// parameters.
struct TcOneSrc {
  const CUtensorMap *ah, *al, *bh, *bl;
  const TcArgs* g;
  int tiles_m, tiles_n, nkb;
  __device__ __forceinline__ int count() const { return tiles_m * tiles_n; }
  __device__ __forceinline__ TcJob job(int t) const {
    int tm, tn;
    tile_coords(t, tiles_m, tiles_n, &tm, &tn);
    return TcJob{ah, al, bh, bl, tm * TC_BM, tn * TC_BN, nkb, &g->e, g->cdt, g->mode};
  }
  __device__ __forceinline__ void prepare(const TcJob&) const {}
};

// The tiles of many problems, from a device work list (longest K' first); each problem's
// maps were encoded on the host and copied to the device before the launch.
struct TcGroupSrc {
  const TcGroupProb* probs;
  const GroupTile* tiles;
  int ntiles, bk;
  __device__ __forceinline__ int count() const { return ntiles; }
  __device__ __forceinline__ TcJob job(int t) const {
    const GroupTile w = tiles[t];
    const TcGroupProb* p = probs + w.prob;
    return TcJob{&p->maps[0], &p->maps[1], &p->maps[2], &p->maps[3], w.tm * TC_BM, w.tn * TC_BN,
                 static_cast<int>(p->Kp / bk), &p->e, p->cdt, p->mode};
  }
  // order the TMA unit's reads of the maps after their copy to global memory
  __device__ __forceinline__ void prepare(const TcJob& j) const {
    const CUtensorMap* m[4] = {j.ah, j.al, j.bh, j.bl};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m[i]) : "memory");
  }
};

template <int SPLIT, class Src>
__device__ __forceinline__ void tc_body(const Src& src, int* err) {
  using F = TcFmt<SPLIT>;
  constexpr int TC_STAGES = F::stages;
  constexpr uint32_t STAGE_BYTES = F::stage_bytes;
  constexpr int BK = ROWB / F::elem;        // k elements per 64-byte row
  constexpr int KSTEPS = ROWB / 32;         // MMAs per row (each consumes 32 bytes of K)
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen_base = smem_raw + (base - raw);
  const uint32_t bars = base + TC_STAGES * STAGE_BYTES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gen_base + TC_STAGES * STAGE_BYTES + 8 * NBARS_MAX);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (TC_STAGES + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * TC_STAGES + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * TC_STAGES + 2 + b); };
  const uint32_t drain_bar = bars + 8u * (2 * TC_STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = src.count();

  static_assert(2 * TC_STAGES + 5 <= static_cast<int>(NBARS_MAX), "barrier area");
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), 4);   // one arrival per epilogue warp
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  auto fail = [&]() {
    if (err) atomicExch(err, 1);
    *abort_flag = 1;
  };

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TcJob jb = src.job(t);
        src.prepare(jb);
        const int32_t ym = jb.ym, yn = jb.yn;
        for (int kb = 0; kb < jb.nkb; ++kb, ++it) {
          const int s = static_cast<int>(it % TC_STAGES);
          const uint32_t use = it / TC_STAGES;
          if (!mbar_wait(empty(s), (use & 1u) ^ 1u, abort_flag)) { ok = false; break; }
          const uint32_t st = base + s * STAGE_BYTES;
          mbar_expect_tx(full(s), STAGE_BYTES);
          const int32_t kx = kb * BK;
          // stage layout: A planes (F::planes x TILE_A), then B planes
          tma_load_2d(st, jb.ah, kx, ym, full(s));
          if constexpr (F::planes == 2) tma_load_2d(st + TILE_A, jb.al, kx, ym, full(s));
          tma_load_2d(st + F::planes * TILE_A, jb.bh, kx, yn, full(s));
          if constexpr (F::planes == 2) tma_load_2d(st + 2 * TILE_A + TILE_B, jb.bl, kx, yn, full(s));
        }
      }
      if (!ok) {
        fail();
        // wait (bounded) for this thread's own copies: the last use of every stage
        for (uint32_t j = (it > TC_STAGES ? it - TC_STAGES : 0); j < it; ++j)
          mbar_drain(full(j % TC_STAGES), (j / TC_STAGES) & 1u);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      int j = 0;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++j) {
        const int b = j & 1;
        if (!mbar_wait(acc_empty(b), (static_cast<uint32_t>(j >> 1) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_tmem = tmem + static_cast<uint32_t>(b * TC_BN);
        const int nkb = src.job(t).nkb;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = static_cast<int>(it % TC_STAGES);
          if (!mbar_wait(full(s), (it / TC_STAGES) & 1u, abort_flag)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = base + s * STAGE_BYTES;
          const uint32_t a_hi = st, a_lo = st + TILE_A, b_hi = st + F::planes * TILE_A, b_lo = b_hi + TILE_B;
#pragma unroll
          for (int kk = 0; kk < KSTEPS; ++kk) {
            const uint32_t off = kk * 32;
            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
            mma_issue<SPLIT>(acc_tmem, sw64_desc(a_hi + off), sw64_desc(b_hi + off), first);
            if constexpr (F::planes == 2) {
              mma_issue<SPLIT>(acc_tmem, sw64_desc(a_hi + off), sw64_desc(b_lo + off), 1u);
              mma_issue<SPLIT>(acc_tmem, sw64_desc(a_lo + off), sw64_desc(b_hi + off), 1u);
            }
          }
          mma_commit(empty(s));
        }
        if (!ok) break;
        mma_commit(acc_full(b));
      }
      if (!ok) fail();
      // every MMA this thread issued has completed once the drain barrier flips
      mma_commit(drain_bar);
      mbar_drain(drain_bar, 0);
    }
  } else {
    // epilogue warps 2..5: TMEM lane quarter q = warp % 4
    const int q = warp & 3;
    // this warp's staging buffers for old C values, after the barrier area
    const uint32_t stage_w = bars + 256u + static_cast<uint32_t>(q) * TC_STAGE_WARP_BYTES;
    const uint8_t* stage_w_gen = gen_base + (stage_w - base);
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      const TcJob jb = src.job(t);
      const int b = j & 1;
      const bool ok = mbar_wait(acc_full(b), static_cast<uint32_t>(j >> 1) & 1u, abort_flag);
      if (!__all_sync(0xffffffffu, ok && !*abort_flag)) {
        if (lane == 0 && !ok) fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t m0 = jb.ym, n0 = jb.yn;
      const int64_t row = m0 + 32 * q + lane;
      const EpiArgs& e = *jb.e;
      const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(b * TC_BN);
      with_c_mode(jb.cdt, jb.mode, [&](auto C, auto M) {
        constexpr int CDT = decltype(C)::value, MODE = decltype(M)::value;
        const EpiScalars<float, CDT> sc = epi_scalars<float, CDT>(e);
        tc_epi_row<CDT, MODE, TC_BN>(e, sc, row, n0, tbase, lane, stage_w, stage_w_gen);
      });
      // release the accumulator to the MMA warp
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(b));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}


template <int SPLIT>
__global__ void __launch_bounds__(192, 1)
tc_split_gemm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
              const __grid_constant__ TcArgs g) {
  constexpr int BK = ROWB / TcFmt<SPLIT>::elem;
  const TcOneSrc src{&mAh, &mAl, &mBh, &mBl, &g, static_cast<int>(g.Mp / TC_BM), static_cast<int>(g.Np / TC_BN),
                     static_cast<int>(g.Kp / BK)};
  tc_body<SPLIT>(src, g.err);
}

// Grouped form: a persistent launch over the (problem, tile) work list of a bucket.
template <int SPLIT>
__global__ void __launch_bounds__(192, 1)
tc_grouped_gemm(const TcGroupProb* __restrict__ probs, const GroupTile* __restrict__ tiles, int ntiles, int* err) {
  const TcGroupSrc src{probs, tiles, ntiles, static_cast<int>(ROWB / TcFmt<SPLIT>::elem)};
  tc_body<SPLIT>(src, err);
}

template <int SPLIT>
cudaError_t launch_one(const CUtensorMap* maps, const TcArgs& g, int sms, cudaStream_t s) {
  auto kern = tc_split_gemm<SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (g.Mp / TC_BM) * (g.Np / TC_BN);
  const int grid = static_cast<int>(ntiles < sms ? ntiles : sms);
  kern<<<grid, 192, TC_SMEM, s>>>(maps[0], maps[1], maps[2], maps[3], g);
  return cudaGetLastError();
}

template <int SPLIT>
cudaError_t launch_grouped(const TcGroupProb* probs, const GroupTile* tiles, int ntiles, int* err, int grid,
                           cudaStream_t s) {
  auto kern = tc_grouped_gemm<SPLIT>;
  cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (r != cudaSuccess) return r;
  kern<<<grid, 192, TC_SMEM, s>>>(probs, tiles, ntiles, err);
  return cudaGetLastError();
}

// The instantiations, in four translation units (the epilogue's 16 C datatype / output
// mode pairs dominate their compile time): the single-problem kernel of the split
// formats in gemm_tc.cu and of the one-pass formats in gemm_tc_one.cu, the grouped
// kernel in gemm_tc_grouped.cu and gemm_tc_grouped_one.cu.
cudaError_t launch_single_split(int split, const CUtensorMap* maps, const TcArgs& g, int sms, cudaStream_t s);
cudaError_t launch_single_one(int split, const CUtensorMap* maps, const TcArgs& g, int sms, cudaStream_t s);
cudaError_t launch_grouped_split(int split, const TcGroupProb* probs, const GroupTile* tiles, int ntiles, int* err,
                                 int grid, cudaStream_t s);
cudaError_t launch_grouped_one(int split, const TcGroupProb* probs, const GroupTile* tiles, int ntiles, int* err,
                               int grid, cudaStream_t s);

}  // namespace tcs
}  // namespace mxg
