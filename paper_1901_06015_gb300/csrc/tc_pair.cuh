// Tensor-core contraction on CTA pairs (tcgen05 cta_group::2, sm_103a).
//
// The same product as tc_split_gemm (one pass for the binary16 / bfloat16 computation
// precisions, hi*hi + hi*lo + lo*hi for the split forms, FP32 accumulation over the
// whole K' in tensor memory, the fused epilogue of Sec. 7.1), computed on 256 x 256
// tiles of P by a cluster of two CTAs on two SMs. Each CTA loads its own 128 rows of A
// and its own 128 rows of B (plain per-CTA TMA loads, no multicast); one MMA of
// M = 256, N = 256 issued by the even CTA of the pair reads A from both CTAs' shared
// memory (one half each) and B from both (one half each), and writes each CTA's 128
// rows of the accumulator into that CTA's tensor memory. Per k-block a CTA therefore
// moves 128 + 128 rows of operands for a 128 x 256 share of the tile, against 128 +
// 256 rows in the one-CTA kernel: a third fewer bytes from L2 per flop, in half as many
// row requests (128-byte rows), which is what bounds the one-pass 16-bit form there.
//
// Two variants of the kernel: whole tiles with the epilogue warps loading old C (warps
// 0..5, 192 threads), and the one with the stream-K tail and the C loader (warps 0..6,
// 224 threads); the host picks per call (the loader where a tile has at most 64 MMA
// steps or the tail runs, the tail when the last wave leaves enough pairs idle).
// Roles (one CTA per SM, persistent over pair tiles):
//   warp 0      TMA producer in both CTAs: its halves of A and B, in 128-byte k rows
//               with the 128-byte swizzle, into its own 6- (split forms: 3-) stage
//               ring (2 stages with a short k, see warp 6); the completion of both CTAs'
//               copies is counted on the even CTA's "full" barrier (.cta_group::2
//               copies);
//   warp 1      both CTAs allocate the two 128 x 256 FP32 accumulators together
//               (cta_group::2); in the even CTA one lane issues the MMAs, frees each
//               stage in both CTAs and hands a finished accumulator to both CTAs'
//               epilogues (one tcgen05.commit per CTA, no multicast);
//   warps 2..5  epilogue in both CTAs over the CTA's own 128 rows, then an arrival on
//               the even CTA's accumulator-empty barrier (eight arrivals per use);
//   warp 6      C loader, when C has unit row stride and beta != 0: TMA tile loads of
//               the old C values of each 32-column chunk the epilogue will update, in
//               the epilogue's order, into a ring of chunk buffers in the space the
//               operand ring leaves (a short k leaves it two stages and room for up to
//               24 chunks). The epilogue then reads old C from shared memory: the loads
//               are in flight ahead of use without taking registers, which is what
//               limited the epilogue's C bandwidth when the epilogue warps loaded C
//               themselves.
// Every wait is bounded in time; on expiry a CTA sets the error word and both CTAs'
// abort flags, skips its stores, drains its own MMAs and copies (bounded), and the pair
// meets at a final cluster barrier before freeing tensor memory, so neither CTA exits
// while the other may still touch its shared or tensor memory.
//
// Stream-K tail. When the pair tiles do not fill a whole number of waves (T tiles on P
// resident pairs, r = T mod P > 0), the last r tiles of the order are cut along k into P
// equal ranges of the r * nkb (tile, k-block) steps, one per pair, processed before the
// pair's whole tiles: every pair then does the same work, instead of r pairs running a
// last wave alone. A range covers the ends of at most two tiles. Its epilogue writes the
// FP32 partial accumulator to the workspace (one slot per pair, range part and CTA) and
// takes a ticket on the tile's counter; the warp that takes the last ticket adds the
// tile's partials in increasing k (a fixed order, so the result does not depend on which
// pair finished last) and applies the epilogue of Sec. 7.1 to the sum. Nothing waits on
// another pair: the ticket replaces the wait.
#pragma once

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "tc_common.cuh"

namespace mxg {
namespace pairk {

using namespace tc;


constexpr int P_BM = 128;                         // rows of A per CTA (256 per pair)
constexpr int P_BN = 256;                         // columns of the pair tile (MMA N)
constexpr int P_GM = 8;                           // pair rows per group of the tile order
// Bytes of K per tile row, with the swizzle of that width. 128-byte rows halve the
// number of row requests TMA sends to L2 per byte against 64-byte rows; with 64-byte
// rows the request path, not the bytes, limited the one-pass 16-bit form (measured on
// GB300 at 8192^3: 1.25 PF/s with 64-byte rows, 1.66 PF/s with 128-byte rows).
constexpr int P_RB = 128;
constexpr uint32_t P_RING = 192 * 1024;
constexpr uint32_t P_BAR_AREA = 1024;             // barriers, TMEM address, abort flag
// alignment slack, barriers, operand ring, epilogue staging; the operand ring and the
// staging area form one span that the C prefetch shares with the ring (below)
constexpr uint32_t P_SMEM = 1024 + P_BAR_AREA + P_RING + TC_STAGE_BYTES;
constexpr uint32_t P_SPAN = P_RING + TC_STAGE_BYTES;
constexpr uint32_t P_TMEM_COLS = 2 * P_BN;        // two accumulators
constexpr int P_NCB = 24;                         // C prefetch buffers at most
// threads of the two kernel variants: with the C loader warp (XT) and without
constexpr int P_THREADS_XT = 224;
constexpr int P_THREADS = 192;

// RB: bytes of K per tile row (64 or 128, with the swizzle of that width).
template <int SPLIT, int RB> struct PairFmt {
  static constexpr int planes = (SPLIT == SPLIT_F16_ONE || SPLIT == SPLIT_BF16_ONE) ? 1 : 2;
  static constexpr int elem = (SPLIT == SPLIT_TF32) ? 4 : 2;
  static constexpr uint32_t fmt = (SPLIT == SPLIT_TF32) ? 2u : (SPLIT == SPLIT_F16_ONE ? 0u : 1u);
  static constexpr uint32_t tile_a = P_BM * RB;          // this CTA's rows of A
  static constexpr uint32_t tile_b = (P_BN / 2) * RB;    // this CTA's half of B
  static constexpr uint32_t stage_bytes = planes * (tile_a + tile_b);
  // 128-byte rows: 6 stages one-pass, 3 split (64-byte rows: 12 and 6)
  static constexpr int stages = static_cast<int>(P_RING / stage_bytes);
};
// full, empty (12 each at most), acc_full, acc_empty, drain, c_full, c_empty
constexpr int P_NBARS = 2 * 12 + 2 + 2 + 1 + 2 * P_NCB;
static_assert(8 * P_NBARS + 8 <= P_BAR_AREA, "barrier area");

struct PairArgs {
  int64_t Mp, Np, Kp;
  EpiArgs e;
  int cdt, mode;
  int* err;
  // stream-K tail (sk_r > 0): tiles [sk_full * P, sk_full * P + sk_r) of the order are
  // cut along k; sk_part holds 4 slots of P_BM x P_BN FP32 per pair, sk_cnt 8 counters
  // per tail tile (CTA, epilogue warp), zero at launch
  float4* sk_part;
  int* sk_cnt;
  int sk_full, sk_r;
  // operand ring stages in use (at most the format's); C prefetch (cpf): ncb buffers of
  // c_bytes after the stages, one per 32-column accumulator chunk of old C values
  // (c_rows x c_cols elements as the chunk's C region, column by column)
  int stages;
  int cpf, ncb, c_rows;
  int c_rep;            // map elements per C element (2 for double complex, else 1)
  uint32_t c_bytes;
};

// One item of a pair's work: tile t (index in the order), k-blocks [kb0, kb1); for a
// range of a stream-K tile, tl is the tile's index in the tail and seg the range's part
// (0 or 1) in this pair's slots, else tl = -1.
struct PairItem {
  int t, kb0, kb1, tl, seg;
};

// First k-block step of pair c's range: c * W / P of the W tail steps.
__device__ __forceinline__ int64_t sk_begin(int64_t W, int P, int c) { return W * c / P; }
// The pair whose range holds tail step x: the largest c with sk_begin(c) <= x.
__device__ __forceinline__ int sk_owner(int64_t W, int P, int64_t x) {
  return static_cast<int>(((x + 1) * P + W - 1) / W) - 1;
}

// Item i of pair cid (ncl pairs): its stream-K ranges first, then its whole tiles. XT:
// the kernel variant that has the stream-K tail (the other has whole tiles only).
template <bool XT>
__device__ __forceinline__ bool pair_item(const PairArgs& g, int ntiles, int nkb, int cid, int ncl, int i,
                                          PairItem* w) {
  if (!XT || g.sk_r == 0) {
    const int t = cid + i * ncl;
    if (t >= ntiles) return false;
    *w = PairItem{t, 0, nkb, -1, -1};
    return true;
  }
  const int64_t W = static_cast<int64_t>(g.sk_r) * nkb;
  const int64_t kb = sk_begin(W, ncl, cid), ke = sk_begin(W, ncl, cid + 1);
  int nseg = 0, tl0 = 0;
  if (ke > kb) {
    tl0 = static_cast<int>(kb / nkb);
    nseg = static_cast<int>((ke - 1) / nkb) - tl0 + 1;
  }
  if (i < nseg) {
    const int tl = tl0 + i;
    const int64_t t0 = static_cast<int64_t>(tl) * nkb;
    const int lo = static_cast<int>(max(kb, t0) - t0), hi = static_cast<int>(min(ke, t0 + nkb) - t0);
    *w = PairItem{g.sk_full * ncl + tl, lo, hi, tl, i};
    return true;
  }
  const int t = cid + (i - nseg) * ncl;
  if (t >= g.sk_full * ncl) return false;
  *w = PairItem{t, 0, nkb, -1, -1};
  return true;
}

__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared-memory object in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}
// Wait with cluster-scope acquire (barriers completed by the other CTA of the pair).
__device__ __forceinline__ bool mbar_try_cl(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_cl(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_cl(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > kWaitNs) return false;
    }
  }
}
__device__ __forceinline__ void mbar_drain_cl(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try_cl(bar, parity))
    if (gtimer() - t0 > kWaitNs) return;
}
// TMA tile load into this CTA's shared memory whose completion is counted on `bar`,
// which may be the barrier of either CTA of the pair (shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                                 uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
template <int SPLIT>
__device__ __forceinline__ void mma_pair(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  constexpr uint32_t idesc = make_idesc(PairFmt<SPLIT, 64>::fmt, 2 * P_BM, P_BN);
  if constexpr (SPLIT != SPLIT_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  }
}
// Arrive on `cluster_bar` (either CTA's barrier) once every MMA this thread issued so
// far has completed.
__device__ __forceinline__ void commit_pair(uint32_t cluster_bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(cluster_bar)
               : "memory");
}

// Pair tile t of the grouped order -> (pair row, column tile).
__device__ __forceinline__ void pair_coords(int t, int pairs_m, int tiles_n, int* pm, int* tn) {
  const int per_group = P_GM * tiles_n;
  const int g = t / per_group, r = t - g * per_group;
  const int gm0 = g * P_GM;
  const int gsz = min(P_GM, pairs_m - gm0);
  *pm = gm0 + r % gsz;
  *tn = r / gsz;
}

// float4 index of the slot of pair c, range part seg, CTA rank: P_BM x P_BN FP32 as
// [column / 4][row][4], so a warp's 32 rows of four columns are 512 contiguous bytes.
constexpr int SK_SLOT4 = P_BM * P_BN / 4;
// Bytes of the partial slots for `pairs` pairs (two range parts, two CTAs each).
constexpr size_t sk_part_bytes(int64_t pairs) { return static_cast<size_t>(pairs) * 4 * SK_SLOT4 * 16; }
__device__ __forceinline__ int64_t sk_slot(int c, int seg, uint32_t rank) {
  return ((static_cast<int64_t>(c) * 2 + seg) * 2 + rank) * SK_SLOT4;
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
      ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
        "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
        "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

// The sum of a stream-K tile's partial accumulators for this thread's row (the ranges
// of pairs c_first .. c_last, in increasing k), written over the accumulator in tensor
// memory (tbase), where the tile's ordinary epilogue then reads it.
__device__ __forceinline__ void sk_sum_to_tmem(const PairArgs& g, uint32_t tbase, int rl, uint32_t rank, int tl,
                                               int nkb, int ncl, int c_first, int c_last) {
  const int64_t W = static_cast<int64_t>(g.sk_r) * nkb;
#pragma unroll 1
  for (int c0 = 0; c0 < P_BN; c0 += 32) {
    float a[32];
#pragma unroll 1
    for (int c = c_first; c <= c_last; ++c) {
      const int seg = tl - static_cast<int>(sk_begin(W, ncl, c) / nkb);
      const float4* slot = g.sk_part + sk_slot(c, seg, rank) + rl + (c0 >> 2) * P_BM;
      float4 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = __ldcg(slot + u * P_BM);
      if (c == c_first) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          a[4 * u] = x[u].x; a[4 * u + 1] = x[u].y; a[4 * u + 2] = x[u].z; a[4 * u + 3] = x[u].w;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          a[4 * u] = __fadd_rn(a[4 * u], x[u].x);
          a[4 * u + 1] = __fadd_rn(a[4 * u + 1], x[u].y);
          a[4 * u + 2] = __fadd_rn(a[4 * u + 2], x[u].z);
          a[4 * u + 3] = __fadd_rn(a[4 * u + 3], x[u].w);
        }
      }
    }
    uint32_t v[32];
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) v[jj] = __float_as_uint(a[jj]);
    tmem_st32(tbase + static_cast<uint32_t>(c0), v);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// An epilogue warp's view of the C prefetch ring: buffers, their barriers, and the
// number of chunks consumed so far (the loader issues the same sequence).
struct CRing {
  uint32_t buf;            // shared-memory address of buffer 0
  const uint8_t* buf_gen;  // the same, generic
  uint32_t full, empty;    // barrier of buffer 0 (8 bytes per buffer)
  int ncb;
  uint32_t c_bytes;
  uint32_t cit;
};

// Wait (bounded) until the next chunk of the ring has landed; its buffer index in *b.
__device__ __forceinline__ bool cring_wait(const CRing& r, volatile int* abort_flag, int* b) {
  *b = static_cast<int>(r.cit % static_cast<uint32_t>(r.ncb));
  const uint32_t use = r.cit / static_cast<uint32_t>(r.ncb);
  return mbar_wait(r.full + 8u * static_cast<uint32_t>(*b), use & 1u, abort_flag);
}
// Hand the chunk's buffer back to the loader (four epilogue warps arrive per use).
__device__ __forceinline__ void cring_release(CRing& r, int b, int lane) {
  __syncwarp();
  if (lane == 0) mbar_arrive(r.empty + 8u * static_cast<uint32_t>(b));
  ++r.cit;
}

// Old C values of a chunk from its prefetched region (element (r, c) at c * c_rows + r):
// the same positions as tc_epi_load reads from global memory, relative to the chunk.
template <int CDT, int MODE>
__device__ __forceinline__ void pf_read(const uint8_t* chunk, int rl, int lane,
                                        COld<CDT> (&old)[TcChunk<MODE>::nold]) {
  using CT = typename CStore<CDT>::T;
  constexpr bool CX = CStore<CDT>::cplx;
  constexpr int ESZ = static_cast<int>(sizeof(CT)) * (CX ? 2 : 1);
#pragma unroll
  for (int t = 0; t < TcChunk<MODE>::nold; ++t) {
    int idx;
    if constexpr (MODE == OUT_ROWPAIR) idx = (2 * t + (lane & 1)) * (P_BM / 2) + (rl >> 1);
    else idx = t * P_BM + rl;
    const CT* p = reinterpret_cast<const CT*>(chunk + idx * ESZ);
    old[t].re = p[0];
    if constexpr (CX) old[t].im = p[1];
    else old[t].im = to_ct<CT>(0.0f);
  }
}

// The epilogue of one thread's row (as tc_epi_row) with the old C values taken from the
// prefetch ring. False when a wait ran out or the pair aborted (stores of the remaining
// chunks skipped).
template <int CDT, int MODE, int BN>
__device__ __forceinline__ bool tc_epi_row_pf(const EpiArgs& e, const EpiScalars<float, CDT>& sc, int64_t row,
                                              int64_t n0, uint32_t tbase, int lane, int rl, CRing& cr,
                                              volatile int* abort_flag) {
  constexpr int NO = TcChunk<MODE>::nold;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    int b;
    const bool ok = cring_wait(cr, abort_flag, &b);
    if (!__all_sync(0xffffffffu, ok)) return false;
    COld<CDT> old[NO];
    pf_read<CDT, MODE>(cr.buf_gen + static_cast<size_t>(b) * cr.c_bytes, rl, lane, old);
    cring_release(cr, b, lane);
    uint32_t v[32];
    tmem_ld32(tbase + static_cast<uint32_t>(c0), v);
    tc_epi_finish<CDT, MODE>(e, sc, row, n0 + c0, v, lane, old);
  }
  return true;
}

// XT: the variant with the stream-K tail and the C loader (warp 6); without them
// (whole tiles, old C read by the epilogue warps) the epilogue keeps more registers for
// its loads in flight, which that path needs (measured: 40% more C bandwidth at a short
// k, 3% at 8192^3 than the same code compiled with the tail in).
template <int SPLIT, int RB, bool XT>
__global__ void __launch_bounds__(XT ? P_THREADS_XT : P_THREADS, 1)
tc_pair_gemm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
             const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
             const __grid_constant__ CUtensorMap mC, PairArgs g) {
  using F = PairFmt<SPLIT, RB>;
  constexpr int S = F::stages;
  constexpr uint32_t STAGE_BYTES = F::stage_bytes;
  constexpr uint32_t P_TILE_A = F::tile_a, P_TILE_B = F::tile_b;
  constexpr int BK = RB / F::elem;          // k elements per row
  constexpr int KSTEPS = RB / 32;           // MMAs per row (each consumes 32 bytes of K)
  static_assert(2 * S + 5 + 2 * P_NCB <= P_NBARS, "barrier area");
  static_assert(S * STAGE_BYTES <= P_RING, "operand ring");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen_base = smem_raw + (base - raw);
  const uint32_t bars = base;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gen_base + 8 * P_NBARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t ring = base + P_BAR_AREA;        // 1024-aligned, as the 128-byte swizzle needs
  const int SR = XT ? g.stages : S;               // operand stages in use
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (S + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * S + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * S + 2 + b); };
  const uint32_t drain_bar = bars + 8u * (2 * S + 4);
  const uint32_t c_full0 = bars + 8u * (2 * S + 5), c_empty0 = c_full0 + 8u * P_NCB;
  const uint32_t cbuf0 = ring + static_cast<uint32_t>(SR) * STAGE_BYTES;   // C buffers after the stages

  const uint32_t rank = cta_rank();               // 0: issues the MMAs; 1: its peer
  const bool leader = (rank == 0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pairs_m = static_cast<int>((g.Mp + 2 * P_BM - 1) / (2 * P_BM));
  const int tiles_n = static_cast<int>(g.Np / P_BN);
  const int ntiles = pairs_m * tiles_n;
  const int nkb = static_cast<int>(g.Kp / BK);
  const int cid = static_cast<int>(blockIdx.x >> 1), ncl = static_cast<int>(gridDim.x >> 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);      // the even CTA's arrive.expect_tx, plus both CTAs' bytes
      mbar_init(empty(s), 1);     // one commit of the even CTA's MMAs
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), 8);   // four epilogue warps in each CTA of the pair
    }
    mbar_init(drain_bar, 1);
    if (XT)
      for (int b = 0; b < g.ncb; ++b) {
        mbar_init(c_full0 + 8u * b, 1);    // the loader's arrive.expect_tx plus the chunk's bytes
        mbar_init(c_empty0 + 8u * b, 4);   // the four epilogue warps
      }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {   // both CTAs allocate together: the same columns in each
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(P_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();   // both CTAs' barriers exist before either touches the other's
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t peer = rank ^ 1u;
  auto fail = [&]() {
    if (g.err) atomicExch(g.err, 1);
    *abort_flag = 1;
    st_cluster_u32(peer_addr(smem_u32(const_cast<int*>(abort_flag)), peer), 1u);
  };

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      int s = 0;          // stage of step it, and the parity of its use (no division
      uint32_t ph = 0;    // in the issue loop)
      bool ok = true;
      PairItem w;
      for (int i = 0; ok && pair_item<XT>(g, ntiles, nkb, cid, ncl, i, &w); ++i) {
        int pm, tn;
        pair_coords(w.t, pairs_m, tiles_n, &pm, &tn);
        const int32_t ym = pm * 2 * P_BM + static_cast<int32_t>(rank) * P_BM;
        const int32_t yn = tn * P_BN + static_cast<int32_t>(rank) * (P_BN / 2);
        for (int kb = w.kb0; kb < w.kb1; ++kb, ++it) {
          if (!mbar_wait_cl(empty(s), ph ^ 1u, abort_flag)) { ok = false; break; }
          const uint32_t st = ring + s * STAGE_BYTES;
          // both CTAs' copies complete on the even CTA's full barrier; only the even CTA
          // arrives on it, announcing both halves' bytes
          const uint32_t fb = leader ? full(s) : peer_addr(full(s), 0);
          if (leader) mbar_expect_tx(full(s), 2 * STAGE_BYTES);
          const int32_t kx = kb * BK;
          tma_load_2d_pair(st, &mAh, kx, ym, fb);
          if constexpr (F::planes == 2) tma_load_2d_pair(st + P_TILE_A, &mAl, kx, ym, fb);
          tma_load_2d_pair(st + F::planes * P_TILE_A, &mBh, kx, yn, fb);
          if constexpr (F::planes == 2) tma_load_2d_pair(st + 2 * P_TILE_A + P_TILE_B, &mBl, kx, yn, fb);
          if (++s == SR) { s = 0; ph ^= 1u; }
        }
      }
      if (!ok) {
        fail();
        // the even CTA waits (bounded) for the copies it counted: the last use of every stage
        if (leader)
          for (uint32_t j = (it > static_cast<uint32_t>(SR) ? it - SR : 0); j < it; ++j)
            mbar_drain_cl(full(static_cast<int>(j % static_cast<uint32_t>(SR))), (j / static_cast<uint32_t>(SR)) & 1u);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      PairItem w;
      for (int j = 0; ok && pair_item<XT>(g, ntiles, nkb, cid, ncl, j, &w); ++j) {
        const int b = j & 1;
        if (!mbar_wait_cl(acc_empty(b), (static_cast<uint32_t>(j >> 1) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_tmem = tmem + static_cast<uint32_t>(b * P_BN);
        for (int kb = w.kb0; kb < w.kb1; ++kb) {
          if (!mbar_wait_cl(full(s), ph, abort_flag)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = ring + s * STAGE_BYTES;
          const uint32_t a_hi = st, a_lo = st + P_TILE_A, b_hi = st + F::planes * P_TILE_A, b_lo = b_hi + P_TILE_B;
#pragma unroll
          for (int kk = 0; kk < KSTEPS; ++kk) {
            const uint32_t off = kk * 32;
            const uint32_t first = (kb == w.kb0 && kk == 0) ? 0u : 1u;
            mma_pair<SPLIT>(acc_tmem, swz_desc<RB>(a_hi + off), swz_desc<RB>(b_hi + off), first);
            if constexpr (F::planes == 2) {
              mma_pair<SPLIT>(acc_tmem, swz_desc<RB>(a_hi + off), swz_desc<RB>(b_lo + off), 1u);
              mma_pair<SPLIT>(acc_tmem, swz_desc<RB>(a_lo + off), swz_desc<RB>(b_hi + off), 1u);
            }
          }
          commit_pair(empty(s));                    // this CTA's stage is free ...
          commit_pair(peer_addr(empty(s), peer));   // ... and the peer's
          if (++s == SR) { s = 0; ph ^= 1u; }
        }
        if (!ok) break;
        commit_pair(acc_full(b));
        commit_pair(peer_addr(acc_full(b), peer));
      }
      if (!ok) fail();
      // every MMA this thread issued has completed once the drain barrier flips
      commit_pair(drain_bar);
      mbar_drain_cl(drain_bar, 0);
    }
  } else if (warp <= 5) {
    // epilogue warps 2..5: TMEM lane quarter q = warp % 4 of this CTA's 128 rows
    const int q = warp & 3;
    // this warp's staging buffers for old C values (no C prefetch), after the ring
    const uint32_t stage_w = ring + P_RING + static_cast<uint32_t>(q) * TC_STAGE_WARP_BYTES;
    const uint8_t* stage_w_gen = gen_base + (stage_w - base);
    const int rl = 32 * q + lane;   // this thread's row of the CTA's 128
    CRing cr{cbuf0, gen_base + (cbuf0 - base), c_full0, c_empty0, g.ncb, g.c_bytes, 0u};
    auto release = [&](int b) {       // hand the accumulator back to the even CTA's MMA thread
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        if (leader) mbar_arrive(acc_empty(b));
        else mbar_arrive_cluster(peer_addr(acc_empty(b), 0));
      }
    };
    PairItem w;
    for (int j = 0; pair_item<XT>(g, ntiles, nkb, cid, ncl, j, &w); ++j) {
      int pm, tn;
      pair_coords(w.t, pairs_m, tiles_n, &pm, &tn);
      const int b = j & 1;
      const bool ok = mbar_wait_cl(acc_full(b), static_cast<uint32_t>(j >> 1) & 1u, abort_flag);
      if (!__all_sync(0xffffffffu, ok && !*abort_flag)) {
        if (lane == 0 && !ok) fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t m0 = static_cast<int64_t>(pm) * 2 * P_BM + static_cast<int64_t>(rank) * P_BM;
      const int64_t n0 = static_cast<int64_t>(tn) * P_BN;
      const int64_t row = m0 + rl;
      const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(b * P_BN);
      if (XT && w.tl >= 0) {
        // a range of a stream-K tile: its partial accumulator to this pair's slot
        float4* slot = g.sk_part + sk_slot(cid, w.seg, rank) + rl;
#pragma unroll 1
        for (int c0 = 0; c0 < P_BN; c0 += 32) {
          uint32_t v[32];
          tmem_ld32(tbase + static_cast<uint32_t>(c0), v);
#pragma unroll
          for (int u = 0; u < 8; ++u)
            __stcg(slot + ((c0 >> 2) + u) * P_BM,
                   make_float4(__uint_as_float(v[4 * u]), __uint_as_float(v[4 * u + 1]),
                               __uint_as_float(v[4 * u + 2]), __uint_as_float(v[4 * u + 3])));
        }
        // a ticket on the tile's counter for this CTA and warp: the last of the tile's
        // ranges sums them all into its accumulator and runs the epilogue
        const int64_t W = static_cast<int64_t>(g.sk_r) * nkb;
        const int c_first = sk_owner(W, ncl, static_cast<int64_t>(w.tl) * nkb);
        const int c_last = sk_owner(W, ncl, static_cast<int64_t>(w.tl + 1) * nkb - 1);
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0)
          last = (atomicAdd(g.sk_cnt + (w.tl * 2 + static_cast<int>(rank)) * 4 + q, 1) == c_last - c_first);
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) {
          release(b);
          // the tile's prefetched C chunks are the finishing range's: pass them by
          bool cok = true;
          if (g.cpf) {
            for (int c0 = 0; c0 < P_BN && cok; c0 += 32) {
              int cb;
              cok = __all_sync(0xffffffffu, cring_wait(cr, abort_flag, &cb));
              if (cok) cring_release(cr, cb, lane);
            }
          }
          if (!cok) {
            if (lane == 0) fail();
            break;
          }
          continue;
        }
        __threadfence();
        sk_sum_to_tmem(g, tbase, rl, rank, w.tl, nkb, ncl, c_first, c_last);
      }
      bool eok = true;
      with_c_mode(g.cdt, g.mode, [&](auto C, auto M) {
        constexpr int CDT = decltype(C)::value, MODE = decltype(M)::value;
        const EpiScalars<float, CDT> sc = epi_scalars<float, CDT>(g.e);
        if constexpr (XT) {
          if (g.cpf) {
            eok = tc_epi_row_pf<CDT, MODE, P_BN>(g.e, sc, row, n0, tbase, lane, rl, cr, abort_flag);
            return;
          }
        }
        tc_epi_row<CDT, MODE, P_BN>(g.e, sc, row, n0, tbase, lane, stage_w, stage_w_gen);
      });
      if (!eok) {
        if (lane == 0) fail();
        break;
      }
      release(b);
    }
  } else if (XT && warp == 6 && lane == 0 && g.cpf) {
    // C loader: the old C values of every item's 32-column chunks, in the order the
    // epilogue takes them, into the ring of ncb buffers (TMA, zero past C's edges)
    uint32_t cit = 0;
    bool ok = true;
    PairItem w;
    for (int i = 0; ok && pair_item<XT>(g, ntiles, nkb, cid, ncl, i, &w); ++i) {
      int pm, tn;
      pair_coords(w.t, pairs_m, tiles_n, &pm, &tn);
      const int32_t m0 = pm * 2 * P_BM + static_cast<int32_t>(rank) * P_BM;
      const int32_t x = ((g.mode == OUT_ROWPAIR) ? m0 / 2 : m0) * g.c_rep;
      for (int c0 = 0; c0 < P_BN; c0 += 32, ++cit) {
        const int b = static_cast<int>(cit % static_cast<uint32_t>(g.ncb));
        const uint32_t use = cit / static_cast<uint32_t>(g.ncb);
        if (!mbar_wait(c_empty0 + 8u * b, (use & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        const int32_t n = tn * P_BN + c0;
        const int32_t y = (g.mode == OUT_COLPAIR) ? n / 2 : n;
        mbar_expect_tx(c_full0 + 8u * b, g.c_bytes);
        tma_load_2d(cbuf0 + static_cast<uint32_t>(b) * g.c_bytes, &mC, x, y, c_full0 + 8u * b);
      }
    }
    if (!ok) fail();
    // every copy issued has landed before the CTA may leave (the last use of each buffer)
    const uint32_t nb = static_cast<uint32_t>(g.ncb);
    for (uint32_t j = (cit > nb ? cit - nb : 0); j < cit; ++j) mbar_drain(c_full0 + 8u * (j % nb), (j / nb) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  __syncwarp();
  cluster_sync_all();   // neither CTA leaves while the other may still use its memory
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P_TMEM_COLS) : "memory");
  }
}

// Bytes of one C element (a complex element counted whole).
inline int c_elem_bytes(int cdt) {
  switch (cdt) {
    case MXG_S: return 4;
    case MXG_D: return 8;
    case MXG_H: case MXG_B: return 2;
    case MXG_C: return 8;
    case MXG_Z: return 16;
    case MXG_K: case MXG_W: return 4;
    default: return 0;
  }
}
// MXG_TC_C_PREFETCH=0 in the environment turns the C prefetch off (for measurement).
inline bool c_prefetch_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("MXG_TC_C_PREFETCH");
    return !(v && v[0] == '0' && v[1] == '\0');
  }();
  return on;
}

template <int SPLIT, int RB>
cudaError_t launch_pair(const CUtensorMap* maps, PairArgs g, int sms, void* sk_ws, size_t sk_bytes, int sk_mode,
                        cudaStream_t s) {
  auto kern_xt = tc_pair_gemm<SPLIT, RB, true>;
  auto kern_plain = tc_pair_gemm<SPLIT, RB, false>;
  cudaError_t e = cudaFuncSetAttribute(kern_xt, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM);
  if (e != cudaSuccess) return e;
  using F = PairFmt<SPLIT, RB>;
  const int64_t npairs = ((g.Mp + 2 * P_BM - 1) / (2 * P_BM)) * (g.Np / P_BN);
  const int64_t nkb = g.Kp * F::elem / RB;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(P_THREADS_XT, 1, 1);
  cfg.dynamicSmemBytes = P_SMEM;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(static_cast<unsigned>(2 * (sms / 2)), 1, 1);
  // persistent: as many pairs as can be resident at once (at most one CTA per SM)
  int max_clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&max_clusters, kern_xt, &cfg) != cudaSuccess || max_clusters <= 0) {
    cudaGetLastError();
    max_clusters = sms / 2;
  }
  const int64_t resident = std::min(max_clusters, sms / 2);
  int64_t ncl = std::min<int64_t>(npairs, resident);
  g.sk_part = nullptr; g.sk_cnt = nullptr; g.sk_full = 0; g.sk_r = 0;
  if (sk_ws && tc_pair_stream_k(npairs, nkb, resident, sk_mode) && tc_pair_stream_k_bytes(resident) <= sk_bytes) {
    ncl = resident;
    g.sk_full = static_cast<int>(npairs / ncl);
    g.sk_r = static_cast<int>(npairs % ncl);
    g.sk_part = static_cast<float4*>(sk_ws);
    g.sk_cnt = reinterpret_cast<int*>(static_cast<char*>(sk_ws) + sk_part_bytes(resident));
    e = cudaMemsetAsync(g.sk_cnt, 0, static_cast<size_t>(g.sk_r) * 8 * sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  // C prefetch: with a short k the epilogue bounds the kernel, so two operand stages
  // suffice and the rest of the span holds C chunks (as many as 24); with a long k the
  // ring keeps its stages (giving up at most two) and the rest holds two chunks or more
  CUtensorMap cmap;
  std::memset(&cmap, 0, sizeof(cmap));
  g.stages = F::stages;
  g.cpf = 0; g.ncb = 0; g.c_rows = 0; g.c_bytes = 0; g.c_rep = 1;
  const int cesz = c_elem_bytes(g.cdt);
  const int rep = (cesz > 8) ? cesz / 8 : 1;   // a double complex element is two 8-byte map elements
  // the loader pays off where the epilogue is exposed (up to 64 MMA steps per tile) or
  // where the kernel variant that has it runs anyway (stream-K tail); with long tiles
  // and no tail the whole-tile variant is faster (measured: 3% at 8192^3, TC16)
  const int64_t mma_steps = nkb * (F::planes == 2 ? 3 : 1);
  if (c_prefetch_enabled() && cesz > 0 && g.e.C && !g.e.beta_zero && g.e.rs == 1 && g.e.m > 0 && g.e.n > 0 &&
      (g.sk_r > 0 || mma_steps <= 64)) {
    const int rows = (g.mode == OUT_ROWPAIR) ? P_BM / 2 : P_BM;
    const int cols = (g.mode == OUT_COLPAIR) ? 16 : 32;
    const uint32_t cb = static_cast<uint32_t>(rows * cols * cesz);
    // a long k keeps the ring: the one-pass ring (6 stages) gives up at most two stages
    // to hold two chunks, the split forms' 3 stages none (measured: a double C on
    // TF32x3 at 4096^3 ran 14% slower with two stages)
    int stages = (nkb >= 8) ? F::stages : 2;
    const int floor_st = (nkb >= 8) ? (F::stages >= 6 ? F::stages - 2 : F::stages) : 2;
    while (stages > floor_st && P_SPAN - static_cast<uint32_t>(stages) * F::stage_bytes < 2 * cb) --stages;
    const uint32_t room = P_SPAN - static_cast<uint32_t>(stages) * F::stage_bytes;
    const int ncb = static_cast<int>(std::min<uint32_t>(P_NCB, room / cb));
    if (ncb >= 2 && tc_make_c_map(&cmap, g.e.C, cesz / rep, g.e.m * rep, g.e.n, g.e.cs * cesz,
                                  static_cast<uint32_t>(rows * rep), static_cast<uint32_t>(cols))) {
      g.stages = stages; g.cpf = 1; g.ncb = ncb; g.c_rows = rows; g.c_bytes = cb; g.c_rep = rep;
    }
  }
  if (ncl <= 0) return cudaErrorInvalidValue;
  cfg.gridDim = dim3(static_cast<unsigned>(2 * ncl), 1, 1);
  if (g.cpf || g.sk_r) {
    e = cudaLaunchKernelEx(&cfg, kern_xt, maps[0], maps[1], maps[2], maps[3], cmap, g);
  } else {
    cfg.blockDim = dim3(P_THREADS, 1, 1);
    e = cudaLaunchKernelEx(&cfg, kern_plain, maps[0], maps[1], maps[2], maps[3], cmap, g);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The instantiations, one translation unit per operand format (their compile time is
// dominated by the epilogue's 16 C datatype / output mode pairs, in two kernel variants):
// binary16 in gemm_tc2.cu, bfloat16 in gemm_tc2_bf16one.cu, the split formats in
// gemm_tc2_tf32.cu and gemm_tc2_bf16.cu.
cudaError_t launch_pair_f16(const CUtensorMap* maps, const PairArgs& g, int sms, void* sk_ws, size_t sk_bytes,
                            int sk_mode, cudaStream_t s);
cudaError_t launch_pair_bf16_one(const CUtensorMap* maps, const PairArgs& g, int sms, void* sk_ws,
                                 size_t sk_bytes, int sk_mode, cudaStream_t s);
cudaError_t launch_pair_tf32(const CUtensorMap* maps, const PairArgs& g, int sms, void* sk_ws, size_t sk_bytes,
                             int sk_mode, cudaStream_t s);
cudaError_t launch_pair_bf16(const CUtensorMap* maps, const PairArgs& g, int sms, void* sk_ws, size_t sk_bytes,
                             int sk_mode, cudaStream_t s);

}  // namespace pairk
}  // namespace mxg
