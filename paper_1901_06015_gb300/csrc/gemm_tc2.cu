// Tensor-core contraction on CTA pairs: host side (the stream-K decision and workspace,
// tensor maps, dispatch) and the kernels of the one-pass binary16 format. The kernel
// itself is in tc_pair.cuh; the other formats' instantiations are in gemm_tc2_*.cu.
#include "tc_pair.cuh"

namespace mxg {

using namespace pairk;

namespace pairk {

cudaError_t launch_pair_f16(const CUtensorMap* maps, const PairArgs& g, int sms, void* sk_ws, size_t sk_bytes,
                            int sk_mode, cudaStream_t s) {
  return launch_pair<SPLIT_F16_ONE, P_RB>(maps, g, sms, sk_ws, sk_bytes, sk_mode, s);
}

}  // namespace pairk

bool tc_pair_stream_k(int64_t tiles, int64_t nkb, int64_t pairs, int mode) {
  if (mode <= 0 || tiles <= 0 || nkb <= 0 || pairs <= 0) return false;
  const int64_t r = tiles % pairs;
  // every pair's range must hold at least one k-block (a tile's ranges are then the
  // consecutive pairs c_first .. c_last, each taking one ticket)
  if (r == 0 || r * nkb < pairs) return false;
  if (mode >= 2) return true;
  // automatic: the pairs idle in the last wave are at least 6% of the whole run, and
  // every range holds at least 16 k-blocks (measured on GB300: with 13.5 waves of
  // short tiles the partial sums cost more than the idle share they recover)
  const int64_t full = tiles / pairs;
  return 100 * (pairs - r) >= 6 * pairs * (full + 1) && r * nkb >= 16 * pairs;
}

size_t tc_pair_stream_k_bytes(int64_t pairs) {
  return pairs <= 0 ? 0 : sk_part_bytes(pairs) + ((static_cast<size_t>(pairs) * 8 * sizeof(int) + 255) & ~size_t(255));
}

size_t tc_pair_stream_k_workspace(int split, int64_t Mp, int64_t Np, int64_t Kp, int sm_count, int mode) {
  const int64_t elem = (split == SPLIT_TF32) ? 4 : 2;
  const int64_t pairs = (sm_count > 0 ? sm_count : 152) / 2;
  const int64_t tiles = ((Mp + 2 * P_BM - 1) / (2 * P_BM)) * (Np / P_BN);
  return tc_pair_stream_k(tiles, Kp * elem / P_RB, pairs, mode) ? tc_pair_stream_k_bytes(pairs) : 0;
}

// planes: A_hi, A_lo (Mp x Kp, K-major), B_hi, B_lo (Np x Kp, K-major); one plane per
// operand for the one-pass formats (the lo entries are ignored)
cudaError_t launch_gemm_tc_pair(int split, int c_dt, int mode, const void* const planes[4], int64_t Mp, int64_t Np,
                                int64_t Kp, const EpiArgs& e, int* err, void* sk_ws, size_t sk_bytes, int sk_mode,
                                cudaStream_t s) {
  if (!tc_get_encoder()) return cudaErrorNotSupported;
  const int elem = (split == SPLIT_TF32) ? 4 : 2;
  if (Mp % P_BM || Np % P_BN || (Kp * elem) % P_RB) return cudaErrorInvalidValue;
  if (Mp == 0 || Np == 0) return cudaSuccess;
  if (((Mp + 2 * P_BM - 1) / (2 * P_BM)) * (Np / P_BN) > 0x7fffffffLL) return cudaErrorInvalidValue;
  int sms = 0;
  const cudaError_t ce = tc_current_sm_count(&sms);
  if (ce != cudaSuccess) return ce;
  if (sms < 2) return cudaErrorNotSupported;
  CUtensorMap maps[4];
  if (!tc_make_map(&maps[0], planes[0], split, Mp, Kp, P_BM, P_RB) ||
      !tc_make_map(&maps[1], planes[1], split, Mp, Kp, P_BM, P_RB) ||
      !tc_make_map(&maps[2], planes[2], split, Np, Kp, P_BN / 2, P_RB) ||
      !tc_make_map(&maps[3], planes[3], split, Np, Kp, P_BN / 2, P_RB))
    return cudaErrorInvalidValue;
  PairArgs g{Mp, Np, Kp, e, c_dt, mode, err, nullptr, nullptr, 0, 0};
  bool valid = false;
  with_c_mode(c_dt, mode, [&](auto, auto) { valid = true; });
  if (!valid) return cudaErrorInvalidValue;
  switch (split) {
    case SPLIT_TF32: return launch_pair_tf32(maps, g, sms, sk_ws, sk_bytes, sk_mode, s);
    case SPLIT_BF16: return launch_pair_bf16(maps, g, sms, sk_ws, sk_bytes, sk_mode, s);
    case SPLIT_F16_ONE: return launch_pair_f16(maps, g, sms, sk_ws, sk_bytes, sk_mode, s);
    case SPLIT_BF16_ONE: return launch_pair_bf16_one(maps, g, sms, sk_ws, sk_bytes, sk_mode, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mxg
