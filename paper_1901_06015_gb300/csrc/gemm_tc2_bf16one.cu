// Tensor-core contraction on CTA pairs: the kernels of the one-pass bfloat16 format, in a translation
// unit of their own. The kernel is in tc_pair.cuh.
#include "tc_pair.cuh"

namespace mxg {
namespace pairk {

cudaError_t launch_pair_bf16_one(const CUtensorMap* maps, const PairArgs& g, int sms, void* sk_ws, size_t sk_bytes,
                                 int sk_mode, cudaStream_t s) {
  return launch_pair<SPLIT_BF16_ONE, P_RB>(maps, g, sms, sk_ws, sk_bytes, sk_mode, s);
}

}  // namespace pairk
}  // namespace mxg
