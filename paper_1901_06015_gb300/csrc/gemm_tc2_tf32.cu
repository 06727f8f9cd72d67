// Tensor-core contraction on CTA pairs: the kernels of the TF32x3 split format, in a translation
// unit of their own. The kernel is in tc_pair.cuh.
#include "tc_pair.cuh"

namespace mxg {
namespace pairk {

cudaError_t launch_pair_tf32(const CUtensorMap* maps, const PairArgs& g, int sms, void* sk_ws, size_t sk_bytes,
                             int sk_mode, cudaStream_t s) {
  return launch_pair<SPLIT_TF32, P_RB>(maps, g, sms, sk_ws, sk_bytes, sk_mode, s);
}

}  // namespace pairk
}  // namespace mxg
