// Tensor-core contraction on one CTA per tile: the single-problem kernels of the one-pass binary16 and bfloat16 formats, in a translation unit of
// their own. The kernel is in tc_single.cuh.
#include "tc_single.cuh"

namespace mxg {
namespace tcs {

cudaError_t launch_single_one(int split, const CUtensorMap* maps, const TcArgs& g, int sms, cudaStream_t s) {
  switch (split) {
    case SPLIT_F16_ONE: return launch_one<SPLIT_F16_ONE>(maps, g, sms, s);
    case SPLIT_BF16_ONE: return launch_one<SPLIT_BF16_ONE>(maps, g, sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace tcs
}  // namespace mxg
