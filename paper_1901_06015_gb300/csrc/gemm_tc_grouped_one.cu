// Tensor-core contraction on one CTA per tile: the grouped (many-problem) kernels of the one-pass formats, in a translation unit of
// their own. The kernel is in tc_single.cuh.
#include "tc_single.cuh"

namespace mxg {
namespace tcs {

cudaError_t launch_grouped_one(int split, const TcGroupProb* probs, const GroupTile* tiles, int ntiles, int* err,
                               int grid, cudaStream_t s) {
  switch (split) {
    case SPLIT_F16_ONE: return launch_grouped<SPLIT_F16_ONE>(probs, tiles, ntiles, err, grid, s);
    case SPLIT_BF16_ONE: return launch_grouped<SPLIT_BF16_ONE>(probs, tiles, ntiles, err, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace tcs
}  // namespace mxg
