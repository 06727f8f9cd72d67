// Device work lists and launchers of the grouped persistent launch.
#pragma once

#include <cuda.h>

#include <vector>

#include "mxg_internal.h"

namespace mxg {

// Contraction kernels a bucket of the group may run (tile size in brackets).
enum GroupVariant : int {
  VAR_FFMA_128 = 0,   // FP32 FFMA, 128 x 128
  VAR_FFMA_64 = 1,    // FP32 FFMA, 64 x 64
  VAR_DFMA_64 = 2,    // FP64 DFMA, 64 x 64
  VAR_DFMA_32 = 3,    // FP64 DFMA, 32 x 32
  VAR_DMMA_64 = 4,    // FP64 DMMA, 64 x 64
  VAR_FFMA_32 = 5,    // FP32 FFMA, 32 x 32
  VAR_DFMA_16 = 6     // FP64 DFMA, 16 x 16 (64-thread CTAs)
};
constexpr int VAR_COUNT = 7;

// Tile schedules of the persistent kernels: DYNAMIC takes the next entry of the
// (longest-first) work list from an atomic counter; STATIC gives CTA b the entries
// b, b + grid, b + 2 grid, ...
enum GroupSched : int { SCHED_DYNAMIC = 0, SCHED_STATIC = 1 };

struct GroupProb {
  const void* A;       // packed A' of the problem (MN-major)
  const void* B;       // packed B'
  int64_t lda, ldb;    // padded M', N'
  int64_t Kp;          // padded K'
  EpiArgs e;           // epilogue of the problem
  int cdt, mode;       // C datatype, output mode
};

struct GroupTile {
  int prob;            // index into the problem array
  int tm, tn;          // tile coordinates in units of the variant's tile
};

// One problem of a tensor-core bucket (TF32X3, BF16X3 or TC16): the tensor maps of its
// K-major planes (A hi, A lo, B hi, B lo; the one-plane formats repeat the hi maps),
// encoded on the host, and its epilogue. Tiles are 128 x 256.
struct alignas(64) TcGroupProb {
  CUtensorMap maps[4];
  int64_t Mp, Np, Kp;  // padded real problem
  EpiArgs e;
  int cdt, mode;
};

#ifdef __CUDACC__
// Fetch the next work-list index for the whole CTA (dynamic schedule: one atomic per
// tile on the bucket's counter; static schedule: CTA b takes b, b + grid, ...).
__device__ __forceinline__ int next_tile(int* counter, int* slot, int prev, int sched) {
  if (sched == SCHED_STATIC) return prev < 0 ? static_cast<int>(blockIdx.x) : prev + static_cast<int>(gridDim.x);
  __syncthreads();
  if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
  __syncthreads();
  return *slot;
}

#endif

int variant_tile(int variant);

struct Plan;
// The grouped-launch description of one planned problem (PLAN_GEMM on the SIMT / DMMA
// layout) whose packed operands start at pa (A' then B'): its GroupProb and its two
// pack tasks.
// dbg: error word of the debug builds' bounds checks (may be null).
void group_describe_problem(const Plan& P, char* pa, GroupProb* gp, PackArgs* ta, PackArgs* tb, int* dbg);
// Work list of (problem, tile) for a variant, ordered longest-K' first.
std::vector<GroupTile> group_tiles(const std::vector<GroupProb>& probs, int variant);
cudaError_t launch_dmma(int mode, int cdt, const GemmArgs& g, cudaStream_t s, dim3 grid);
cudaError_t launch_dmma_grouped(const GroupProb* probs, const GroupTile* tiles, int ntiles, int* counter, int sched,
                                int grid, cudaStream_t s);
int dmma_grouped_blocks_per_sm();
cudaError_t launch_dmma_partial(const GemmArgs& g, int64_t kslice, double* ws, dim3 grid, cudaStream_t s);
int grouped_blocks_per_sm(int variant);
cudaError_t launch_gemm_grouped(int variant, const GroupProb* probs, const GroupTile* tiles, int ntiles,
                                int* counter, int sched, int grid, cudaStream_t s);
int64_t pack_tiles(const PackArgs& a);
// Grouped pack into the K-major planes of one tensor-core format (SplitKind).
cudaError_t launch_pack_grouped_tc(const PackArgs* tasks, const int64_t* tile_start, int ntasks, int64_t ntiles,
                                   int split, cudaStream_t s);
// Encode the four maps of a tensor-core problem (planes as for launch_gemm_tc).
bool tc_group_problem(TcGroupProb* p, int split, const void* const planes[4], int64_t Mp, int64_t Np, int64_t Kp,
                      const EpiArgs& e, int cdt, int mode);
// Persistent tcgen05 contraction over a bucket's work list (static schedule, 128 x 256
// tiles, one CTA per SM); err: the device error word for wait timeouts.
cudaError_t launch_gemm_tc_grouped(int split, const TcGroupProb* probs, const GroupTile* tiles, int ntiles, int* err,
                                   cudaStream_t s);
cudaError_t launch_pack_grouped(const PackArgs* tasks, const int64_t* tile_start, int ntasks, int64_t ntiles,
                                int comp_double, cudaStream_t s);

}  // namespace mxg
