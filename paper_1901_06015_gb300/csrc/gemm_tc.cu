// Tensor-core contraction on one CTA per tile (tcgen05, sm_103a): host side (tensor-map
// encoder and maps, SM count, dispatch), the wait-limit self-test, and the kernels of
// the split formats. The kernel itself is in tc_single.cuh.
#include <atomic>
#include <mutex>

#include "tc_single.cuh"

namespace mxg {

using namespace tcs;

namespace tcs {

cudaError_t launch_single_split(int split, const CUtensorMap* maps, const TcArgs& g, int sms, cudaStream_t s) {
  switch (split) {
    case SPLIT_TF32: return launch_one<SPLIT_TF32>(maps, g, sms, s);
    case SPLIT_BF16: return launch_one<SPLIT_BF16>(maps, g, sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace tcs

namespace {

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing will
// arrive on, for at most limit_ns, then records the timeout in the error word.
__global__ void wait_timeout_probe(int* err, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const unsigned long long t0 = gtimer();
  while (!mbar_try(b, 0)) {
    if (gtimer() - t0 > limit_ns) {
      atomicExch(err, 1);
      return;
    }
  }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
// SM count per device, filled on first use with that device current (several host
// threads may race to fill an entry; they store the same value)
constexpr int kMaxDevices = 64;
std::atomic<int> g_sms[kMaxDevices];

cudaError_t current_sm_count(int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int v = g_sms[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (v <= 0) return cudaErrorInvalidValue;
    g_sms[dev].store(v, std::memory_order_relaxed);
  }
  *out = v;
  return cudaSuccess;
}

bool get_encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  });
  return g_encode != nullptr;
}

// 2-D map over a K-major plane (rows x Kp elements, row pitch Kp elements), box
// (rows_box x 64 bytes), 64-byte swizzle.
bool make_map(CUtensorMap* map, const void* ptr, int split, int64_t rows, int64_t Kp, uint32_t rows_box,
              uint32_t rowb = ROWB) {
  const int elem = (split == SPLIT_TF32) ? 4 : 2;
  const CUtensorMapDataType dtype = (split == SPLIT_TF32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                    : (split == SPLIT_F16_ONE) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(Kp), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(Kp) * elem};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(rowb / elem), rows_box};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = g_encode(map, dtype, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool tc_get_encoder() { return get_encoder(); }
bool tc_make_map(CUtensorMap* map, const void* ptr, int split, int64_t rows, int64_t Kp, uint32_t rows_box,
                 uint32_t rowb) {
  return make_map(map, ptr, split, rows, Kp, rows_box, rowb);
}
cudaError_t tc_current_sm_count(int* out) { return current_sm_count(out); }

bool tc_make_c_map(CUtensorMap* map, const void* C, int esz, int64_t rows, int64_t cols, int64_t ld_bytes,
                   uint32_t box_rows, uint32_t box_cols) {
  if (!get_encoder() || !C || rows <= 0 || cols <= 0) return false;
  if ((reinterpret_cast<uintptr_t>(C) & 15u) || (ld_bytes & 15) || ld_bytes < rows * esz) return false;
  if ((box_rows * static_cast<uint32_t>(esz)) % 16u || box_rows > 256 || box_cols > 256) return false;
  const CUtensorMapDataType dtype = (esz == 2)   ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                    : (esz == 4) ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                    : (esz == 8) ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                                 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  if (esz != 2 && esz != 4 && esz != 8) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(cols)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld_bytes)};
  const cuuint32_t box[2] = {box_rows, box_cols};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = g_encode(map, dtype, 2, const_cast<void*>(C), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_group_problem(TcGroupProb* p, int split, const void* const planes[4], int64_t Mp, int64_t Np, int64_t Kp,
                      const EpiArgs& e, int cdt, int mode) {
  if (!get_encoder()) return false;
  const int bk = static_cast<int>(ROWB) / (split == SPLIT_TF32 ? 4 : 2);
  if (Mp % TC_BM || Np % TC_BN || Kp % bk || Mp <= 0 || Np <= 0 || Kp <= 0) return false;
  if (!make_map(&p->maps[0], planes[0], split, Mp, Kp, TC_BM) || !make_map(&p->maps[1], planes[1], split, Mp, Kp, TC_BM) ||
      !make_map(&p->maps[2], planes[2], split, Np, Kp, TC_BN) || !make_map(&p->maps[3], planes[3], split, Np, Kp, TC_BN))
    return false;
  p->Mp = Mp; p->Np = Np; p->Kp = Kp;
  p->e = e;
  p->cdt = cdt;
  p->mode = mode;
  bool valid = false;
  with_c_mode(cdt, mode, [&](auto, auto) { valid = true; });
  return valid;
}

cudaError_t launch_gemm_tc_grouped(int split, const TcGroupProb* probs, const GroupTile* tiles, int ntiles, int* err,
                                   cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  int sms = 0;
  cudaError_t e = current_sm_count(&sms);
  if (e != cudaSuccess) return e;
  const int grid = ntiles < sms ? ntiles : sms;
  switch (split) {
    case SPLIT_TF32: case SPLIT_BF16: return launch_grouped_split(split, probs, tiles, ntiles, err, grid, s);
    case SPLIT_F16_ONE: case SPLIT_BF16_ONE: return launch_grouped_one(split, probs, tiles, ntiles, err, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_wait_timeout_probe(int* err, double seconds, cudaStream_t s) {
  wait_timeout_probe<<<1, 32, 0, s>>>(err, static_cast<unsigned long long>(seconds * 1e9));
  return cudaGetLastError();
}

// planes: A_hi, A_lo (Mp x Kp, K-major), B_hi, B_lo (Np x Kp, K-major)
cudaError_t launch_gemm_tc(int method, int split, int c_dt, int mode, const void* const planes[4], int64_t Mp,
                           int64_t Np, int64_t Kp, const EpiArgs& e, int* err, cudaStream_t s) {
  if (!get_encoder()) return cudaErrorNotSupported;
  (void)method;
  const int bk = static_cast<int>(ROWB) / (split == SPLIT_TF32 ? 4 : 2);
  if (Mp % TC_BM || Np % TC_BN || Kp % bk) return cudaErrorInvalidValue;
  if ((Mp / TC_BM) * (Np / TC_BN) > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (Mp == 0 || Np == 0) return cudaSuccess;
  int sms = 0;
  const cudaError_t ce = current_sm_count(&sms);
  if (ce != cudaSuccess) return ce;
  CUtensorMap maps[4];
  if (!make_map(&maps[0], planes[0], split, Mp, Kp, TC_BM) || !make_map(&maps[1], planes[1], split, Mp, Kp, TC_BM) ||
      !make_map(&maps[2], planes[2], split, Np, Kp, TC_BN) || !make_map(&maps[3], planes[3], split, Np, Kp, TC_BN))
    return cudaErrorInvalidValue;
  TcArgs g{Mp, Np, Kp, e, c_dt, mode, err};
  bool valid = false;
  with_c_mode(c_dt, mode, [&](auto, auto) { valid = true; });
  if (!valid) return cudaErrorInvalidValue;
  switch (split) {
    case SPLIT_TF32: case SPLIT_BF16: return launch_single_split(split, maps, g, sms, s);
    case SPLIT_F16_ONE: case SPLIT_BF16_ONE: return launch_single_one(split, maps, g, sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mxg
