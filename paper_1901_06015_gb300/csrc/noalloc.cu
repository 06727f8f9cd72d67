// mxgemm_noalloc: the plain mixed-datatype gemm for callers that must not allocate
// device memory. Some callers cannot call cudaMalloc: latency-critical loops that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree, and
// applications whose device memory is all owned by another allocator (a framework's
// caching pool, an embedded runtime with a fixed memory plan) that forbids side
// allocations. This entry point runs the same pack and contraction kernels as
// mxgemm_ex, but its packed operands live in one fixed, file-scope device array of
// MXG_NOALLOC_SCRATCH_BYTES bytes instead of a cudaMalloc'd workspace, and the error
// word its tensor-core kernels set on a wait timeout is a file-scope device int.
#include <mutex>

#include "plan.h"
#include "../../include/mxgemm.h"

namespace mxg {
extern thread_local int g_last_cuda_error;
}

using namespace mxg;

// The fixed scratch: every GPU that loads this code holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MXG_NOALLOC_SCRATCH_BYTES];
// Error word of this entry point: a bounded device-side wait that runs out sets it to 1
// (the kernel then skips its stores); it stays set until
// mxgemm_noalloc_check_device_error reads and clears it.
static __device__ int g_noalloc_err;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
int* g_noalloc_err_ptr[kMaxDevices] = {};

int noalloc_cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MXG_OK;
  g_last_cuda_error = static_cast<int>(e);
  return MXG_ECUDA;
}

// Device addresses of the scratch array and the error word on the current device. The
// name of a __device__ variable in host code is only a host-side stand-in, so the
// addresses are looked up once per device, with that device current, and cached.
int scratch_address(void** out, int** err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_cuda_status(e);
  if (dev < 0 || dev >= kMaxDevices) return MXG_EINVAL;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_err);
    if (e != cudaSuccess || p == nullptr || q == nullptr)
      return noalloc_cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
    g_noalloc_err_ptr[dev] = static_cast<int*>(q);
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  *err = g_noalloc_err_ptr[dev];
  return MXG_OK;
}
}  // namespace

extern "C" int mxgemm_noalloc(void* stream, int method, int transa, int transb,
                              int64_t m, int64_t n, int64_t k,
                              double alpha_re, double alpha_im,
                              const void* A, int dtA, int64_t rsA, int64_t csA,
                              const void* B, int dtB, int64_t rsB, int64_t csB,
                              double beta_re, double beta_im,
                              void* C, int dtC, int64_t rsC, int64_t csC, int comp_prec) {
  Call c{};
  c.transa = transa; c.transb = transb; c.m = m; c.n = n; c.k = k;
  c.alpha_re = alpha_re; c.alpha_im = alpha_im; c.beta_re = beta_re; c.beta_im = beta_im;
  c.A = A; c.dtA = dtA; c.rsA = rsA; c.csA = csA;
  c.B = B; c.dtB = dtB; c.rsB = rsB; c.csB = csB;
  c.C = C; c.dtC = dtC; c.rsC = rsC; c.csC = csC; c.comp = comp_prec;
  Plan P;
  int st = make_plan(c, method, &P);
  if (st != MXG_OK) return st;
  if (P.kind == PLAN_NOOP) return MXG_OK;
  if (!C) return MXG_EINVAL;
  if (P.kind == PLAN_GEMM && (!A || !B)) return MXG_EINVAL;
  if (P.kind == PLAN_GEMM && P.workspace > static_cast<size_t>(MXG_NOALLOC_SCRATCH_BYTES))
    return MXG_ESCRATCH;
  void* ws = nullptr;
  int* err = nullptr;
  st = scratch_address(&ws, &err);
  if (st != MXG_OK) return st;
  // The pack kernels write every byte of the padded packed operands (zeros included),
  // so nothing left in the scratch by an earlier call needs clearing. The error word is
  // only ever set by a kernel and cleared by the check below.
  return enqueue_plan(P, ws, static_cast<cudaStream_t>(stream), nullptr, err);
}

extern "C" int mxgemm_noalloc_check_device_error(void* stream, int* flag) {
  if (!flag) return MXG_EINVAL;
  void* ws = nullptr;
  int* err = nullptr;
  int st = scratch_address(&ws, &err);
  if (st != MXG_OK) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && v) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess && v) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_cuda_status(e);
  }
  *flag = v;
  return MXG_OK;
}
