// The handle behind mxg_handle (internal).
#pragma once

#include <mutex>
#include <vector>

#include <cuda_runtime.h>

struct mxg_context {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = true;
  int* dev_err = nullptr;
  bool timing = false;
  bool literal_alpha = false;
  int split_k = 0;
  int cta_pairs = 0;
  int stream_k = 1;
  int sm_count = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<cudaEvent_t> ev_rec;   // triples: before packs, before contraction, after
  std::mutex mu;
};

inline cudaEvent_t take_event(mxg_context* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

inline void recycle_events(mxg_context* h) {
  for (cudaEvent_t e : h->ev_rec) h->ev_pool.push_back(e);
  h->ev_rec.clear();
}

