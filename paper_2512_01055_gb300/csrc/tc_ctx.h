// The context behind the opaque tc_ctx handle of include/tc.h (internal).
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tc {

// Grow-only device buffer: re-allocated only when a larger size is needed, so
// repeated calls reuse the same memory.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) { cudaFree(p); p = nullptr; cap = 0; }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes; else p = nullptr;
    return e;
  }
  void release() { if (p) cudaFree(p); p = nullptr; cap = 0; }
};

struct Server;                              // serving engine (tc_serve.cu)
void server_destroy(Server *s);

}  // namespace tc

struct tc_ctx {
  int device = 0;
  size_t budget = 0;
  int default_prec = TC_FP64;
  int default_slices = 3;
  int timeout_ms = 60000;
  int max_inflight = 16;
  int max_queue = 4096;
  int iteration_ms = 50;
  int num_sms = 0;
  std::mutex mu;                            // serialises the blocking entry points
  std::string err;
  cudaStream_t stream = nullptr;
  tc::DevBuf ws;                            // tables, partials and sums, reused across calls
  tc::DevBuf ws_split;                      // BF16 operand images, FP32 copies, W buffer
  tc::DevBuf in_eps, in_t1, in_t2, in_ovvv, in_ovoo, in_ovov;   // tc_energy's device copies; tc_energy_df_dev's integrals
  tc::DevBuf df_b;                          // tc_energy_df(_dev): scratch of the integral assembly (scales, digit images)
  tc::DevBuf df_in;                         // tc_energy_df: the device copy of B
  cudaEvent_t dfev[2] = {nullptr, nullptr}; // around the integral assembly
  double *host_out = nullptr;               // pinned read-back slot
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};     // kernel timing
  std::vector<cudaEvent_t> wev;             // split path: a pair around each W-term launch (grown on demand)
  cudaStream_t copy_stream = nullptr;       // tc_energy: host-to-device copies of the inputs, by occupied-index chunk
  std::vector<cudaEvent_t> cev;             // tc_energy: one per chunk, recorded on copy_stream after its copies
  std::vector<cudaEvent_t> pev;             // staged split path: a pair around each chunk's slicing
  std::mutex serve_mu;                      // guards creation of the serving engine
  tc::Server *server = nullptr;
};
