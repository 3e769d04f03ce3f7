// rf_ctx.h -- internal definition of rf_ctx (the library's workspace) and
// helpers shared by the entry points.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rf.h"
#include "rf_device.cuh"

struct rf_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t last_stream = nullptr;
  rf::DevState *state = nullptr;  // device status word and counters
  long long timeout_ns = 2000000000LL;  // bound of every device wait
  long long adj_park_ns = 2000000;      // RF_ADJ_TILES: stall before a tile yields its CTA

  // grown on demand
  unsigned *progress = nullptr;  // per-band progress tokens
  size_t progress_cap = 0;
  int *changed = nullptr;  // per-sweep changed flags
  size_t changed_cap = 0;
  float *tbuf = nullptr;  // second buffer of the ping-pong sweeps
  size_t tbuf_cap = 0;
  float *lbuf = nullptr;  // adjoint: lambda ping-pong buffers
  size_t lbuf_cap = 0;
  void *scratch = nullptr;  // adjoint (ordered): sort keys/values/temp
  size_t scratch_cap = 0;
  unsigned long long *adj_state = nullptr;  // adjoint (ordered): (epoch << 32 | lambda bits)
  size_t adj_state_cap = 0;
  unsigned adj_epoch = 0;  // host count of adjoint launches (the tag itself: DevState::adj_epoch)
  float4 *recbuf = nullptr;  // streamed sweep: node records, both orientations
  size_t recbuf_cap = 0;
  float *tvbuf = nullptr;  // total variation: per-block partial sums
  size_t tvbuf_cap = 0;
  unsigned char *tilebuf = nullptr;  // tile-queue solve: queue, tile states, halos
  size_t tilebuf_cap = 0;
  uint16_t *wpack = nullptr;  // tcgen05 convolution: BF16 weights in the order its stages hold them
  size_t wpack_cap = 0;
  unsigned char *stepbuf = nullptr;  // rf_step_host: two input/output sets and the intermediates
  size_t stepbuf_cap = 0;
  cudaStream_t step_in = nullptr, step_out = nullptr;  // rf_step_host: copy streams (created on first use)
  cudaEvent_t step_ev[6] = {};                         // rf_step_host: in / done / out per set
};

namespace rf {

inline rf_status cuda_status(cudaError_t e) {
  return e == cudaSuccess ? RF_OK : RF_ERR_CUDA;
}

template <class T>
inline rf_status ensure(T **ptr, size_t *cap, size_t count) {
  if (*cap >= count && *ptr) return RF_OK;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  size_t n = count < 1 ? 1 : count;
  if (cudaMalloc((void **)ptr, n * sizeof(T)) != cudaSuccess) {
    *ptr = nullptr;
    return RF_ERR_NO_MEMORY;
  }
  *cap = n;
  return RF_OK;
}

inline bool grid_ok(const rf_grid *g) {
  return g && g->ny >= 1 && g->nx >= 1 && g->h > 0.0f &&
         (long long)g->ny * (long long)g->nx < (1LL << 31);
}

inline int blocks_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

}  // namespace rf
