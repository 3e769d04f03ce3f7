// rf_sweep_stream.h -- internal interface of the streamed forward sweep
// (rf_sweep_stream.cu), used by rf_sweep_forward.
#pragma once

#include "rf_ctx.h"
#include "rf_sweep_common.cuh"

namespace rf {

struct StreamPlan {
  int R, K, grid, threads;
  size_t smem;
  const void *kernel;
};

// Pick the compiled shape closest to the requested (R, K) (0 = default)
// and check that it fits the device (shared memory, co-resident CTAs).
rf_status stream_plan(rf_ctx *ctx, int ny, int nx, int R, int K, StreamPlan *pl);

// float4 elements of the node-record buffer (both orientations).
size_t stream_record_floats4(int ny, int nx);

// Node records of every node, both orientations, into recbuf.
rf_status stream_records(int ny, int nx, float h, float eps, const float *proj5, const uint8_t *src,
                         float4 *recbuf, cudaStream_t s);

// One cooperative launch running every sweep of the solve.
rf_status stream_launch(const StreamPlan &pl, int ny, int nx, const float4 *recbuf, float *T, float *Tb,
                        int max_sweeps, float tol, float rtol, unsigned *progress, int *changed,
                        const LaunchCtl &ctl, cudaStream_t s);

}  // namespace rf
