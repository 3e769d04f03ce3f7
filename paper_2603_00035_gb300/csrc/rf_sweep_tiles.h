// rf_sweep_tiles.h -- internal interface of the tile-queue forward solve
// (rf_sweep_tiles.cu), used by rf_sweep_forward.
#pragma once

#include "rf_ctx.h"
#include "rf_sweep_common.cuh"

namespace rf {

// Per-solve workspace of the tile queue (one device allocation, carved).
struct TileWork {
  unsigned long long *counters;  // [0] node updates, [1] warp evaluations
  unsigned *ctrl;                // round slots (count, grab, kmin, pad) x 3, mean edge cost, its sum
  unsigned *tstate;              // per tile: (round last written << 1) | buffer parity
  unsigned *visits;              // per tile: visits so far
  unsigned *queued;              // per tile: last round it was queued for
  unsigned *key;                 // [2][tiles] float bits of the queue key, by round parity
  int *list;                     // [3][tiles] queued tiles, by round mod 3
  float *halo;                   // [tiles][4 * ts + 4] halo seen at the previous visit
};

// Tile side used for a requested one (0 or < 32: 16; >= 32: 32).
int tile_side(int requested);
int tiles_count(int ny, int nx, int ts);
size_t tile_work_bytes(int ny, int nx, int ts);
TileWork tile_work_carve(void *base, int ny, int nx, int ts);

// Seed the queue and run the whole solve in one cooperative launch.  T holds
// the initial state (init_kernel) and receives the result; Tb is a second
// buffer of ny * nx floats.  ts: tile side (16 or 32); window:
// delta-stepping window in tile crossings (<= 0: 2).
rf_status tiles_launch(int num_sms, int ny, int nx, int ts, float h, float eps, const float *proj5,
                       const uint8_t *src, float *T, float *Tb, int warm, int max_sweeps, float tol, float rtol,
                       float window, const TileWork &w, const LaunchCtl &ctl, cudaStream_t s);

}  // namespace rf
