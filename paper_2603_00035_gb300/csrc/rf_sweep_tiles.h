// rf_sweep_tiles.h -- internal interface of the tile-queue forward solve
// (rf_sweep_tiles.cu), used by rf_sweep_forward and rf_batch_solve.
#pragma once

#include "rf_ctx.h"
#include "rf_sweep_common.cuh"

namespace rf {

// Per-grid tile geometry (device, written by the plan kernels).
struct TGrid {
  long long node_off;  // first node of the grid in the packed arrays
  int ny, nx;          // grid shape
  int tny, tnx;        // tiles along y and x
  int tile_off;        // first tile of the grid
  float h;             // spacing
  float inv_scale;     // 1 / (tile side x mean edge cost): keys in tile crossings
  int has_src;         // the grid holds a source node
  unsigned long long esum_fx;  // sum of the edge costs (seed), fixed point (2^-32), order-independent
};
// (copied into each tile group's shared memory per visit: keep it 48 bytes)
static_assert(sizeof(TGrid) == 48, "TGrid layout");

// Per-solve workspace of the tile queue (one device allocation, carved).
struct TileWork {
  unsigned long long *counters;  // [0] node updates, [1] warp evaluations
  unsigned *ctrl;                // round slots x 8, tile count, completed round, stop flag, rounds
  TGrid *grids;                  // [grids]
  unsigned long long *gupd;      // [grids] node updates per grid
  unsigned long long *list;      // [8][tiles cap] queued tiles (round << 32 | tile), by round mod 8
  unsigned *tstate;              // per tile: (round last written << 9) | (buffer parity << 8) | pending rounds
                                 // (bit r mod 8: queued for round r and not yet done)
  unsigned *visits;              // per tile: visits so far
  unsigned *key;                 // [4][tiles cap] float bits of the queue key, by round mod 4
  int *tile_grid;                // [tiles cap] grid of each tile (batches)
  float *halo;                   // [tiles cap][4 * ts + 4] halo seen at the previous visit
};

// What one tile-queue solve needs (a single grid: descs = NULL and ny, nx,
// h; a batch: the device descriptors and max_line).
struct TileLaunch {
  int num_sms;
  int ts;                        // tile side, 16 or 32
  int n_grids;
  const rf_batch_desc *descs;    // batch descriptors (device) or NULL
  int ny, nx;                    // single grid
  float h;                       // single grid
  int max_line;                  // max over grids of max(ny, nx)
  long long total_nodes;
  int ntiles_cap;
  float eps;
  const float *proj5;
  const uint8_t *src;
  float *T, *Tb;
  int warm, max_sweeps;
  float tol, rtol, window;
  float tau;                     // > 0: the soft-min relaxation instead of the minimum
  int *grid_status;              // batch: [3 * grids] status, forward sweep equivalent (adjoint left alone)
};

// Initial state of a solve (rf_sweep.cu): T = 0 on sources, +inf elsewhere
// (cold) or the caller's guess (warm); *has_src |= 1 when a source exists.
void init_state(float *T, const uint8_t *src, long long n, int warm, DevState *st, int *has_src, int num_sms,
                cudaStream_t s);
// RF_ERR_NO_SOURCE in the status word when *has_src is 0 (after init_state).
void check_source_flag(const int *has_src, DevState *st, cudaStream_t s);

// Tile side used for a requested one (0 or < 32: 16; >= 32: 32).
int tile_side(int requested);
// Upper bound of the tile count of a batch (exact for one grid up to edge
// tiles).
int tiles_cap(int n_grids, long long total_nodes, int max_line, int ts);
size_t tile_work_bytes(int n_grids, int ntiles_cap, int ts);
TileWork tile_work_carve(void *base, int n_grids, int ntiles_cap, int ts);

// Plan and seed the queue, then run the whole solve in one cooperative
// launch.  T holds the initial state (init_kernel) and receives the result;
// Tb is a second buffer of total_nodes floats.
rf_status tiles_launch(const TileLaunch &L, const TileWork &w, const LaunchCtl &ctl, cudaStream_t s);

}  // namespace rf
