// rf_adjoint.h -- internal interface of the ordered adjoint (rf_adjoint.cu)
// and of the tiled adjoint (rf_adjoint_tiles.cu), used by rf_adjoint,
// rf_step_host and the tile-queue path of rf_batch_solve.
#pragma once

#include "rf_ctx.h"

namespace rf {

struct TGrid;

// Alg. 2 on one ny x nx grid: radix sort by decreasing T, then the
// dependency-ordered gather; writes dLdproj5 (5 planes of stride ny * nx)
// and lambda (nullable).
rf_status adjoint_ordered(rf_ctx *ctx, int ny, int nx, const uint8_t *src, const float *T, const rf_record *rec,
                          const float *dLdT, float *dLdproj5, float *lambda, cudaStream_t s);

// Alg. 2 on one grid with the dependency chain followed inside 16 x 16
// tiles in shared memory (RF_ADJ_TILES); same outputs as adjoint_ordered,
// bit for bit.
rf_status adjoint_tiles(rf_ctx *ctx, int ny, int nx, const uint8_t *src, const float *T, const rf_record *rec,
                        const float *dLdT, float *dLdproj5, float *lambda, cudaStream_t s);

// The same on packed grids (device descriptors with increasing node
// offsets, n nodes in all, no side above max_line): tiles handed out grid
// by grid in the packed order.
rf_status adjoint_tiles_packed(rf_ctx *ctx, long long n, const TGrid *grids, int n_grids, int max_line,
                               const uint8_t *src, const float *T, const rf_record *rec, const float *dLdT,
                               float *dLdproj5, float *lambda, cudaStream_t s);

// Next epoch of the context's tagged per-node state words (n of them):
// enqueues the device-side bump on s and returns the device word the
// adjoint kernels read it from; clears the words on first use and near the
// 32-bit wrap.
rf_status adjoint_next_epoch(rf_ctx *ctx, long long n, cudaStream_t s, const unsigned **epoch);

}  // namespace rf
