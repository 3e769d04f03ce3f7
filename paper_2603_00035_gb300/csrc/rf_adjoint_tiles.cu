// rf_adjoint_tiles.cu -- a6-a8 by tiles (RF_ADJ_TILES): the adjoint of the
// converged system (Sec. 3.3, Eqs. 4-6; App. A, Alg. 2) with its dependency
// chain followed in shared memory.
//
// The multipliers obey lambda_p = g_p + sum over children q of p of
// (dT_q / dT_p) lambda_q, children having a strictly larger T.  The ordered
// gather (rf_adjoint.cu) hands every link of this DAG through L2 -- a child
// publishes, its parent polls -- and the DAG of a large grid is well over a
// thousand links deep.  Here one CTA owns a 16 x 16 tile at a time: its 256
// compute threads (one node each) follow the links inside the tile through
// shared memory, each node finishing as soon as its children have, while
// one more warp copies in the multipliers of the halo nodes the tile needs,
// as the tiles around it publish them.  Only links across a tile edge go
// through L2.
//
// Tiles are handed out in decreasing order of their latest arrival time (a
// radix sort of per-tile keys), so a tile is taken about when the reverse
// front reaches it.  The order is a heuristic, not a schedule: a tile may
// need a node of a tile taken after it (where the characteristics run along
// a tile edge, or near a source).  A tile whose compute warps see no
// progress for park_ns therefore gives up: what it finished stays
// published, it goes into a retry ring, and the CTA takes the next tile.
// Ring tiles are taken once the main list is empty; on re-entry the tile
// reloads the multipliers it had finished.  The unfinished node of largest
// T can always finish once its tile is held, so the solve always
// progresses.
//
// Every multiplier is computed once from its children's final values, in
// the ordered gather's fixed neighbour order with the same fused
// multiply-adds, and published with the same epoch-tagged 64-bit word: the
// multipliers and dL/dtheta = lambda dT0/dtheta (Alg. 2, last loop; zero at
// sources and unreached nodes) equal RF_ADJ_ORDERED's bit for bit.
#include <algorithm>

#include <cub/device/device_radix_sort.cuh>

#include "rf_adjoint.h"
#include "rf_ctx.h"
#include "rf_sweep_common.cuh"
#include "rf_sweep_tiles.h"

namespace rf {
namespace {

constexpr int kTS = 16;                    // tile side
constexpr int kHS = kTS + 2;               // with the halo ring
constexpr int kNodes = kTS * kTS;          // compute threads
constexpr int kHalo = 4 * kTS + 4;         // halo nodes
constexpr int kCompWarps = kNodes / 32;
constexpr int kThreads = kNodes + 32;      // + the halo warp
constexpr unsigned long long kTagMask = 0xffffffff00000000ull;
// A warp that has seen no progress for kSpinFree polls sleeps kSleepNs
// between polls, leaving issue slots to the warps of other tiles that have
// work; with that, three tiles per SM are in flight.  2048^2 workload:
// 1.00 ms at two per SM without sleeping, 0.96 at three with 16 / 100 ns
// (0.97 with 64 / 300, 1.04 with 16 / 200 at four).
constexpr unsigned kSpinFree = 16;
constexpr unsigned kSleepNs = 100;
constexpr int kCtasPerSm = 3;
constexpr int kGridGroup = 8;  // packed grids ordered together (see tile_keys_kernel)

struct TileAdjArgs {
  int ny, nx, tiles_x, n_tiles;  // one grid (n_grids == 1)
  int n_grids;                   // > 1: packed grids
  const TGrid *grids;            // their shapes and node offsets
  const int *toff;               // first 16 x 16 tile of each grid
  const int *tgrid;              // grid of each tile (-1: past the last tile)
  const unsigned *ntiles_dev;    // packed grids: the number of tiles (device)
  long long n;
  const uint8_t *src;
  const float *T;
  const uint8_t *id;
  const float *w1;
  const float *dT;  // 5 planes of stride n
  const float *g;
  const unsigned *order;      // tile indices by decreasing latest T
  unsigned long long *state;  // (epoch << 32) | lambda bits, per node
  const unsigned *epoch;      // this launch's tag (device word, bumped before the launch)
  unsigned *words;  // [0] main-list ticket, [1] finished tiles, [2] ring head, [3] ring tail, [4] parks
  unsigned *ring;   // retry ring: tile + 1, 0 = empty
  unsigned ring_cap;
  float *grad;     // 5 planes out
  float *lam_out;  // nullable
  long long park_ns;
  LaunchCtl ctl;
};

// Halo slot h (0..kHalo-1) <-> position in the kHS x kHS array: the top
// row, the bottom row, then the left and right columns without corners.
__device__ __forceinline__ int halo_pos(int h) {
  if (h < kHS) return h;
  if (h < 2 * kHS) return (kHS - 1) * kHS + (h - kHS);
  if (h < 2 * kHS + kTS) return (h - 2 * kHS + 1) * kHS;
  return (h - 2 * kHS - kTS + 1) * kHS + kHS - 1;
}
__device__ __forceinline__ int halo_slot(int r, int c) {
  if (r == 0) return c;
  if (r == kHS - 1) return kHS + c;
  if (c == 0) return 2 * kHS + r - 1;
  return 2 * kHS + kTS + r - 1;
}

// Shared-memory words are read and written whole (64-bit, single-copy
// atomic), as in global memory: the tag says whether the value is final.
__device__ __forceinline__ unsigned long long lds_u64(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void sts_u64(unsigned long long *p, unsigned long long v) {
  *(volatile unsigned long long *)p = v;
}

// Where a tile lies: its grid's node offset and shape, and its first row
// and column.  False for a tile past the last one (packed grids: the tile
// arrays are sized by an upper bound).
struct TileGeo {
  long long goff;
  int gny, gnx, ti0, tj0;
  int gid;  // grid of the tile (0: one grid)
};
__device__ __forceinline__ bool tile_geo(const TileAdjArgs &a, int tile, TileGeo &g) {
  int tl = tile, tx = a.tiles_x;
  if (!a.grids) {
    g.goff = 0;
    g.gny = a.ny;
    g.gnx = a.nx;
    g.gid = 0;
  } else {
    const int gid = a.tgrid[tile];
    if (gid < 0) return false;
    const TGrid &d = a.grids[gid];
    g.goff = d.node_off;
    g.gny = d.ny;
    g.gnx = d.nx;
    g.gid = gid;
    tl = tile - a.toff[gid];
    tx = (d.nx + kTS - 1) / kTS;
  }
  g.ti0 = (tl / tx) * kTS;
  g.tj0 = (tl - (tl / tx) * tx) * kTS;
  return true;
}

// Packed grids: the first 16 x 16 tile of every grid (an exclusive scan of
// the grids' tile counts, one block) and the total.
__global__ void __launch_bounds__(1024) adjt_plan_kernel(const TGrid *grids, int n_grids, int *toff,
                                                        unsigned *ntiles) {
  __shared__ int part[1024];
  int carry = 0;
  for (int base = 0; base < n_grids; base += 1024) {
    const int g = base + (int)threadIdx.x;
    const int c = g < n_grids ? ((grids[g].ny + kTS - 1) / kTS) * ((grids[g].nx + kTS - 1) / kTS) : 0;
    part[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int v = (int)threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    if (g < n_grids) toff[g] = carry + part[threadIdx.x] - c;
    carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *ntiles = (unsigned)carry;
}

// Packed grids: the grid of each tile (the array is preset to -1).
__global__ void adjt_map_kernel(const TGrid *grids, int n_grids, const int *toff, int *tgrid) {
  for (int g = blockIdx.x; g < n_grids; g += gridDim.x) {
    const int c = ((grids[g].ny + kTS - 1) / kTS) * ((grids[g].nx + kTS - 1) / kTS);
    for (int k = threadIdx.x; k < c; k += blockDim.x) tgrid[toff[g] + k] = g;
  }
}

// Sort key of a tile: ascending key = group of kGridGroup grids (packed
// grids, in their packed order), then decreasing latest finite T; tiles
// without a reached node last in their group, tiles past the last one at
// the very end.  A group's tiles are handed out together, so a tile only
// waits for tiles of a few grids, taken about when they are needed -- as
// with one grid -- while the groups' grids still overlap their dependency
// chains.  Batched workload (256 grids, sides 64..1024): 70.2 ms per batch
// with one grid per group, 65.5 / 61.6 / 59.6 / 59.8 / 64.5 with 2 / 4 / 8 /
// 16 / 32; with 64 grids, or all 256, ordered together by time the CTAs end
// up holding tiles of many grids that each wait for a neighbour no CTA has
// taken (0.4-1.8 s of yields).
__global__ void tile_keys_kernel(TileAdjArgs a, int n_tiles, unsigned long long *keys, unsigned *vals) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < n_tiles; tile += warps) {
    TileGeo g;
    float m = -1.0f;
    const bool real = tile_geo(a, tile, g);
    if (real) {
      for (int k = lane; k < kNodes; k += 32) {
        const int i = g.ti0 + (k >> 4), j = g.tj0 + (k & (kTS - 1));
        if (i < g.gny && j < g.gnx) {
          const float t = a.T[g.goff + (long long)i * g.gnx + j];
          if (t < kInf) m = fmaxf(m, t);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      const unsigned kt = m >= 0.0f ? ~__float_as_uint(m) : 0xffffffffu;
      keys[tile] = real ? ((unsigned long long)(g.gid / kGridGroup) << 32) | kt : ~0ull;
      vals[tile] = (unsigned)tile;
    }
  }
}

// Next tile of the CTA (thread 0): the main list, then the retry ring
// until every tile is finished; -1 when there is nothing left (or the
// launch was aborted).
__device__ int take_tile(const TileAdjArgs &a, unsigned n_tiles, unsigned long long t_start) {
  if (ld_acquire_s32(a.ctl.abort)) return -1;
  const unsigned k = atomicAdd(&a.words[0], 1u);
  if (k < n_tiles) return (int)a.order[k];
  unsigned spins = 0;
  while (true) {
    if (ld_acquire_u32(&a.words[1]) >= n_tiles) return -1;
    const unsigned h = ld_acquire_u32(&a.words[2]), tl = ld_acquire_u32(&a.words[3]);
    if (h < tl) {
      if (atomicCAS(&a.words[2], h, h + 1) == h) {
        // the pusher advanced the tail before writing the entry
        unsigned *slot = &a.ring[h % a.ring_cap];
        unsigned v = 0;
        while ((v = atomicExch(slot, 0u)) == 0u) {
          if ((long long)(gtimer() - t_start) > a.ctl.timeout_ns || ld_acquire_s32(a.ctl.abort)) {
            raise_timeout(a.ctl);
            return -1;
          }
        }
        return (int)v - 1;
      }
      continue;
    }
    if ((++spins & 15) == 0 &&
        ((long long)(gtimer() - t_start) > a.ctl.timeout_ns || ld_acquire_s32(a.ctl.abort))) {
      raise_timeout(a.ctl);
      return -1;
    }
    __nanosleep(256);
  }
}

// A tile that gave up goes to the back of the retry ring (thread 0, after
// the CTA barrier that follows its last published multiplier).
__device__ void park_tile(const TileAdjArgs &a, int tile) {
  const unsigned pos = atomicAdd(&a.words[3], 1u);
  atomicAdd(&a.words[4], 1u);
  __threadfence();
  atomicExch(&a.ring[pos % a.ring_cap], (unsigned)tile + 1u);
}

}  // namespace

__global__ void __launch_bounds__(kThreads) tile_adjoint_kernel(TileAdjArgs a) {
  __shared__ unsigned long long sw[kHS * kHS];  // tile + halo: tag | lambda
  __shared__ unsigned need[(kHalo + 31) / 32];  // halo nodes some tile node waits for
  __shared__ int s_tile, s_left, s_park;        // current tile, compute warps done, give up
  __shared__ TileGeo s_geo;                     // where it lies
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool compute = warp < kCompWarps;
  const long long n = a.n;
  const unsigned long long tag = (unsigned long long)__ldg(a.epoch) << 32;
  const unsigned long long t_start = gtimer();
  const unsigned n_tiles = a.ntiles_dev ? *(const volatile unsigned *)a.ntiles_dev : (unsigned)a.n_tiles;
  const int li = (t >> 4) & (kTS - 1), lj = t & (kTS - 1);
  const int slot = (li + 1) * kHS + lj + 1;
  while (true) {
    if (t == 0) {
      s_tile = take_tile(a, n_tiles, t_start);
      if (s_tile >= 0 && !tile_geo(a, s_tile, s_geo)) s_geo.gny = s_geo.gnx = 0;  // cannot happen: tile < n_tiles
    }
    for (int k = t; k < kHS * kHS; k += kThreads) sw[k] = 0ull;
    if (t < (kHalo + 31) / 32) need[t] = 0u;
    if (t == 0) {
      s_left = 0;
      s_park = 0;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile < 0) {
      if (t == 0) atomicMax(&a.ctl.st->adj_sweeps, (int)ld_acquire_u32(&a.words[4]));  // tiles that yielded
      break;
    }
    const int ti0 = s_geo.ti0, tj0 = s_geo.tj0, gny = s_geo.gny, gnx = s_geo.gnx;
    const long long goff = s_geo.goff;

    // ---- compute threads: own node, its children and their weights ----
    long long p = -1;
    bool done = true, act = false;
    unsigned cmask = 0;
    float cw[8], dTp[5], gsum = 0.0f;
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) cw[nb] = 0.0f;
#pragma unroll
    for (int c = 0; c < 5; ++c) dTp[c] = 0.0f;
    const int gi = ti0 + li, gj = tj0 + lj;
    if (compute && gi < gny && gj < gnx) {
      p = goff + (long long)gi * gnx + gj;
      // every load of the node and its neighbours first (one round trip),
      // the decisions after
      const unsigned long long w0 = ld_relaxed_u64(&a.state[p]);
      const float tp = a.T[p], gp = a.g[p];
      const bool actp = a.id[p] != 0 && !a.src[p];
      float d5[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) d5[c] = a.dT[c * n + p];
#pragma unroll
      for (int nb = 0; nb < 8; ++nb) {
        const int ii = gi + nb_dy(nb), jj = gj + nb_dx(nb);
        if (ii >= 0 && ii < gny && jj >= 0 && jj < gnx) {
          const long long q = goff + (long long)ii * gnx + jj;
          cw[nb] = child_weight(a.id[q], a.w1[q], (nb + 4) & 7);
        }
      }
      if ((w0 & kTagMask) == tag) {
        sw[slot] = w0;  // finished before the tile was parked
      } else if (!(tp < kInf)) {
        // unreached: no residual, no children; zero gradient and lambda
        st_relaxed_u64(&a.state[p], tag);
        sw[slot] = tag;
#pragma unroll
        for (int c = 0; c < 5; ++c) a.grad[c * n + p] = 0.0f;
        if (a.lam_out) a.lam_out[p] = 0.0f;
      } else {
        done = false;
        gsum = gp;
        act = actp;
#pragma unroll
        for (int c = 0; c < 5; ++c) dTp[c] = act ? d5[c] : 0.0f;
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) {
          if (cw[nb] != 0.0f) {
            cmask |= 1u << nb;
            const int r = li + 1 + nb_dy(nb), c = lj + 1 + nb_dx(nb);
            if (r == 0 || r == kHS - 1 || c == 0 || c == kHS - 1) {
              const int h = halo_slot(r, c);
              atomicOr(&need[h >> 5], 1u << (h & 31));
            }
          }
        }
      }
    }
    __syncthreads();

    if (compute) {
      // each node finishes once every child has: children inside the tile
      // through shared memory, halo children once the halo warp copied them
      unsigned prev = __ballot_sync(0xffffffffu, !done);
      unsigned long long tlast = gtimer();
      unsigned spins = 0;
      while (prev) {
        if (!done) {
          bool ready = true;
          float acc = gsum;
#pragma unroll
          for (int nb = 0; nb < 8; ++nb) {
            if (cmask & (1u << nb)) {
              const unsigned long long v = lds_u64(&sw[slot + nb_dy(nb) * kHS + nb_dx(nb)]);
              ready = ready && ((v & kTagMask) == tag);
              acc = fmaf(cw[nb], __uint_as_float((unsigned)v), acc);
            }
          }
          if (ready) {
            const unsigned long long w = tag | __float_as_uint(acc);
            sts_u64(&sw[slot], w);
            st_relaxed_u64(&a.state[p], w);
#pragma unroll
            for (int c = 0; c < 5; ++c) a.grad[c * n + p] = act ? acc * dTp[c] : 0.0f;
            if (a.lam_out) a.lam_out[p] = acc;
            done = true;
          }
        }
        const unsigned pend = __ballot_sync(0xffffffffu, !done);
        if (pend != prev) {
          prev = pend;
          spins = 0;
          tlast = gtimer();
        } else if (++spins > kSpinFree) {
          // a warp that has waited a while polls less often: tiles taken
          // ahead of the reverse front leave the issue slots to the others
          __nanosleep(kSleepNs);
        }
        if (spins && (spins & 63) == 0) {
          const unsigned long long now = gtimer();
          int stop = *(volatile int *)&s_park;
          if ((long long)(now - t_start) > a.ctl.timeout_ns || ld_acquire_s32(a.ctl.abort)) {
            if (lane == 0) raise_timeout(a.ctl);
            stop = 1;
          } else if ((long long)(now - tlast) > a.park_ns) {
            stop = 1;
          }
          stop = __shfl_sync(0xffffffffu, stop, 0);
          if (stop) {
            if (lane == 0) *(volatile int *)&s_park = 1;
            break;
          }
        }
      }
      if (lane == 0) atomicAdd(&s_left, 1);
    } else {
      // ---- halo warp: copy each needed halo multiplier once it is final ----
      unsigned pend = 0;
      long long q[3] = {0, 0, 0};
      int pos[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int h = lane + 32 * k;
        if (h < kHalo && ((need[h >> 5] >> (h & 31)) & 1u)) {
          pos[k] = halo_pos(h);
          const int r = pos[k] / kHS, c = pos[k] - r * kHS;
          q[k] = goff + (long long)(ti0 + r - 1) * gnx + (tj0 + c - 1);  // inside the grid: a child was found there
          pend |= 1u << k;
        }
      }
      unsigned polls = 0;
      while (true) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (pend & (1u << k)) {
            const unsigned long long v = ld_relaxed_u64(&a.state[q[k]]);
            if ((v & kTagMask) == tag) {
              sts_u64(&sw[pos[k]], v);
              pend &= ~(1u << k);
            }
          }
        }
        const bool fin = *(volatile int *)&s_left == kCompWarps;
        if (__all_sync(0xffffffffu, fin || pend == 0u)) break;
        if (++polls > kSpinFree / 8) __nanosleep(kSleepNs);
      }
    }
    __syncthreads();
    if (t == 0) {
      if (s_park) {
        park_tile(a, tile);
      } else {
        __threadfence();
        atomicAdd(&a.words[1], 1u);
      }
    }
  }
}

}  // namespace rf

namespace rf {

namespace {

// One grid (grids == NULL: ny x nx, n = ny * nx nodes, cap = its tiles) or
// packed grids (device descriptors, n nodes in all, cap >= their tiles).
rf_status adjoint_tiles_impl(rf_ctx *ctx, int ny, int nx, long long n, const TGrid *grids, int n_grids, int cap,
                             const uint8_t *src, const float *T, const rf_record *rec, const float *dLdT,
                             float *dLdproj5, float *lambda, cudaStream_t s) {
  ctx->last_stream = s;
  // scratch: keys in/out, values in/out, retry ring, control words, packed
  // grids' tile offsets and tile -> grid map, CUB temp
  // keys: the grid in the high word (packed grids), the time in the low one
  int end_bit = 32;
  while (grids && end_bit < 64 && (1ll << (end_bit - 32)) < n_grids) ++end_bit;
  size_t temp_bytes = 0;
  if (cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, (unsigned long long *)nullptr,
                                      (unsigned long long *)nullptr, (unsigned *)nullptr, (unsigned *)nullptr, cap, 0,
                                      end_bit, s) != cudaSuccess)
    return RF_ERR_CUDA;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t arr = up((size_t)cap * sizeof(unsigned));
  const size_t arr64 = up((size_t)cap * sizeof(unsigned long long));
  const unsigned ring_cap = 2u * (unsigned)cap;
  const size_t ring_bytes = up((size_t)ring_cap * sizeof(unsigned));
  const size_t toff_bytes = grids ? up((size_t)n_grids * sizeof(int)) : 0;
  const size_t map_bytes = grids ? arr : 0;
  const size_t need = 2 * arr64 + 2 * arr + ring_bytes + 256 + toff_bytes + map_bytes + up(temp_bytes);
  rf_status rs;
  if ((rs = ensure((unsigned char **)&ctx->scratch, &ctx->scratch_cap, need)) != RF_OK) return rs;
  unsigned char *base = (unsigned char *)ctx->scratch;
  unsigned long long *kin = (unsigned long long *)base, *kout = (unsigned long long *)(base + arr64);
  unsigned char *b2 = base + 2 * arr64;
  unsigned *vin = (unsigned *)b2, *vout = (unsigned *)(b2 + arr);
  unsigned *ring = (unsigned *)(b2 + 2 * arr);
  unsigned *words = (unsigned *)(b2 + 2 * arr + ring_bytes);  // [0..4] queue, [5] abort, [6] tiles
  int *toff = (int *)(b2 + 2 * arr + ring_bytes + 256);
  int *tgrid = (int *)(b2 + 2 * arr + ring_bytes + 256 + toff_bytes);
  void *temp = b2 + 2 * arr + ring_bytes + 256 + toff_bytes + map_bytes;
  const unsigned *epoch;
  if ((rs = adjoint_next_epoch(ctx, n, s, &epoch)) != RF_OK) return rs;
  if (cudaMemsetAsync(ring, 0, ring_bytes + 256, s) != cudaSuccess ||
      cudaMemsetAsync(&ctx->state->adj_sweeps, 0, sizeof(int), s) != cudaSuccess)
    return RF_ERR_CUDA;

  TileAdjArgs a;
  a.ny = ny;
  a.nx = nx;
  a.tiles_x = (nx + kTS - 1) / kTS;
  a.n_tiles = cap;
  a.n_grids = grids ? n_grids : 1;
  a.grids = grids;
  a.toff = toff;
  a.tgrid = tgrid;
  a.ntiles_dev = grids ? words + 6 : nullptr;
  a.n = n;
  a.src = src;
  a.T = T;
  a.id = rec->id;
  a.w1 = rec->w1;
  a.dT = rec->dT;
  a.g = dLdT;
  a.order = vout;
  a.state = ctx->adj_state;
  a.epoch = epoch;
  a.words = words;
  a.ring = ring;
  a.ring_cap = ring_cap;
  a.grad = dLdproj5;
  a.lam_out = lambda;
  a.park_ns = ctx->adj_park_ns;
  a.ctl.st = ctx->state;
  a.ctl.abort = (int *)(words + 5);
  a.ctl.timeout_ns = ctx->timeout_ns;
  if (grids) {
    if (cudaMemsetAsync(tgrid, 0xff, (size_t)cap * sizeof(int), s) != cudaSuccess) return RF_ERR_CUDA;
    adjt_plan_kernel<<<1, 1024, 0, s>>>(grids, n_grids, toff, words + 6);
    adjt_map_kernel<<<std::max(1, std::min(n_grids, 4 * ctx->num_sms)), 256, 0, s>>>(grids, n_grids, toff, tgrid);
  }
  tile_keys_kernel<<<blocks_for((long long)cap * 32, 256, ctx->num_sms * 8), 256, 0, s>>>(a, cap, kin, vin);
  if (cub::DeviceRadixSort::SortPairs(temp, temp_bytes, kin, kout, vin, vout, cap, 0, end_bit, s) != cudaSuccess)
    return RF_ERR_CUDA;

  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_adjoint_kernel, kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return RF_ERR_CUDA;
  // resident CTAs only (a cooperative launch checks it): a CTA that waits
  // for a tile held by a CTA that never started would only end by parking.
  // Two per SM: the waiting warps of more tiles cost the working ones issue
  // slots (2048^2 workload: 1.07 ms at two per SM, 1.70 at one, 2.53 at
  // four)
  const long long want = ((long long)cap + 1) / 2;
  const int grid = (int)std::min<long long>((long long)std::min(per_sm, kCtasPerSm) * ctx->num_sms,
                                            std::max<long long>(want, 1));
  void *args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void *)tile_adjoint_kernel, dim3(grid), dim3(kThreads), args, 0, s) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  return cuda_status(cudaGetLastError());
}

}  // namespace

rf_status adjoint_tiles(rf_ctx *ctx, int ny, int nx, const uint8_t *src, const float *T, const rf_record *rec,
                        const float *dLdT, float *dLdproj5, float *lambda, cudaStream_t s) {
  const int n_tiles = ((ny + kTS - 1) / kTS) * ((nx + kTS - 1) / kTS);
  return adjoint_tiles_impl(ctx, ny, nx, (long long)ny * nx, nullptr, 1, n_tiles, src, T, rec, dLdT, dLdproj5,
                            lambda, s);
}

rf_status adjoint_tiles_packed(rf_ctx *ctx, long long n, const TGrid *grids, int n_grids, int max_line,
                               const uint8_t *src, const float *T, const rf_record *rec, const float *dLdT,
                               float *dLdproj5, float *lambda, cudaStream_t s) {
  const int cap = tiles_cap(n_grids, n, max_line, kTS);
  return adjoint_tiles_impl(ctx, 0, 0, n, grids, n_grids, cap, src, T, rec, dLdT, dLdproj5, lambda, s);
}

}  // namespace rf
