// rf_sweep_tiles.cu -- a2-a4, the tile-queue variant of the forward solve.
//
// Same discrete system as the line sweeps (Sec. 3.2, Eqs. 2-3; Alg. 1): every
// non-source node takes the minimum over its valid one-point and two-point
// candidates (replacement update), and the solve stops at a state where no
// node would change by more than tol + rtol T.  Only the schedule differs.
// The paper's column/row fronts need one dependent step per grid line and
// per sweep (2048 x 15 at 2048^2); here the grid is cut into 32 x 32 tiles
// and the work is organised in rounds:
//
//  * a round processes the tiles in its queue; a processed tile loads its
//    nodes' cone-form constants (rf_cone.cuh) into registers -- one thread
//    per node -- and its current T plus a one-node halo ring into shared
//    memory, then iterates Jacobi updates with the halo held fixed until no
//    node changes (a local fixed point).  A warp owns an 8 x 4 patch and
//    only evaluates when a node next to one of its nodes changed in the
//    previous iteration (per-row change masks, one byte per warp and row);
//  * a tile whose boundary nodes changed queues its neighbours for the next
//    round, keyed by the smallest new boundary time; a round processes the
//    queued tiles whose key is within a window of the smallest key and
//    defers the others (delta-stepping on tiles: tiles far ahead of the
//    front would only be revisited once the front reaches them);
//  * tiles read their neighbours' state as of the start of the round: every
//    tile's latest version lives in one of two T buffers, tagged per tile
//    with (round written, parity); a tile writes its new version into the
//    other buffer, so results do not depend on the order in which the CTAs
//    take tiles, and the solve is deterministic;
//  * the solve ends when a round queues nothing: every tile then sits at a
//    local fixed point of an unchanged halo, i.e. the whole grid is a fixed
//    point of T = min valid candidate(T) to the change tolerance.
//
// The dependent chain is the number of Jacobi iterations along the path of
// the front (a few thousand at 2048^2) instead of sweeps x grid lines.
#include <algorithm>

#include "rf_cone.cuh"
#include "rf_ctx.h"
#include "rf_sweep_common.cuh"
#include "rf_sweep_tiles.h"

namespace rf {

constexpr int kTS = 32;              // tile side in nodes
constexpr int kTW = kTS + 2;         // tile side with the halo ring
constexpr int kHalo = 4 * kTS + 4;   // halo ring nodes
constexpr int kTP = kTW + 6;         // shared-memory row pitch: rows 8 banks apart, so the
                                     // 4 rows x 8 columns of a warp's patch hit 32 banks
constexpr int kTileThreads = kTS * kTS;
constexpr unsigned kInfBits = 0x7f800000u;
constexpr int kSlots = 3;            // list / counter slots (round mod 3)

// control words of one round slot
struct TileSlot {
  unsigned count;  // tiles queued for the round
  unsigned grab;   // next list entry to hand out
  unsigned kmin;   // float bits of the smallest queued key
  unsigned pad;
};

struct TileArgs {
  int ny, nx, tny, tnx, ntiles;
  float h, eps;
  const float *f;
  const uint8_t *src;
  float *T[2];  // buffer 0 = the caller's T, buffer 1 = workspace
  float tol, rtol;
  float window;  // delta-stepping window in tile crossings
  int warm;
  int max_rounds, max_local;
  TileWork w;
  LaunchCtl ctl;
};

// Halo index -> (row, column) in the (kTW x kTW) tile frame.
__device__ __forceinline__ void halo_rc(int k, int &r, int &c) {
  if (k < kTW) { r = 0; c = k; }
  else if (k < 2 * kTW) { r = kTW - 1; c = k - kTW; }
  else if (k < 2 * kTW + kTS) { r = 1 + (k - 2 * kTW); c = 0; }
  else { r = 1 + (k - 2 * kTW - kTS); c = kTW - 1; }
}

// Change masks: one 64-bit word per frame row; bits 0..31 are the interior
// columns 0..31 (byte k written by the warps of patch column k), bit 32 the
// left halo column, bit 33 the right one.  colspace() maps a word to frame
// column order (bit c = frame column c, 0..33).
__device__ __forceinline__ unsigned long long colspace(unsigned long long w) {
  return ((w & 0xffffffffull) << 1) | ((w >> 32) & 1ull) | (((w >> 33) & 1ull) << 33);
}
__device__ __forceinline__ unsigned long long frame_bit(int c) {
  return c == 0 ? (1ull << 32) : (c == kTW - 1) ? (1ull << 33) : (1ull << (c - 1));
}

// Buffer holding tile t's version as of the start of round r.
__device__ __forceinline__ int start_parity(unsigned st, int r) {
  const int par = (int)(st & 1u);
  return ((int)(st >> 1) == r) ? 1 - par : par;
}

__device__ __forceinline__ void enqueue(const TileWork &w, int ntiles, int t, int rr) {
  if (atomicMax(&w.queued[t], (unsigned)rr) < (unsigned)rr) {
    TileSlot *s = reinterpret_cast<TileSlot *>(w.ctrl) + (rr % kSlots);
    const unsigned idx = atomicAdd(&s->count, 1u);
    w.list[(size_t)(rr % kSlots) * ntiles + idx] = t;
  }
}

// Queue tile t for round rr with key bits kb.
__device__ __forceinline__ void push(const TileWork &w, int ntiles, int t, int rr, unsigned kb) {
  atomicMin(&w.key[(size_t)(rr & 1) * ntiles + t], kb);
  TileSlot *s = reinterpret_cast<TileSlot *>(w.ctrl) + (rr % kSlots);
  atomicMin(&s->kmin, kb);
  enqueue(w, ntiles, t, rr);
}

__global__ void __launch_bounds__(kTileThreads, 1) tile_solve_kernel(TileArgs a) {
  __shared__ float Ts[2][kTW][kTP];
  __shared__ unsigned long long rowm[2][kTW];  // change masks (see colspace)
  __shared__ unsigned nkey[9];                 // smallest changed boundary time per neighbour
  __shared__ int s_tile, s_go, s_par[9];
  __shared__ unsigned s_key;

  // warp w owns the 8 x 4 patch (w >> 2, w & 3) of the tile
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int pr = wp >> 2, pc = wp & 3, ao = lane >> 3;
  const int row = pr * 4 + ao, col = pc * 8 + (lane & 7);
  const TileWork &w = a.w;
  const int NT = a.ntiles;
  const long long plane = (long long)a.ny * a.nx;
  TileSlot *slots = reinterpret_cast<TileSlot *>(w.ctrl);
  unsigned long long my_updates = 0, my_warp_evals = 0;
  bool converged = false, abort = false;
  int r = 1;
  const float ebar = __uint_as_float(w.ctrl[kSlots * 4]);  // mean edge cost (seed kernel)
  const float delta = a.window * (float)kTS * ebar;

  for (;; ++r) {
    TileSlot *cur = slots + (r % kSlots);
    if (blockIdx.x == 0 && tid == 0) {
      // the slot last used two rounds ago is free: ready it for round r + 2
      TileSlot *old = slots + ((r + 2) % kSlots);
      old->count = 0;
      old->grab = 0;
      old->kmin = kInfBits;
    }
    const unsigned n = __ldcg(&cur->count);
    if (n == 0) {
      converged = true;
      break;
    }
    if (r > a.max_rounds) break;
    const float theta = __uint_as_float(__ldcg(&cur->kmin)) + delta;
    while (true) {
      if (tid == 0) {
        const unsigned k = atomicAdd(&cur->grab, 1u);
        s_go = k < n;
        if (k < n) {
          const int t = __ldcg(&w.list[(size_t)(r % kSlots) * NT + k]);
          s_tile = t;
          unsigned *kp = &w.key[(size_t)(r & 1) * NT + t];
          s_key = __ldcg(kp);
          __stcg(kp, kInfBits);
        }
      }
      __syncthreads();
      if (!s_go) break;
      const int t = s_tile;
      const unsigned kb = s_key;
      if (__uint_as_float(kb) > theta) {
        // too far ahead of the front: keep it for a later round
        if (tid == 0) push(w, NT, t, r + 1, kb);
        __syncthreads();
        continue;
      }
      const int ti = t / a.tnx, tj = t - ti * a.tnx;
      const int i0 = ti * kTS, j0 = tj * kTS;
      // buffer parities of this tile and its eight neighbours as of the
      // round's start (index (di + 1) * 3 + (dj + 1))
      if (tid < 9) {
        const int di = tid / 3 - 1, dj = tid % 3 - 1;
        const int ni = ti + di, nj = tj + dj;
        int p = 0;
        if (ni >= 0 && ni < a.tny && nj >= 0 && nj < a.tnx)
          p = start_parity(__ldcg(&w.tstate[ni * a.tnx + nj]), r);
        s_par[tid] = p;
        nkey[tid] = kInfBits;
      }
      if (tid < kTW) {
        rowm[0][tid] = 0ull;
        rowm[1][tid] = 0ull;
      }
      __syncthreads();
      const int pt = s_par[4];
      const float *Tin = a.T[pt];
      float *Tout = a.T[1 - pt];
      // this thread's node and its cone-form constants
      const int i = i0 + row, j = j0 + col;
      const bool inb = (i < a.ny) && (j < a.nx);
      const long long p = (long long)i * a.nx + j;
      float4 q[kPlanes];
      bool is_src = false;
      float tcur = kInf;
      if (inb) {
        is_src = a.src[p] != 0;
        node_record(__ldg(a.f + p), __ldg(a.f + plane + p), __ldg(a.f + 2 * plane + p), __ldg(a.f + 3 * plane + p),
                    __ldg(a.f + 4 * plane + p), a.h, a.eps, is_src, q);
        tcur = __ldcg(Tin + p);
      } else {
#pragma unroll
        for (int c = 0; c < kPlanes; ++c) q[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const bool upd = inb && !is_src;
      const float tinit = tcur;
      Ts[0][row + 1][col + 1] = tcur;
      Ts[1][row + 1][col + 1] = tcur;
      // halo ring, from the neighbours' round-start versions; nodes whose
      // value differs from this tile's previous visit seed the change masks
      if (tid < kHalo) {
        int hr, hc;
        halo_rc(tid, hr, hc);
        const int gi = i0 - 1 + hr, gj = j0 - 1 + hc;
        float v = kInf;
        if (gi >= 0 && gi < a.ny && gj >= 0 && gj < a.nx) {
          const int di = (hr == 0) ? -1 : (hr == kTW - 1) ? 1 : 0;
          const int dj = (hc == 0) ? -1 : (hc == kTW - 1) ? 1 : 0;
          v = __ldcg(a.T[s_par[(di + 1) * 3 + dj + 1]] + (long long)gi * a.nx + gj);
        }
        Ts[0][hr][hc] = v;
        Ts[1][hr][hc] = v;
        float *hp = w.halo + (size_t)t * kHalo + tid;
        const float prev = __ldcg(hp);
        if (node_changed(v, prev, a.tol, a.rtol)) atomicOr(&rowm[0][hr], frame_bit(hc));
        __stcg(hp, v);
      }
      // first visit: the sources (cold) or every node (warm) start changed
      const bool first = __ldcg(&w.visits[t]) == 0u;
      if (first) {
        const bool seed = inb && (a.warm ? true : is_src);
        const unsigned bal = __ballot_sync(0xffffffffu, seed);
        const unsigned long long byte = (bal >> (8 * ao)) & 0xffu;
        if ((lane & 7) == 0 && byte) atomicOr(&rowm[0][row + 1], byte << (8 * pc));
      }
      __syncthreads();

      // Jacobi iterations with the halo fixed
      int cb = 0, it = 0;
      bool capped = false;
      const int sr = row + 1, sc = col + 1;
      while (true) {
        const unsigned long long nb = ((colspace(rowm[cb][sr - 1]) | colspace(rowm[cb][sr + 1])) >> (sc - 1)) & 7ull |
                                      ((colspace(rowm[cb][sr]) >> (sc - 1)) & 5ull);
        const bool dirty = nb != 0ull;
        const unsigned dball = __ballot_sync(0xffffffffu, dirty && upd);
        float tnew = tcur;
        if (dball) {
          if (upd) {
            float Tn[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) Tn[k] = Ts[cb][sr + nb_dy(k)][sc + nb_dx(k)];
            tnew = cone_min(q[0], q[1], q[2], q[3], q[4], q[5], Tn);
          }
          if (lane == 0) {
            my_updates += (unsigned long long)__popc(dball);
            my_warp_evals += 1;
          }
        }
        Ts[cb ^ 1][sr][sc] = tnew;
        const bool ch = upd && node_changed(tnew, tcur, a.tol, a.rtol);
        const unsigned cbal = __ballot_sync(0xffffffffu, ch);
        // this warp's byte of each of its four rows (plain byte stores: the
        // four patch columns of a row write disjoint bytes)
        if ((lane & 7) == 0)
          reinterpret_cast<unsigned char *>(&rowm[cb ^ 1][sr])[pc] = (unsigned char)((cbal >> (8 * ao)) & 0xffu);
        // slot 0 still holds the initial halo bits, read only by iteration 0:
        // clear them before iteration 2 reads the slot again
        if (it == 1 && tid < kTW) {
          reinterpret_cast<unsigned *>(&rowm[0][tid])[1] = 0u;
          if (tid == 0 || tid == kTW - 1) reinterpret_cast<unsigned *>(&rowm[0][tid])[0] = 0u;
        }
        tcur = tnew;
        const int any = __syncthreads_or(ch);
        cb ^= 1;
        ++it;
        if (!any) break;
        if (it >= a.max_local) {
          capped = true;
          break;
        }
      }

      // publish: a new version only if some node moved beyond the tolerance
      const bool moved = upd && node_changed(tcur, tinit, a.tol, a.rtol);
      if (__syncthreads_or(moved)) {
        if (inb) __stcg(Tout + p, tcur);
        if (moved) {
          const unsigned kbits = __float_as_uint(tcur);
          const bool top = row == 0, bot = row == kTS - 1, lft = col == 0, rgt = col == kTS - 1;
          if (top) atomicMin(&nkey[1], kbits);
          if (bot) atomicMin(&nkey[7], kbits);
          if (lft) atomicMin(&nkey[3], kbits);
          if (rgt) atomicMin(&nkey[5], kbits);
          if (top && lft) atomicMin(&nkey[0], kbits);
          if (top && rgt) atomicMin(&nkey[2], kbits);
          if (bot && lft) atomicMin(&nkey[6], kbits);
          if (bot && rgt) atomicMin(&nkey[8], kbits);
        }
        __syncthreads();
        if (tid == 0) __stcg(&w.tstate[t], ((unsigned)r << 1) | (unsigned)(1 - pt));
        if (tid < 9 && tid != 4 && nkey[tid] != kInfBits) {
          const int ni = ti + tid / 3 - 1, nj = tj + tid % 3 - 1;
          if (ni >= 0 && ni < a.tny && nj >= 0 && nj < a.tnx) push(w, NT, ni * a.tnx + nj, r + 1, nkey[tid]);
        }
      }
      if (tid == 0) {
        __stcg(&w.visits[t], __ldcg(&w.visits[t]) + 1u);
        // a visit cut short by the iteration cap is resumed next round
        if (capped) push(w, NT, t, r + 1, kb);
      }
      __syncthreads();
    }
    if (!grid_sync(a.ctl)) {
      abort = true;
      break;
    }
  }
  if (lane == 0 && (my_updates || my_warp_evals)) {
    atomicAdd(&w.counters[0], my_updates);
    atomicAdd(&w.counters[1], my_warp_evals);
  }
  if (!abort) {
    // hand the latest version of every tile back in the caller's buffer
    for (int t = blockIdx.x; t < NT; t += gridDim.x) {
      if ((__ldcg(&w.tstate[t]) & 1u) == 0u) continue;
      const int ti = t / a.tnx, tj = t - ti * a.tnx;
      const int i = ti * kTS + row, j = tj * kTS + col;
      if (i < a.ny && j < a.nx) {
        const long long p = (long long)i * a.nx + j;
        a.T[0][p] = __ldcg(a.T[1] + p);
      }
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    a.ctl.st->rounds = (unsigned)(r - 1);
    a.ctl.st->converged = converged ? 1 : 0;
    if (!converged && !abort) set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
  }
}

// Workspace reset and the first round's queue: the tiles holding a source
// (cold) or every tile (warm), key 0; the mean edge cost of the field
// (mean of (|m_x|_M + |m_y|_M) / 2) for the delta-stepping window.
__global__ void tile_seed_kernel(TileArgs a, float *esum) {
  const TileWork &w = a.w;
  const int NT = a.ntiles;
  const long long plane = (long long)a.ny * a.nx;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g0 == 0) {
    TileSlot *slots = reinterpret_cast<TileSlot *>(w.ctrl);
    for (int k = 0; k < kSlots; ++k) {
      slots[k].count = 0u;
      slots[k].grab = 0u;
      slots[k].kmin = kInfBits;
    }
  }
  for (long long t = g0; t < NT; t += stride) {
    w.tstate[t] = 0u;
    w.visits[t] = 0u;
    w.key[t] = kInfBits;
    w.key[NT + t] = kInfBits;
    w.queued[t] = 0u;
    if (a.warm) w.queued[t] = 1u;
  }
  for (long long k = g0; k < (long long)NT * kHalo; k += stride) w.halo[k] = kInf;
  float part = 0.0f;
  for (long long p = g0; p < plane; p += stride) {
    const float l11 = a.f[p], l21 = a.f[plane + p], l22 = a.f[2 * plane + p];
    const float m11 = fmaf(l11, l11, a.eps), m22 = fmaf(l21, l21, fmaf(l22, l22, a.eps));
    part += 0.5f * a.h * (sqrtf(m11) + sqrtf(m22));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(esum, part);
}

// Queue the first round (runs after tile_seed_kernel), key 0: every tile
// (warm) or the tiles around the sources (cold).
__global__ void tile_queue_kernel(TileArgs a) {
  const TileWork &w = a.w;
  const int NT = a.ntiles;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a.warm) {
    for (long long t = g0; t < NT; t += stride) {
      w.key[NT + t] = 0u;  // round 1 reads key slot 1
      w.list[(size_t)(1 % kSlots) * NT + t] = (int)t;
    }
    return;
  }
  // every tile that holds a source or one of its neighbours: a source never
  // changes, so the tiles across a tile edge next to it must see it in
  // their halo on their own first visit
  const long long plane = (long long)a.ny * a.nx;
  for (long long p = g0; p < plane; p += stride) {
    if (!a.src[p]) continue;
    const int i = (int)(p / a.nx), j = (int)(p - (long long)i * a.nx);
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj) {
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || ii >= a.ny || jj < 0 || jj >= a.nx) continue;
        const int t = (ii / kTS) * a.tnx + jj / kTS;
        atomicMin(&w.key[NT + t], 0u);
        enqueue(w, NT, t, 1);
      }
  }
}

__global__ void tile_finish_seed_kernel(TileArgs a, const float *esum) {
  if (threadIdx.x != 0) return;
  TileSlot *slots = reinterpret_cast<TileSlot *>(a.w.ctrl);
  if (a.warm) slots[1 % kSlots].count = (unsigned)a.ntiles;
  slots[1 % kSlots].kmin = 0u;
  const float ebar = *esum / (float)((long long)a.ny * a.nx);
  a.w.ctrl[kSlots * 4] = __float_as_uint(ebar > 0.0f && ebar < kInf ? ebar : 1.0f);
}

// Statistics of the solve: node updates and their sweep equivalent.
__global__ void tile_stats_kernel(const unsigned long long *counters, DevState *st, long long n) {
  if (threadIdx.x != 0) return;
  const unsigned long long u = counters[0];
  st->cell_updates = u;
  st->sweeps = (int)((u + (unsigned long long)n - 1ull) / (unsigned long long)n);
}

}  // namespace rf

namespace rf {

int tiles_count(int ny, int nx) { return ((ny + kTS - 1) / kTS) * ((nx + kTS - 1) / kTS); }

size_t tile_work_bytes(int ny, int nx) {
  const size_t NT = (size_t)tiles_count(ny, nx);
  // tstate, visits, queued, key[2], list[3], halo, ctrl, counters
  return NT * 4 * 5 + NT * 4 * kSlots + NT * kHalo * 4 + 256 + 64;
}

TileWork tile_work_carve(void *base, int ny, int nx) {
  const size_t NT = (size_t)tiles_count(ny, nx);
  unsigned char *b = (unsigned char *)base;
  TileWork w;
  w.counters = (unsigned long long *)b;  // 8-byte aligned first
  b += 64;
  w.ctrl = (unsigned *)b;
  b += 256;
  w.tstate = (unsigned *)b;
  b += NT * 4;
  w.visits = (unsigned *)b;
  b += NT * 4;
  w.queued = (unsigned *)b;
  b += NT * 4;
  w.key = (unsigned *)b;
  b += NT * 8;
  w.list = (int *)b;
  b += NT * 4 * kSlots;
  w.halo = (float *)b;
  return w;
}

rf_status tiles_launch(int device, int num_sms, int ny, int nx, float h, float eps, const float *proj5,
                       const uint8_t *src, float *T, float *Tb, int warm, int max_sweeps, float tol, float rtol,
                       float window, const TileWork &w, const LaunchCtl &ctl, cudaStream_t s) {
  TileArgs a;
  a.ny = ny;
  a.nx = nx;
  a.tny = (ny + kTS - 1) / kTS;
  a.tnx = (nx + kTS - 1) / kTS;
  a.ntiles = a.tny * a.tnx;
  a.h = h;
  a.eps = eps;
  a.f = proj5;
  a.src = src;
  a.T[0] = T;
  a.T[1] = Tb;
  a.tol = tol;
  a.rtol = rtol;
  a.window = window > 0.0f ? window : 2.0f;
  a.warm = warm;
  // a sweep moves information across the grid, a round across one tile
  a.max_rounds = max_sweeps * std::max(a.tny, a.tnx);
  a.max_local = 16 * kTS;
  a.w = w;
  a.ctl = ctl;
  if (cudaMemsetAsync(w.counters, 0, 64 + 256, s) != cudaSuccess) return RF_ERR_CUDA;
  float *esum = (float *)(w.ctrl + kSlots * 4 + 1);
  const long long n = (long long)ny * nx;
  const int blocks = blocks_for(std::max(n, (long long)a.ntiles * kHalo), 256, num_sms * 8);
  tile_seed_kernel<<<blocks, 256, 0, s>>>(a, esum);
  tile_queue_kernel<<<blocks, 256, 0, s>>>(a);
  tile_finish_seed_kernel<<<1, 32, 0, s>>>(a, esum);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_solve_kernel, kTileThreads, 0) != cudaSuccess)
    return RF_ERR_CUDA;
  if (per_sm < 1) return RF_ERR_UNSUPPORTED;
  const int grid = per_sm * num_sms;
  void *args[] = {&a};
  (void)device;
  if (cudaLaunchCooperativeKernel((const void *)tile_solve_kernel, dim3(grid), dim3(kTileThreads), args, 0, s) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  tile_stats_kernel<<<1, 32, 0, s>>>(w.counters, ctl.st, n);
  return cuda_status(cudaGetLastError());
}

}  // namespace rf
