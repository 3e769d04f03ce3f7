// rf_sweep_tiles.cu -- a2-a4, the tile-queue variant of the forward solve.
//
// Same discrete system as the line sweeps (Sec. 3.2, Eqs. 2-3; Alg. 1): every
// non-source node takes the minimum over its valid one-point and two-point
// candidates (replacement update), and the solve stops at a state where no
// node would change by more than tol + rtol T.  Only the schedule differs.
// The paper's column/row fronts need one dependent step per grid line and
// per sweep (2048 x 15 at 2048^2); here the grid is cut into square tiles
// (16 x 16 by default, or 32 x 32) and the work is organised in rounds:
//
//  * a round processes the tiles in its queue.  A CTA of 1024 threads runs
//    1024 / tile-nodes independent tile groups (one thread per node, a named
//    barrier per group), so four 16 x 16 tiles iterate side by side on an
//    SM.  A processed tile computes its nodes' cone-form constants
//    (rf_cone.cuh) into shared memory and loads its current T plus a
//    one-node halo ring, then iterates Jacobi updates with the halo held
//    fixed until no node changes (a local fixed point).  A warp owns an
//    8 x 4 patch and only evaluates when a node next to one of its nodes
//    changed in the previous iteration (per-row change masks, one byte per
//    warp and row);
//  * a tile whose boundary nodes changed queues its neighbours for the next
//    round, keyed by the smallest new boundary time; a round processes the
//    queued tiles whose key is within a window of the smallest key and
//    defers the others (delta-stepping on tiles: tiles far ahead of the
//    front would only be revisited once the front reaches them);
//  * tiles read their neighbours' state as of the start of the round: every
//    tile's latest version lives in one of two T buffers, tagged per tile
//    with (round written, parity); a tile writes its new version into the
//    other buffer, so results do not depend on the order in which tiles are
//    taken, and the solve is deterministic;
//  * when a round queues nothing, the next round certifies: it visits every
//    tile with every node marked changed, so each node is evaluated once with
//    the current values (a change below the tolerance never marks its
//    neighbours, so such changes could otherwise add up); the solve ends
//    after a certification round in which no tile moved -- every node is
//    then within tol + rtol T of min valid candidate(T), the guarantee of
//    the line sweeps' final no-change sweep.
//
// The dependent chain is the number of Jacobi iterations along the path of
// the front (a few thousand at 2048^2) instead of sweeps x grid lines.
#include <algorithm>

#include "rf_cone.cuh"
#include "rf_ctx.h"
#include "rf_sweep_common.cuh"
#include "rf_sweep_tiles.h"

namespace rf {

constexpr int kTileCta = 1024;     // threads per CTA (one or four tile groups)
constexpr unsigned kInfBits = 0x7f800000u;
constexpr int kSlots = 3;          // list / counter slots (round mod 3)

// control words of one round slot
struct TileSlot {
  unsigned count;  // tiles queued for the round
  unsigned grab;   // next list entry to hand out
  unsigned kmin;   // float bits of the smallest queued key
  unsigned pad;
};
// ctrl layout (unsigned words): 3 slots x 4, mean edge cost, its sum, tiles
// that published a new version [3] (by round mod 3)
constexpr int kCtrlEbar = kSlots * 4;
constexpr int kCtrlEsum = kCtrlEbar + 1;
constexpr int kCtrlMoved = kCtrlEbar + 2;

template <int TS>
struct TileGeom {
  static constexpr int TW = TS + 2;              // tile side with the halo ring
  static constexpr int HALO = 4 * TS + 4;        // halo ring nodes
  static constexpr int NODES = TS * TS;          // threads per group
  static constexpr int GROUPS = kTileCta / NODES;
  static constexpr int TP = (TS == 32) ? 40 : 24;  // row pitch: rows 8 banks apart, so
                                                   // a warp's 4 x 8 patch hits 32 banks
  static constexpr int PCOLS = TS / 8;           // 8-column patches per row of patches
  static_assert(TS == 16 || TS == 32, "tile side");
  static_assert(GROUPS * NODES == kTileCta, "groups fill the CTA");
};

// Shared memory of one tile group.
template <int TS>
struct alignas(16) GroupSmem {
  float4 q[kPlanes][TileGeom<TS>::NODES];                  // cone-form constants per node
  float Ts[2][TileGeom<TS>::TW][TileGeom<TS>::TP];         // T, double-buffered, with halo
  unsigned long long rowm[2][TileGeom<TS>::TW];            // change masks (see colspace)
  unsigned nkey[9];                                        // smallest changed boundary time per neighbour
  int par[9];                                              // round-start buffer of the 3 x 3 tiles
  int tile, go, first;
  unsigned key;
};

struct TileArgs {
  int ny, nx, ts, tny, tnx, ntiles;
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

// Named barrier of a tile group (ids 1..4; 0 is __syncthreads).
template <int N>
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ int group_sync_or(int id, int pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.s32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(pred), "r"(id), "n"(N)
      : "memory");
  return r;
}

// Change masks: one 64-bit word per frame row; bits 0..TS-1 are the interior
// columns (byte k written by the warps of patch column k), bit TS the left
// halo column, bit TS+1 the right one.  colspace() maps a word to frame
// column order (bit c = frame column c).
template <int TS>
__device__ __forceinline__ unsigned long long colspace(unsigned long long w) {
  constexpr unsigned long long lo = (1ull << TS) - 1ull;
  return ((w & lo) << 1) | ((w >> TS) & 1ull) | (((w >> (TS + 1)) & 1ull) << (TS + 1));
}
template <int TS>
__device__ __forceinline__ unsigned long long frame_bit(int c) {
  return c == 0 ? (1ull << TS) : (c == TS + 1) ? (1ull << (TS + 1)) : (1ull << (c - 1));
}

// Halo index -> (row, column) in the tile frame.
template <int TS>
__device__ __forceinline__ void halo_rc(int k, int &r, int &c) {
  constexpr int TW = TS + 2;
  if (k < TW) { r = 0; c = k; }
  else if (k < 2 * TW) { r = TW - 1; c = k - TW; }
  else if (k < 2 * TW + TS) { r = 1 + (k - 2 * TW); c = 0; }
  else { r = 1 + (k - 2 * TW - TS); c = TW - 1; }
}

// Buffer holding a tile's version as of the start of round r.
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

template <int TS>
__global__ void __launch_bounds__(kTileCta, 1) tile_solve_kernel(TileArgs a) {
  using G = TileGeom<TS>;
  constexpr int NG = G::NODES;
  extern __shared__ float4 smem4[];
  const int tid = threadIdx.x;
  const int grp = tid / NG, gt = tid - grp * NG;  // group and thread within it
  GroupSmem<TS> &S = reinterpret_cast<GroupSmem<TS> *>(smem4)[grp];
  const int bar = 1 + grp;
  // warp w of the group owns the 8 x 4 patch (w / PCOLS, w % PCOLS)
  const int lane = gt & 31, wp = gt >> 5;
  const int pr = wp / G::PCOLS, pc = wp % G::PCOLS, ao = lane >> 3;
  const int row = pr * 4 + ao, col = pc * 8 + (lane & 7);
  const int sr = row + 1, sc = col + 1;

  const TileWork &w = a.w;
  const int NT = a.ntiles;
  const long long plane = (long long)a.ny * a.nx;
  TileSlot *slots = reinterpret_cast<TileSlot *>(w.ctrl);
  unsigned *moved_ct = w.ctrl + kCtrlMoved;
  unsigned long long my_updates = 0, my_warp_evals = 0;
  bool converged = false, abort = false, prev_cert = false;
  int r = 1;
  const float ebar = __uint_as_float(w.ctrl[kCtrlEbar]);  // mean edge cost (seed kernel)
  const float delta = a.window * (float)TS * ebar;

  for (;; ++r) {
    TileSlot *cur = slots + (r % kSlots);
    if (blockIdx.x == 0 && tid == 0) {
      // the slot last used two rounds ago is free: ready it for round r + 2
      TileSlot *old = slots + ((r + 2) % kSlots);
      old->count = 0;
      old->grab = 0;
      old->kmin = kInfBits;
      // round r - 2's moved count was read at the start of round r - 1
      moved_ct[(r + 1) % kSlots] = 0u;
    }
    unsigned n = __ldcg(&cur->count);
    // an empty queue: done if the previous round certified without a change,
    // else certify (every tile, every node evaluated)
    const bool cert = n == 0;
    if (cert) {
      if (prev_cert && __ldcg(&moved_ct[(r + 2) % kSlots]) == 0u) {
        converged = true;
        break;
      }
      n = (unsigned)NT;
    }
    prev_cert = cert;
    if (r > a.max_rounds) break;
    const float theta = cert ? kInf : __uint_as_float(__ldcg(&cur->kmin)) + delta;

    while (true) {
      if (gt == 0) {
        const unsigned k = atomicAdd(&cur->grab, 1u);
        S.go = k < n;
        if (k < n && cert) {
          S.tile = (int)k;
          S.key = 0u;
        } else if (k < n) {
          const int t = __ldcg(&w.list[(size_t)(r % kSlots) * NT + k]);
          S.tile = t;
          unsigned *kp = &w.key[(size_t)(r & 1) * NT + t];
          S.key = __ldcg(kp);
          __stcg(kp, kInfBits);
        }
      }
      group_sync<NG>(bar);
      if (!S.go) break;
      const int t = S.tile;
      const unsigned kb = S.key;
      if (__uint_as_float(kb) > theta) {
        // too far ahead of the front: keep it for a later round
        if (gt == 0) push(w, NT, t, r + 1, kb);
        group_sync<NG>(bar);
        continue;
      }
      const int ti = t / a.tnx, tj = t - ti * a.tnx;
      const int i0 = ti * TS, j0 = tj * TS;
      // Everything that does not depend on the neighbours' buffer parities is
      // requested first, so that a visit pays two dependent global round
      // trips (parities, then T) instead of one per step.
      const int i = i0 + row, j = j0 + col;
      const bool inb = (i < a.ny) && (j < a.nx);
      const long long p = (long long)i * a.nx + j;
      float fl[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      bool is_src = false;
      if (inb) {
#pragma unroll
        for (int c = 0; c < 5; ++c) fl[c] = __ldg(a.f + c * plane + p);
        is_src = a.src[p] != 0;
      }
      int hr = 0, hc = 0, gi = -1, gj = -1;
      float prev = kInf;
      float *hp = nullptr;
      if (gt < G::HALO) {
        halo_rc<TS>(gt, hr, hc);
        gi = i0 - 1 + hr;
        gj = j0 - 1 + hc;
        hp = w.halo + (size_t)t * G::HALO + gt;
        prev = __ldcg(hp);
      }
      // buffer parities of this tile and its eight neighbours as of the
      // round's start (index (di + 1) * 3 + (dj + 1)); the first-visit flag
      if (gt < 9) {
        const int di = gt / 3 - 1, dj = gt % 3 - 1;
        const int ni = ti + di, nj = tj + dj;
        int pp = 0;
        if (ni >= 0 && ni < a.tny && nj >= 0 && nj < a.tnx)
          pp = start_parity(__ldcg(&w.tstate[ni * a.tnx + nj]), r);
        S.par[gt] = pp;
        S.nkey[gt] = kInfBits;
      }
      if (gt == 9) S.first = __ldcg(&w.visits[t]) == 0u;
      if (gt < G::TW) {
        S.rowm[0][gt] = 0ull;
        S.rowm[1][gt] = 0ull;
      }
      // this thread's node: cone-form constants into shared memory
      if (inb) {
        float4 q[kPlanes];
        node_record(fl[0], fl[1], fl[2], fl[3], fl[4], a.h, a.eps, is_src, q);
#pragma unroll
        for (int c = 0; c < kPlanes; ++c) S.q[c][gt] = q[c];
      }
      group_sync<NG>(bar);
      const int pt = S.par[4];
      float *Tout = a.T[1 - pt];
      float tcur = inb ? __ldcg(a.T[pt] + p) : kInf;
      // halo ring, from the neighbours' round-start versions; nodes whose
      // value differs from this tile's previous visit seed the change masks
      if (gt < G::HALO) {
        float v = kInf;
        if (gi >= 0 && gi < a.ny && gj >= 0 && gj < a.nx) {
          const int di = (hr == 0) ? -1 : (hr == G::TW - 1) ? 1 : 0;
          const int dj = (hc == 0) ? -1 : (hc == G::TW - 1) ? 1 : 0;
          v = __ldcg(a.T[S.par[(di + 1) * 3 + dj + 1]] + (long long)gi * a.nx + gj);
        }
        S.Ts[0][hr][hc] = v;
        S.Ts[1][hr][hc] = v;
        if (node_changed(v, prev, a.tol, a.rtol)) atomicOr(&S.rowm[0][hr], frame_bit<TS>(hc));
        __stcg(hp, v);
      }
      const bool upd = inb && !is_src;
      const float tinit = tcur;
      S.Ts[0][sr][sc] = tcur;
      S.Ts[1][sr][sc] = tcur;
      // first visit: the sources (cold) or every node (warm) start changed;
      // a certification visit evaluates every node
      if (S.first || cert) {
        const bool seed = inb && (a.warm || cert || is_src);
        const unsigned bal = __ballot_sync(0xffffffffu, seed);
        const unsigned long long byte = (bal >> (8 * ao)) & 0xffu;
        if ((lane & 7) == 0 && byte) atomicOr(&S.rowm[0][sr], byte << (8 * pc));
      }
      group_sync<NG>(bar);

      // Jacobi iterations with the halo fixed
      int cb = 0, it = 0;
      bool capped = false;
      while (true) {
        const unsigned long long nb =
            ((colspace<TS>(S.rowm[cb][sr - 1]) | colspace<TS>(S.rowm[cb][sr + 1])) >> (sc - 1)) & 7ull |
            ((colspace<TS>(S.rowm[cb][sr]) >> (sc - 1)) & 5ull);
        const unsigned dball = __ballot_sync(0xffffffffu, nb != 0ull && upd);
        float tnew = tcur;
        if (dball) {
          if (upd) {
            float Tn[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) Tn[k] = S.Ts[cb][sr + nb_dy(k)][sc + nb_dx(k)];
            tnew = cone_min(S.q[0][gt], S.q[1][gt], S.q[2][gt], S.q[3][gt], S.q[4][gt], S.q[5][gt], Tn);
          }
          if (lane == 0) {
            my_updates += (unsigned long long)__popc(dball);
            my_warp_evals += 1;
          }
        }
        S.Ts[cb ^ 1][sr][sc] = tnew;
        const bool ch = upd && node_changed(tnew, tcur, a.tol, a.rtol);
        const unsigned cbal = __ballot_sync(0xffffffffu, ch);
        // this warp's byte of each of its four rows (plain byte stores: the
        // patch columns of a row write disjoint bytes)
        if ((lane & 7) == 0)
          reinterpret_cast<unsigned char *>(&S.rowm[cb ^ 1][sr])[pc] = (unsigned char)((cbal >> (8 * ao)) & 0xffu);
        // slot 0 still holds the initial halo bits, read only by iteration 0:
        // clear them before iteration 2 reads the slot again (the halo bytes
        // of interior rows; halo rows entirely)
        if (it == 1 && gt < G::TW) {
          unsigned char *bytes = reinterpret_cast<unsigned char *>(&S.rowm[0][gt]);
          const int from = (gt == 0 || gt == G::TW - 1) ? 0 : TS / 8;
          for (int b = from; b < 8; ++b) bytes[b] = 0;
        }
        tcur = tnew;
        const int any = group_sync_or<NG>(bar, ch);
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
      if (group_sync_or<NG>(bar, moved)) {
        if (inb) __stcg(Tout + p, tcur);
        if (moved) {
          const unsigned kbits = __float_as_uint(tcur);
          const bool top = row == 0, bot = row == TS - 1, lft = col == 0, rgt = col == TS - 1;
          if (top) atomicMin(&S.nkey[1], kbits);
          if (bot) atomicMin(&S.nkey[7], kbits);
          if (lft) atomicMin(&S.nkey[3], kbits);
          if (rgt) atomicMin(&S.nkey[5], kbits);
          if (top && lft) atomicMin(&S.nkey[0], kbits);
          if (top && rgt) atomicMin(&S.nkey[2], kbits);
          if (bot && lft) atomicMin(&S.nkey[6], kbits);
          if (bot && rgt) atomicMin(&S.nkey[8], kbits);
        }
        group_sync<NG>(bar);
        if (gt == 0) {
          __stcg(&w.tstate[t], ((unsigned)r << 1) | (unsigned)(1 - pt));
          atomicAdd(&moved_ct[r % kSlots], 1u);
        }
        if (gt < 9 && gt != 4 && S.nkey[gt] != kInfBits) {
          const int ni = ti + gt / 3 - 1, nj = tj + gt % 3 - 1;
          if (ni >= 0 && ni < a.tny && nj >= 0 && nj < a.tnx) push(w, NT, ni * a.tnx + nj, r + 1, S.nkey[gt]);
        }
      }
      if (gt == 0) {
        __stcg(&w.visits[t], __ldcg(&w.visits[t]) + 1u);
        // a visit cut short by the iteration cap is resumed next round
        if (capped) push(w, NT, t, r + 1, kb);
      }
      group_sync<NG>(bar);
    }
    if (!grid_sync(a.ctl)) {  // begins with __syncthreads: every group is done
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
    for (long long q = (long long)blockIdx.x * blockDim.x + tid; q < plane; q += (long long)gridDim.x * blockDim.x) {
      const int qi = (int)(q / a.nx), qj = (int)(q - (long long)qi * a.nx);
      if (__ldcg(&w.tstate[(qi / TS) * a.tnx + qj / TS]) & 1u) a.T[0][q] = __ldcg(a.T[1] + q);
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    a.ctl.st->rounds = (unsigned)(r - 1);
    a.ctl.st->converged = converged ? 1 : 0;
    if (!converged && !abort) set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
  }
}

// Workspace reset and the mean edge cost of the field (mean of
// (|m_x|_M + |m_y|_M) / 2, the time scale of the delta-stepping window).
__global__ void tile_seed_kernel(TileArgs a, float *esum) {
  const TileWork &w = a.w;
  const int NT = a.ntiles;
  const int halo = 4 * a.ts + 4;
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
    w.queued[t] = a.warm ? 1u : 0u;
  }
  for (long long k = g0; k < (long long)NT * halo; k += stride) w.halo[k] = kInf;
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
// (warm) or every tile that holds a source or one of its neighbours (cold: a
// source never changes, so the tiles across a tile edge next to it must see
// it in their halo on their own first visit).
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
  const long long plane = (long long)a.ny * a.nx;
  for (long long p = g0; p < plane; p += stride) {
    if (!a.src[p]) continue;
    const int i = (int)(p / a.nx), j = (int)(p - (long long)i * a.nx);
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj) {
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || ii >= a.ny || jj < 0 || jj >= a.nx) continue;
        const int t = (ii / a.ts) * a.tnx + jj / a.ts;
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
  a.w.ctrl[kCtrlEbar] = __float_as_uint(ebar > 0.0f && ebar < kInf ? ebar : 1.0f);
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

int tile_side(int requested) { return requested >= 32 ? 32 : 16; }

int tiles_count(int ny, int nx, int ts) { return ((ny + ts - 1) / ts) * ((nx + ts - 1) / ts); }

size_t tile_work_bytes(int ny, int nx, int ts) {
  const size_t NT = (size_t)tiles_count(ny, nx, ts);
  // counters, ctrl, then tstate, visits, queued, key[2], list[3], halo
  return 64 + 256 + NT * 4 * 5 + NT * 4 * kSlots + NT * (size_t)(4 * ts + 4) * 4;
}

TileWork tile_work_carve(void *base, int ny, int nx, int ts) {
  const size_t NT = (size_t)tiles_count(ny, nx, ts);
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

template <int TS>
static rf_status launch_solve(TileArgs &a, int num_sms, cudaStream_t s) {
  const size_t smem = sizeof(GroupSmem<TS>) * TileGeom<TS>::GROUPS;
  if (cudaFuncSetAttribute(tile_solve_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_solve_kernel<TS>, kTileCta, smem) != cudaSuccess)
    return RF_ERR_CUDA;
  if (per_sm < 1) return RF_ERR_UNSUPPORTED;
  void *args[] = {&a};
  return cuda_status(cudaLaunchCooperativeKernel((const void *)tile_solve_kernel<TS>, dim3(per_sm * num_sms),
                                                 dim3(kTileCta), args, smem, s));
}

rf_status tiles_launch(int num_sms, int ny, int nx, int ts, float h, float eps, const float *proj5,
                       const uint8_t *src, float *T, float *Tb, int warm, int max_sweeps, float tol, float rtol,
                       float window, const TileWork &w, const LaunchCtl &ctl, cudaStream_t s) {
  TileArgs a;
  a.ny = ny;
  a.nx = nx;
  a.ts = ts;
  a.tny = (ny + ts - 1) / ts;
  a.tnx = (nx + ts - 1) / ts;
  a.ntiles = a.tny * a.tnx;
  a.h = h;
  a.eps = eps;
  a.f = proj5;
  a.src = src;
  a.T[0] = T;
  a.T[1] = Tb;
  a.tol = tol;
  a.rtol = rtol;
  a.window = window > 0.0f ? window : (ts == 32 ? 2.0f : 4.0f);
  a.warm = warm;
  // a sweep moves information across the grid, a round across one tile
  a.max_rounds = max_sweeps * std::max(a.tny, a.tnx);
  a.max_local = 16 * ts;
  a.w = w;
  a.ctl = ctl;
  if (cudaMemsetAsync(w.counters, 0, 64 + 256, s) != cudaSuccess) return RF_ERR_CUDA;
  float *esum = (float *)(w.ctrl + kCtrlEsum);
  const long long n = (long long)ny * nx;
  const int blocks = blocks_for(std::max(n, (long long)a.ntiles * (4 * ts + 4)), 256, num_sms * 8);
  tile_seed_kernel<<<blocks, 256, 0, s>>>(a, esum);
  tile_queue_kernel<<<blocks, 256, 0, s>>>(a);
  tile_finish_seed_kernel<<<1, 32, 0, s>>>(a, esum);
  const rf_status rs = ts == 32 ? launch_solve<32>(a, num_sms, s) : launch_solve<16>(a, num_sms, s);
  if (rs != RF_OK) return rs;
  tile_stats_kernel<<<1, 32, 0, s>>>(w.counters, ctl.st, n);
  return cuda_status(cudaGetLastError());
}

}  // namespace rf
