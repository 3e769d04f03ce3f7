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
//    queued tiles whose key is within a window of the previous round's
//    smallest key and defers the others (delta-stepping on tiles: tiles far
//    ahead of the front would only be revisited once the front reaches them);
//  * tiles read their neighbours' state as of the start of the round: every
//    tile's latest version lives in one of two T buffers, tagged per tile
//    with (round written, parity); a tile writes its new version into the
//    other buffer, so results do not depend on the order in which tiles are
//    taken, and the solve is deterministic;
//  * there is no grid barrier between rounds: a group moves on to round r + 1
//    once round r's list is final (round r - 1 complete) and handed out, and
//    a tile of round r + 1 starts once no tile of its 3 x 3 neighbourhood is
//    pending in round r (a pending-round bit per tile and round mod 8), so it
//    reads exactly what a barrier would have given it while the slowest
//    visits of round r still run elsewhere; a round's completion is counted
//    in one word per round (see complete_round);
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
//
// The same kernel solves a batch of grids (rf_batch_solve, Sec. 3.4's
// batched solves): the grids' tiles share one queue, each tile knows its
// grid (per-grid descriptor: shape, spacing, offsets into the packed
// arrays), and keys are normalised per grid to tile crossings (T divided by
// tile side x mean edge cost), so a window means the same front advance on
// every grid whatever its size.  A single grid is a batch of one.
#include <algorithm>

#include "rf_cone.cuh"
#include "rf_ctx.h"
#include "rf_sweep_common.cuh"
#include "rf_sweep_tiles.h"

namespace rf {

constexpr int kTileCta = 1024;     // threads per CTA with 32 x 32 tiles (one tile group)
// threads per CTA with 16 x 16 tiles (four tile groups).  Fewer groups per
// SM leave registers for each but fewer visits in flight: 2048^2 forward
// 4.51 / 4.61 / 5.50 ms at 4 / 3 / 2 groups (window 2)
constexpr int kTileCta16 = 1024;
constexpr unsigned kInfBits = 0x7f800000u;
constexpr int kSlots = 8;          // round slots (round mod 8)
constexpr int kKeySlots = 4;       // queue-key slots (round mod 4)

// Control words of one round slot (32 bytes).  A slot serves round r, then
// round r + 8: it is reset for its next round when round r + 4 completes.
struct TileSlot {
  unsigned long long take;  // (round << 32) | list entries handed out past the groups' own first ones
  unsigned count;           // tiles queued for the round
  unsigned kmin;            // float bits of the smallest queued key
  unsigned done;            // entries finished; kPrevDone - (entries) added once the previous round is complete
  unsigned moved;           // tiles that published a new version in the round
  unsigned pad0;
  unsigned round;           // round the slot serves
};
// ctrl layout (unsigned words): 8 slots x 8 words, then the tile count, the
// last round up to which every round is complete, the stop flag (1
// converged, 2 round cap) and the rounds of the solve
constexpr int kCtrlNT = kSlots * 8;
constexpr int kCtrlComplete = kCtrlNT + 1;
constexpr int kCtrlStop = kCtrlNT + 2;
constexpr int kCtrlRounds = kCtrlNT + 3;
constexpr int kCtrlBytes = 512;
static_assert(sizeof(TileSlot) == 32, "slot layout");
static_assert((kCtrlRounds + 1) * 4 <= kCtrlBytes, "ctrl words");

template <int TS>
struct TileGeom {
  static constexpr int TW = TS + 2;              // tile side with the halo ring
  static constexpr int HALO = 4 * TS + 4;        // halo ring nodes
  static constexpr int NODES = TS * TS;          // threads per group
  static constexpr int CTA = TS == 16 ? kTileCta16 : kTileCta;
  static constexpr int GROUPS = CTA / NODES;
  static constexpr int TP = (TS == 32) ? 40 : 24;  // row pitch: rows 8 banks apart, so
                                                   // a warp's 4 x 8 patch hits 32 banks
  static constexpr int PCOLS = TS / 8;           // 8-column patches per row of patches
  static_assert(TS == 16 || TS == 32, "tile side");
  static_assert(GROUPS * NODES == CTA, "groups fill the CTA");
};

// Shared memory of one tile group.
template <int TS>
struct alignas(16) GroupSmem {
  float4 q[kPlanes][TileGeom<TS>::NODES];                  // cone-form constants per node
  float Ts[2][TileGeom<TS>::TW][TileGeom<TS>::TP];         // T, double-buffered, with halo
  unsigned long long rowm[2][TileGeom<TS>::TW];            // change masks (see colspace)
  unsigned nkey[9];                                        // smallest changed boundary time per neighbour
  int par[9];                                              // round-start buffer of the 3 x 3 tiles
  float t0[TileGeom<TS>::NODES];  // node values at the start of the visit
  TGrid gd;      // grid of the current tile
  int tile, go, first, gid;
  int mdefer;  // the key read before the neighbourhood was ready is above the threshold
  unsigned key;
  unsigned tsw;  // the tile's state word without its pending bits, as of the visit's start
  unsigned upd;  // node updates of the current visit
};

struct TileArgs {
  int n_grids, ts, ntiles_cap;  // tiles of all grids <= ntiles_cap (strides of the queue arrays)
  long long plane;              // nodes of all grids: plane stride of the 5-plane fields
  float eps;
  const float *f;
  const uint8_t *src;
  float *T[2];  // buffer 0 = the caller's T, buffer 1 = workspace
  float tol, rtol;
  float window;  // delta-stepping window in tile crossings
  float tau;     // soft-min temperature (the SOFT kernels only)
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

// Tile state word: pending-round bits 0..7 (bit r mod 8 set while the tile
// is queued for round r and that round's visit has not finished), the
// parity of the buffer holding its latest version (bit 8) and the round that
// version was written in (bits 9..31).
constexpr unsigned kPendMask = 0xffu;
constexpr unsigned kPrevDone = 0x80000000u;  // TileSlot::done: the previous round is complete
__device__ __forceinline__ bool pending_in(unsigned st, int r) { return (st >> (r & 7)) & 1u; }

// Buffer holding a tile's version as of the start of round r.
__device__ __forceinline__ int start_parity(unsigned st, int r) {
  const int par = (int)((st >> 8) & 1u);
  return ((int)(st >> 9) == r) ? 1 - par : par;
}

__device__ __forceinline__ TileSlot &slot_of(const TileWork &w, int r) {
  return reinterpret_cast<TileSlot *>(w.ctrl)[r % kSlots];
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void fence_sc() { asm volatile("fence.sc.gpu;" ::: "memory"); }

// Append tile t to round rr's list unless it is already pending there.  The
// entry carries its round, so a reader never takes a stale entry of the
// slot's previous round.
__device__ __forceinline__ void enqueue(const TileWork &w, int ntiles, int t, int rr) {
  const unsigned bit = 1u << (rr & 7);
  if (!(atomicOr(&w.tstate[t], bit) & bit)) {
    const unsigned idx = atomicAdd(&slot_of(w, rr).count, 1u);
    st_release_u64(&w.list[(size_t)(rr % kSlots) * ntiles + idx], ((unsigned long long)rr << 32) | (unsigned)t);
  }
}

// Queue tile t for round rr with key bits kb.
__device__ __forceinline__ void push(const TileWork &w, int ntiles, int t, int rr, unsigned kb) {
  atomicMin(&w.key[(size_t)(rr % kKeySlots) * ntiles + t], kb);
  atomicMin(&slot_of(w, rr).kmin, kb);
  enqueue(w, ntiles, t, rr);
}

__device__ __forceinline__ void reset_slot(TileSlot &s, int r) {
  s.round = 0xffffffffu;  // readers that see a reset field see this first
  __threadfence();
  s.count = 0u;
  s.kmin = kInfBits;
  s.done = 0u;
  s.moved = 0u;
  s.round = (unsigned)r;
  __threadfence();
  s.take = (unsigned long long)(unsigned)r << 32;
}

// Round completion.  Round q is complete when round q - 1 is and all its
// entries are done; both facts meet in one word: every finished entry adds 1
// to TileSlot::done, and the completer of q - 1, which knows the final entry
// count n of q, adds kPrevDone - n, so the word equals kPrevDone exactly when
// both happened, and exactly one atomic (the last of them) produces that
// value: its thread completes the round.  The completer
// decides on round q + 1, whose list is final now (converged: q + 1 would
// certify after a certification round q that moved nothing; stop at the
// round cap), readies the slot of round q + 4, publishes the completion and
// passes kPrevDone on to round q + 1, completing that round too if its
// entries are all done already.
__device__ void complete_round(const TileWork &w, int q, int ntiles_all, int max_rounds) {
  unsigned *ctrl = w.ctrl;
  for (int guard = 0; guard < (1 << 20); ++guard, ++q) {
    __threadfence();  // every entry's effects, seen through the done word, before what follows
    TileSlot &s = slot_of(w, q);
    const unsigned cnt = __ldcg(&s.count);
    const unsigned cnt1 = __ldcg(&slot_of(w, q + 1).count);
    if (cnt == 0u && cnt1 == 0u && __ldcg(&s.moved) == 0u) {
      ctrl[kCtrlRounds] = (unsigned)q;
      ctrl[kCtrlStop] = 1u;
    } else if (q + 1 > max_rounds) {
      ctrl[kCtrlRounds] = (unsigned)q;
      ctrl[kCtrlStop] = 2u;
    }
    reset_slot(slot_of(w, q + 4), q + 4);
    __threadfence();
    st_release_u32(&ctrl[kCtrlComplete], (unsigned)q);
    const unsigned n1 = cnt1 ? cnt1 : (unsigned)ntiles_all;
    const unsigned old = atomicAdd(&slot_of(w, q + 1).done, kPrevDone - n1);
    if (old + (kPrevDone - n1) != kPrevDone) return;
  }
}

// End of an entry of round rg (a visit or a deferral), by one thread after
// the group's stores and queue pushes: the tile is no longer pending in rg,
// and the round counts the entry.
// End of an entry of round rg (a visit or a deferral), by one thread after
// the group's stores and queue pushes, in two halves so that the group's
// next ticket is requested while the count is in flight: the tile is no
// longer pending in rg, and the round counts the entry.
__device__ __forceinline__ unsigned finish_begin(const TileWork &w, int t, int rg) {
  __threadfence();  // the group's stores and pushes, ordered by its barrier, before both words
  atomicAnd(&w.tstate[t], ~(1u << (rg & 7)));
  return atomicAdd(&slot_of(w, rg).done, 1u);
}
__device__ __forceinline__ void finish_end(const TileWork &w, int rg, unsigned old, int ntiles_all, int max_rounds) {
  if (old + 1u == kPrevDone) complete_round(w, rg, ntiles_all, max_rounds);
}

// SOFT: the node update is the soft-min relaxation (cone_softmin; a value
// below zero means no finite fixed point: RF_ERR_NOT_CONVERGED, the launch
// stops) instead of the minimum.
template <int TS, bool SOFT>
__global__ void __launch_bounds__(TileGeom<TS>::CTA, 1) tile_solve_kernel(TileArgs a) {
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
  const int NT = (int)w.ctrl[kCtrlNT];  // tiles of all grids
  const int NC = a.ntiles_cap;          // stride of the per-round queue arrays
  const long long plane = a.plane;
  unsigned long long my_warp_evals = 0;
  bool abort = false;
  // Rounds without a grid barrier: a group takes entries of its round rg
  // until the round's list is final and exhausted, then moves to rg + 1.  A
  // taken tile waits until no tile of its 3 x 3 neighbourhood is pending in
  // round rg - 1; its visit then reads exactly the versions the neighbourhood
  // had at the end of round rg - 1, as with a barrier between rounds, so the
  // result does not depend on timing.  Rounds rg and rg + 1 overlap.
  int rg = 1;
  int fin_t = -1, fin_rg = 0;  // thread 0: an entry whose end is still to be counted
  unsigned long long pre = 0ull;  // thread 0: a ticket of round rg requested during the last visit
  bool have_pre = false;

  while (true) {
    if (gt == 0) {
      // code: 0 list entry, 1 certification entry, 2 nothing more in round
      // rg for this group, 3 stop (converged, round cap, timeout)
      int code = -1, t = -1;
      unsigned k = 0;
      TileSlot &sl = slot_of(w, rg);
      {
        // a ticket: the next list index of round rg.  A slot is reset for
        // its next round only once round rg + 4 is complete, and round rg
        // cannot complete before this group's previous entry of it did, so
        // the tag check below never fails for a group that just finished
        // an entry; it guards a group arriving from an older round.
        unsigned fold = 0u;
        const int frg = fin_rg;
        if (fin_t >= 0) fold = finish_begin(w, fin_t, fin_rg);
        const unsigned long long v = have_pre ? pre : atomicAdd(&sl.take, 1ull);
        have_pre = false;
        if (fin_t >= 0) {
          // before any wait: the round may be waiting for this count
          finish_end(w, frg, fold, NT, a.max_rounds);
          fin_t = -1;
        }
        if ((unsigned)(v >> 32) != (unsigned)rg) code = 2;
        k = (unsigned)v;
      }
      const unsigned long long t0 = gtimer();
      for (unsigned spins = 0; code < 0; ++spins) {
        // the entry itself first: its tag names the round that wrote it
        if (k < (unsigned)NC) {
          const unsigned long long e = ld_acquire_u64(&w.list[(size_t)(rg % kSlots) * NC + k]);
          if ((unsigned)(e >> 32) == (unsigned)rg) {
            t = (int)(unsigned)e;
            code = 0;
            break;
          }
        }
        // loads after an acquire are ordered after it
        const int comp = (int)ld_acquire_u32(&w.ctrl[kCtrlComplete]);
        const unsigned stop = __ldcg(&w.ctrl[kCtrlStop]);
        const unsigned cnt = __ldcg(&sl.count);
        const unsigned srnd = __ldcg(&sl.round);
        if (stop || ld_acquire_s32(a.ctl.abort)) {
          code = 3;
          break;
        }
        if (comp >= rg || srnd != (unsigned)rg) {  // round rg complete: every entry was taken
          code = 2;
          break;
        }
        if (comp >= rg - 1) {  // round rg's list is final
          if (cnt == 0u) {
            // an empty list: certification round (its tiles are not marked
            // pending, so no group moves past it before it completes: that
            // wait ends through comp >= rg above)
            if (k < (unsigned)NT) {
              t = (int)k;
              code = 1;
              break;
            }
          } else if (k >= cnt) {
            code = 2;
            break;
          }
        }
        if ((spins & 15u) == 15u && (long long)(gtimer() - t0) > a.ctl.timeout_ns) {
          raise_timeout(a.ctl);
          code = 3;
          break;
        }
        __nanosleep(64);
      }
      S.go = code;
      S.tile = t;
      S.key = 0u;
      if (t >= 0) {
        const int gid = a.n_grids == 1 ? 0 : __ldg(&w.tile_grid[t]);
        S.gid = gid;
        S.gd = w.grids[gid];
      }
    }
    group_sync<NG>(bar);
    const int code = S.go;
    if (code == 3) break;
    if (code == 2) {
      // on to the next round (or past rounds completed meanwhile)
      if (gt == 0) S.tile = max(rg + 1, (int)ld_acquire_u32(&w.ctrl[kCtrlComplete]) + 1);
      group_sync<NG>(bar);
      rg = S.tile;
      group_sync<NG>(bar);
      continue;
    }
    const int t = S.tile;
    const bool cert = code == 1;
    const int gid = S.gid;
    const TGrid &gd = S.gd;
    const int tl = t - gd.tile_off;
    const int ti = tl / gd.tnx, tj = tl - ti * gd.tnx;
    const int i0 = ti * TS, j0 = tj * TS;
    const int gny = gd.ny, gnx = gd.nx;
    const long long goff = gd.node_off;
    const int i = i0 + row, j = j0 + col;
    const bool inb = (i < gny) && (j < gnx);
    const long long p = goff + (long long)i * gnx + j;
    // the inputs that no visit writes first: fields, source flag, the halo
    // this tile saw at its previous visit
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
    // readiness: no tile of the 3 x 3 neighbourhood (index (di + 1) * 3 +
    // (dj + 1)) pending in round rg - 1; the same words give the buffer
    // parities as of the round's start
    if (gt < 9) {
      const int ni = ti + gt / 3 - 1, nj = tj + gt % 3 - 1;
      int pp = 0;
      if (ni >= 0 && ni < gd.tny && nj >= 0 && nj < gd.tnx) {
        const unsigned *sp = &w.tstate[gd.tile_off + ni * gd.tnx + nj];
        unsigned st = ld_acquire_u32(sp);
        const unsigned long long t0 = gtimer();
        for (unsigned spins = 0; pending_in(st, rg - 1); ++spins) {
          if ((spins & 15u) == 15u &&
              ((long long)(gtimer() - t0) > a.ctl.timeout_ns || ld_acquire_s32(a.ctl.abort))) {
            raise_timeout(a.ctl);
            break;
          }
          __nanosleep(32);
          st = ld_acquire_u32(sp);
        }
        pp = start_parity(st, rg);
        if (gt == 4) S.tsw = st & ~kPendMask;
      }
      S.par[gt] = pp;
      S.nkey[gt] = kInfBits;
    }
    unsigned nvis = 0u;
    if (gt == 9) {
      nvis = __ldcg(&w.visits[t]);
      S.first = nvis == 0u;
    }
    if (gt == 10) {
      // keys only decrease: a key already at or below the threshold stays so
      int md = 0;
      if (!cert) {
        const unsigned k0 = __ldcg(&w.key[(size_t)(rg % kKeySlots) * NC + t]);
        md = __uint_as_float(k0) > __uint_as_float(ld_acquire_u32(&slot_of(w, rg - 1).kmin)) + a.window;
      }
      S.mdefer = md;
    }
    if (gt < G::TW) {
      S.rowm[0][gt] = 0ull;
      S.rowm[1][gt] = 0ull;
    }
    if (gt == 0) S.upd = 0u;
    group_sync<NG>(bar);
    if (S.mdefer) {
      // likely too far ahead of the front: decide on the final key (only the
      // neighbourhood's round rg - 1 visits queue this tile for round rg, and
      // they are done) before anything else is loaded
      if (gt == 0) {
        unsigned *kp = &w.key[(size_t)(rg % kKeySlots) * NC + t];
        const unsigned kbits = __ldcg(kp);
        const float theta = __uint_as_float(ld_acquire_u32(&slot_of(w, rg - 1).kmin)) + a.window;
        int defer = 0;
        if (__uint_as_float(kbits) > theta) {
          // keep it for a later round
          __stcg(kp, kInfBits);
          push(w, NC, t, rg + 1, kbits);
          fin_t = t;
          fin_rg = rg;
          defer = 1;
        }
        S.go = defer;
      }
      group_sync<NG>(bar);
      const int deferred = S.go;
      group_sync<NG>(bar);
      if (deferred) continue;
    }
    // T of the node and of its halo node from the round-start buffers
    const int pt = S.par[4];
    float *Tout = a.T[1 - pt];
    float tcur = inb ? __ldcg(a.T[pt] + p) : kInf;
    float hv = kInf;
    if (gt < G::HALO && gi >= 0 && gi < gny && gj >= 0 && gj < gnx) {
      const int di = (hr == 0) ? -1 : (hr == G::TW - 1) ? 1 : 0;
      const int dj = (hc == 0) ? -1 : (hc == G::TW - 1) ? 1 : 0;
      hv = __ldcg(a.T[S.par[(di + 1) * 3 + dj + 1]] + goff + (long long)gi * gnx + gj);
    }
    if (gt == 0) {
      // the final key (within the threshold now), kept for a capped visit
      unsigned kbits = 0u;
      if (!cert) {
        unsigned *kp = &w.key[(size_t)(rg % kKeySlots) * NC + t];
        kbits = __ldcg(kp);
        __stcg(kp, kInfBits);
      }
      S.key = kbits;
    }
    // this thread's node: cone-form constants into shared memory
    if (inb) {
      float4 q[kPlanes];
      node_record(fl[0], fl[1], fl[2], fl[3], fl[4], gd.h, a.eps, is_src, q);
#pragma unroll
      for (int c = 0; c < kPlanes; ++c) S.q[c][gt] = q[c];
    }
    group_sync<NG>(bar);
    const unsigned kb = S.key;
    if (gt == 9) __stcg(&w.visits[t], nvis + 1u);
    // halo ring, from the neighbours' round-start versions; nodes whose
    // value differs from this tile's previous visit seed the change masks
    if (gt < G::HALO) {
      const float v = hv;
      S.Ts[0][hr][hc] = v;
      S.Ts[1][hr][hc] = v;
      if (node_changed(v, prev, a.tol, a.rtol)) atomicOr(&S.rowm[0][hr], frame_bit<TS>(hc));
      __stcg(hp, v);
    }
    const bool upd = inb && !is_src;
    S.t0[gt] = tcur;
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
            if constexpr (SOFT) {
              tnew = cone_softmin(S.q[0][gt], S.q[1][gt], S.q[2][gt], S.q[3][gt], S.q[4][gt], S.q[5][gt], Tn,
                                  a.tau);
              if (tnew < 0.0f) {
                set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
                atomicExch(a.ctl.abort, 1);
              }
            } else {
              tnew = cone_min(S.q[0][gt], S.q[1][gt], S.q[2][gt], S.q[3][gt], S.q[4][gt], S.q[5][gt], Tn);
            }
          }
          if (lane == 0) {
            atomicAdd(&S.upd, (unsigned)__popc(dball));
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

      // the next ticket, requested while this visit publishes
      if (gt == 0) {
        pre = atomicAdd(&slot_of(w, rg).take, 1ull);
        have_pre = true;
      }
      // publish: a new version only if some node moved beyond the tolerance
      const bool moved = upd && node_changed(tcur, S.t0[gt], a.tol, a.rtol);
      if (group_sync_or<NG>(bar, moved)) {
        if (inb) __stcg(Tout + gd.node_off + (long long)(i0 + row) * gd.nx + (j0 + col), tcur);
        if (moved) {
          // key of the neighbours this node queues: its new time in tile
          // crossings of this grid
          const unsigned kbits = __float_as_uint(tcur * gd.inv_scale);
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
          // the new version's round and buffer, leaving the pending bits
          // (other tiles queue this one concurrently) untouched
          // (a reader that finds the new round takes the other buffer, the
          // round-start version; the new values become readable through the
          // fence before the pending bit is cleared at the entry's end)
          const unsigned nw = ((unsigned)rg << 9) | ((unsigned)(1 - pt) << 8);
          atomicXor(&w.tstate[t], S.tsw ^ nw);
          atomicAdd(&slot_of(w, rg).moved, 1u);
        }
        if (gt < 9 && gt != 4 && S.nkey[gt] != kInfBits) {
          const int ni = ti + gt / 3 - 1, nj = tj + gt % 3 - 1;
          // the neighbour's visit waits for this entry's end (readiness)
          if (ni >= 0 && ni < gd.tny && nj >= 0 && nj < gd.tnx)
            push(w, NC, gd.tile_off + ni * gd.tnx + nj, rg + 1, S.nkey[gt]);
        }
      }
      if (gt == 0) {
        if (S.upd) {
          atomicAdd(&w.gupd[gid], (unsigned long long)S.upd);
          atomicAdd(&w.counters[0], (unsigned long long)S.upd);
        }
        // a visit cut short by the iteration cap is resumed next round
        if (capped) push(w, NC, t, rg + 1, kb);
      }
      group_sync<NG>(bar);
      if (gt == 0) {
        // counted at the next take
        fin_t = t;
        fin_rg = rg;
      }
  }
  if (lane == 0 && my_warp_evals) atomicAdd(&w.counters[1], my_warp_evals);
  // one barrier at the end: every group has left the loop
  if (!grid_sync(a.ctl)) abort = true;
  if (!abort) {
    // hand the latest version of every tile back in the caller's buffer: a
    // tile per group, one thread per node
    for (int t = blockIdx.x * G::GROUPS + grp; t < NT; t += gridDim.x * G::GROUPS) {
      if (((__ldcg(&w.tstate[t]) >> 8) & 1u) == 0u) continue;
      const int gid = a.n_grids == 1 ? 0 : __ldg(&w.tile_grid[t]);
      const TGrid gd = w.grids[gid];
      const int tl = t - gd.tile_off;
      const int i = (tl / gd.tnx) * TS + row, j = (tl % gd.tnx) * TS + col;
      if (i < gd.ny && j < gd.nx) {
        const long long q = gd.node_off + (long long)i * gd.nx + j;
        a.T[0][q] = __ldcg(a.T[1] + q);
      }
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    const bool converged = !abort && __ldcg(&w.ctrl[kCtrlStop]) == 1u;
    a.ctl.st->rounds = __ldcg(&w.ctrl[kCtrlRounds]);
    a.ctl.st->converged = converged ? 1 : 0;
    if (!converged && !abort) set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
  }
}

// ---- seeding -----------------------------------------------------------------
// Plan of one grid (the single-grid entry point): its descriptor and the
// tile count.
__global__ void tile_plan_single_kernel(TileWork w, int ny, int nx, float h, int ts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  TGrid g;
  g.node_off = 0;
  g.ny = ny;
  g.nx = nx;
  g.tny = (ny + ts - 1) / ts;
  g.tnx = (nx + ts - 1) / ts;
  g.tile_off = 0;
  g.h = h;
  g.inv_scale = 0.0f;
  g.has_src = 0;
  g.esum_fx = 0ull;
  w.grids[0] = g;
  w.ctrl[kCtrlNT] = (unsigned)(g.tny * g.tnx);
}

// Plan of a batch: every grid's descriptor with its first tile (an
// exclusive scan of the tile counts, in descriptor order), and the tile
// count.  One CTA.  Descriptors that are not a valid packing (empty or
// non-positive spacing, outside [0, total), out of order or overlapping)
// raise RF_ERR_INVALID_ARG and leave every grid empty, so that no later
// kernel of the call touches memory through them.
__global__ void tile_plan_batch_kernel(TileWork w, const rf_batch_desc *descs, int n_grids, int ts,
                                       long long total, int max_line, int ntiles_cap, DevState *st) {
  __shared__ unsigned long long part[1024];
  __shared__ unsigned long long s_total;
  __shared__ int s_bad;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int per = (n_grids + nth - 1) / nth;
  const int g0 = tid * per, g1 = min(n_grids, g0 + per);
  if (tid == 0) s_bad = 0;
  __syncthreads();
  unsigned long long mine = 0;
  int bad = 0;
  for (int g = g0; g < g1; ++g) {
    const rf_batch_desc d = descs[g];
    const long long end = d.offset + (long long)d.ny * d.nx;
    bad |= d.ny < 1 || d.nx < 1 || d.ny > max_line || d.nx > max_line || !(d.h > 0.0f) || d.offset < 0 ||
           end > total || (g + 1 < n_grids && descs[g + 1].offset < end);
    if (!bad) mine += (unsigned long long)((d.ny + ts - 1) / ts) * (unsigned long long)((d.nx + ts - 1) / ts);
  }
  if (bad) atomicOr(&s_bad, 1);
  part[tid] = mine;
  __syncthreads();
  if (tid == 0) {
    unsigned long long run = 0;
    for (int k = 0; k < nth; ++k) {
      const unsigned long long v = part[k];
      part[k] = run;
      run += v;
    }
    s_total = run;
    // the workspace holds ntiles_cap tiles, a bound for any valid packing
    if (run > (unsigned long long)ntiles_cap) s_bad = 1;
  }
  __syncthreads();
  const bool any_bad = s_bad != 0;
  if (tid == 0) {
    w.ctrl[kCtrlNT] = any_bad ? 0u : (unsigned)s_total;
    if (any_bad) set_error(st, RF_ERR_INVALID_ARG);
  }
  unsigned long long off = any_bad ? 0ull : part[tid];
  for (int g = g0; g < g1; ++g) {
    const rf_batch_desc d = descs[g];
    TGrid t;
    t.node_off = any_bad ? 0 : d.offset;
    t.ny = any_bad ? 0 : d.ny;
    t.nx = any_bad ? 0 : d.nx;
    t.tny = (t.ny + ts - 1) / ts;
    t.tnx = (t.nx + ts - 1) / ts;
    t.tile_off = (int)off;
    t.h = any_bad ? 1.0f : d.h;
    t.inv_scale = 0.0f;
    t.has_src = 0;
    t.esum_fx = 0ull;
    w.grids[g] = t;
    off += (unsigned long long)t.tny * (unsigned long long)t.tnx;
  }
}

// tile -> grid map of a batch (blockIdx.y = grid).
__global__ void tile_map_kernel(TileWork w) {
  const TGrid g = w.grids[blockIdx.y];
  const int n = g.tny * g.tnx;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    w.tile_grid[g.tile_off + k] = (int)blockIdx.y;
}

// Workspace reset (tiles_cap tiles, every round list cleared) and the
// slots: slot k serves round k,
// round 0 is complete (the seed kernels fill round 1's list), and its kmin
// is 0 (round 1's threshold is the window).
__global__ void tile_reset_kernel(TileArgs a) {
  const TileWork &w = a.w;
  const int NC = a.ntiles_cap;
  const int halo = 4 * a.ts + 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g0 == 0) {
    TileSlot *slots = reinterpret_cast<TileSlot *>(w.ctrl);
    for (int k = 0; k < kSlots; ++k) {
      slots[k].take = (unsigned long long)(unsigned)k << 32;
      slots[k].count = 0u;
      slots[k].kmin = k == 0 ? 0u : kInfBits;
      slots[k].done = 0u;  // round 1's share of round 0's completion: tile_finish_seed_kernel
      slots[k].moved = 0u;
      slots[k].pad0 = 0u;
      slots[k].round = (unsigned)k;
    }
    w.ctrl[kCtrlComplete] = 0u;
    w.ctrl[kCtrlStop] = 0u;
    w.ctrl[kCtrlRounds] = 0u;
  }
  for (long long t = g0; t < NC; t += stride) {
    w.tstate[t] = a.warm ? (1u << 1) : 0u;  // warm: every tile pending in round 1
    w.visits[t] = 0u;
#pragma unroll
    for (int k = 0; k < kKeySlots; ++k) w.key[(size_t)k * NC + t] = kInfBits;
    // no entry of an earlier solve may carry a round of this one: a reader
    // that runs ahead of a producer's store must see a foreign tag
#pragma unroll
    for (int k = 0; k < kSlots; ++k) w.list[(size_t)k * NC + t] = 0ull;
  }
  for (long long k = g0; k < (long long)NC * halo; k += stride) w.halo[k] = kInf;
  for (long long g = g0; g < a.n_grids; g += stride) w.gupd[g] = 0ull;
}

// Per grid (blockIdx.y): the sum of the edge costs (|m_x|_M + |m_y|_M) / 2
// (the time scale of the queue keys), and the first round's queue, key 0:
// every tile (warm) or every tile that holds a source or one of its
// neighbours (cold: a source never changes, so the tiles across a tile edge
// next to it must see it in their halo on their own first visit).
constexpr int kSeedThreads = 256;

__global__ void __launch_bounds__(kSeedThreads) tile_seed_kernel(TileArgs a) {
  const TileWork &w = a.w;
  const int NC = a.ntiles_cap;
  TGrid *gp = w.grids + blockIdx.y;
  const TGrid g = *gp;
  const long long n = (long long)g.ny * g.nx;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float part = 0.0f;
  int any_src = 0;
  for (long long q = g0; q < n; q += stride) {
    const long long p = g.node_off + q;
    const float l11 = a.f[p], l21 = a.f[a.plane + p], l22 = a.f[2 * a.plane + p];
    const float m11 = fmaf(l11, l11, a.eps), m22 = fmaf(l21, l21, fmaf(l22, l22, a.eps));
    part += 0.5f * g.h * (sqrtf(m11) + sqrtf(m22));
    if (!a.src[p]) continue;
    any_src = 1;
    if (a.warm) continue;
    const int i = (int)(q / g.nx), j = (int)(q - (long long)i * g.nx);
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj) {
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || ii >= g.ny || jj < 0 || jj >= g.nx) continue;
        const int t = g.tile_off + (ii / a.ts) * g.tnx + jj / a.ts;
        atomicMin(&w.key[(size_t)(1 % kKeySlots) * NC + t], 0u);
        enqueue(w, NC, t, 1);
      }
  }
  if (a.warm) {
    const int nt = g.tny * g.tnx;
    for (long long k = g0; k < nt; k += stride) {
      const int t = g.tile_off + (int)k;
      w.key[(size_t)(1 % kKeySlots) * NC + t] = 0u;
      w.list[(size_t)(1 % kSlots) * NC + t] = (1ull << 32) | (unsigned)t;
    }
  }
  // the block's sum in a fixed order (warps, then the block's warps), then
  // one integer atomic per block: the grid's sum, and the keys it scales,
  // do not depend on the order in which blocks finish (a float atomic per
  // warp also serialised 131 k atomics on one word at 2048^2)
  __shared__ float wpart[kSeedThreads / 32];
  __shared__ int wany[kSeedThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    part += __shfl_xor_sync(0xffffffffu, part, o);
    any_src |= __shfl_xor_sync(0xffffffffu, any_src, o);
  }
  if ((threadIdx.x & 31) == 0) {
    wpart[threadIdx.x >> 5] = part;
    wany[threadIdx.x >> 5] = any_src;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float bsum = 0.0f;
    int bany = 0;
    for (int k = 0; k < kSeedThreads / 32; ++k) {
      bsum += wpart[k];
      bany |= wany[k];
    }
    atomicAdd(&gp->esum_fx, (unsigned long long)((double)bsum * 4294967296.0 + 0.5));
    if (bany) atomicOr(&gp->has_src, 1);
  }
}

// Keys of each grid in tile crossings; round 1's queue minimum; sources.
__global__ void tile_finish_seed_kernel(TileArgs a) {
  const TileWork &w = a.w;
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < a.n_grids; gi += gridDim.x * blockDim.x) {
    TGrid &g = w.grids[gi];
    const float esum = (float)((double)g.esum_fx * (1.0 / 4294967296.0));
    const float ebar = esum / (float)((long long)g.ny * g.nx);
    g.inv_scale = (ebar > 0.0f && ebar < kInf) ? 1.0f / ((float)a.ts * ebar) : 1.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    TileSlot *slots = reinterpret_cast<TileSlot *>(w.ctrl);
    if (a.warm) slots[1 % kSlots].count = w.ctrl[kCtrlNT];
    slots[1 % kSlots].kmin = 0u;
    // round 0 is complete: round 1's list is final (an empty one certifies)
    const unsigned n1 = slots[1 % kSlots].count ? slots[1 % kSlots].count : w.ctrl[kCtrlNT];
    slots[1 % kSlots].done = kPrevDone - n1;
  }
}

// Statistics: node updates of the solve, their sweep equivalent, and per
// grid (batch) status / sweep equivalent.
__global__ void tile_stats_kernel(TileArgs a, DevState *st, int *grid_status, int converged_only_global) {
  const TileWork &w = a.w;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long u = w.counters[0];
    st->cell_updates = u;
    st->sweeps = (int)((u + (unsigned long long)a.plane - 1ull) / (unsigned long long)a.plane);
  }
  if (!grid_status) return;
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < a.n_grids; gi += gridDim.x * blockDim.x) {
    const TGrid g = w.grids[gi];
    const unsigned long long n = (unsigned long long)g.ny * (unsigned long long)g.nx;
    const int code = !g.has_src ? RF_ERR_NO_SOURCE : (st->converged ? RF_OK : RF_ERR_NOT_CONVERGED);
    grid_status[3 * gi] = code;
    grid_status[3 * gi + 1] = n ? (int)((w.gupd[gi] + n - 1ull) / n) : 0;
    if (code != RF_OK) set_error(st, code);
  }
  (void)converged_only_global;
}

}  // namespace rf

namespace rf {

int tile_side(int requested) { return requested >= 32 ? 32 : 16; }

int tiles_cap(int n_grids, long long total_nodes, int max_line, int ts) {
  // ceil(a/t) ceil(b/t) <= ab/t^2 + (a + b)/t + 1 per grid; with floors and
  // a, b <= max_line the sum is below total/t^2 + 1 + grids (2 max_line/t + 2)
  const long long cap =
      total_nodes / ((long long)ts * ts) + 1 + (long long)n_grids * (2LL * max_line / ts + 2);
  return (int)std::min(cap, (long long)1 << 30);
}

size_t tile_work_bytes(int n_grids, int ntiles_cap, int ts) {
  const size_t NC = (size_t)ntiles_cap;
  // counters, ctrl, grids, per-grid updates, list[8] (8-byte entries), then
  // tstate, visits, key[4], tile -> grid, halo
  return 64 + kCtrlBytes + (size_t)n_grids * sizeof(TGrid) + (size_t)n_grids * 8 + NC * 8 * kSlots + NC * 4 * 2 +
         NC * 4 * kKeySlots + NC * 4 + NC * (size_t)(4 * ts + 4) * 4;
}

TileWork tile_work_carve(void *base, int n_grids, int ntiles_cap, int ts) {
  const size_t NC = (size_t)ntiles_cap;
  unsigned char *b = (unsigned char *)base;
  TileWork w;
  w.counters = (unsigned long long *)b;  // 8-byte aligned first
  b += 64;
  w.ctrl = (unsigned *)b;  // the slots' 64-bit words stay 8-byte aligned
  b += kCtrlBytes;
  w.grids = (TGrid *)b;  // 8-byte aligned
  b += (size_t)n_grids * sizeof(TGrid);
  w.gupd = (unsigned long long *)b;
  b += (size_t)n_grids * 8;
  w.list = (unsigned long long *)b;
  b += NC * 8 * kSlots;
  w.tstate = (unsigned *)b;
  b += NC * 4;
  w.visits = (unsigned *)b;
  b += NC * 4;
  w.key = (unsigned *)b;
  b += NC * 4 * kKeySlots;
  w.tile_grid = (int *)b;
  b += NC * 4;
  w.halo = (float *)b;
  (void)ts;
  return w;
}

template <int TS, bool SOFT>
static rf_status launch_solve(TileArgs &a, int num_sms, cudaStream_t s) {
  const size_t smem = sizeof(GroupSmem<TS>) * TileGeom<TS>::GROUPS;
  if (cudaFuncSetAttribute(tile_solve_kernel<TS, SOFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_solve_kernel<TS, SOFT>, TileGeom<TS>::CTA, smem) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  if (per_sm < 1) return RF_ERR_UNSUPPORTED;
  void *args[] = {&a};
  return cuda_status(cudaLaunchCooperativeKernel((const void *)tile_solve_kernel<TS, SOFT>, dim3(per_sm * num_sms),
                                                 dim3(TileGeom<TS>::CTA), args, smem, s));
}

rf_status tiles_launch(const TileLaunch &L, const TileWork &w, const LaunchCtl &ctl, cudaStream_t s) {
  const int ts = L.ts;
  TileArgs a;
  a.n_grids = L.n_grids;
  a.ts = ts;
  a.ntiles_cap = L.ntiles_cap;
  a.plane = L.total_nodes;
  a.eps = L.eps;
  a.f = L.proj5;
  a.src = L.src;
  a.T[0] = L.T;
  a.T[1] = L.Tb;
  a.tol = L.tol;
  a.rtol = L.rtol;
  a.window = L.window > 0.0f ? L.window : (ts == 32 ? 2.0f : 4.0f);
  a.warm = L.warm;
  a.tau = L.tau;
  // a sweep moves information across the grid, a round across one tile
  a.max_rounds = L.max_sweeps * std::max(1, (L.max_line + ts - 1) / ts);
  a.max_local = 16 * ts;
  a.w = w;
  a.ctl = ctl;
  if (cudaMemsetAsync(w.counters, 0, 64 + kCtrlBytes, s) != cudaSuccess) return RF_ERR_CUDA;
  if (L.descs) {
    tile_plan_batch_kernel<<<1, 1024, 0, s>>>(w, L.descs, L.n_grids, ts, L.total_nodes, L.max_line, L.ntiles_cap,
                                              ctl.st);
    tile_map_kernel<<<dim3(std::max(1, std::min(64, L.ntiles_cap / 256 + 1)), L.n_grids), 256, 0, s>>>(w);
  } else {
    tile_plan_single_kernel<<<1, 32, 0, s>>>(w, L.ny, L.nx, L.h, ts);
  }
  const long long per_grid = std::max<long long>(1, L.total_nodes / L.n_grids);
  const int reset_blocks = blocks_for((long long)L.ntiles_cap * (4 * ts + 4), 256, L.num_sms * 8);
  tile_reset_kernel<<<reset_blocks, 256, 0, s>>>(a);
  const int gx = std::max(1, std::min(blocks_for(per_grid, 256, L.num_sms * 8), 65535));
  tile_seed_kernel<<<dim3(gx, L.n_grids), kSeedThreads, 0, s>>>(a);
  tile_finish_seed_kernel<<<blocks_for(L.n_grids, 256, 64), 256, 0, s>>>(a);
  const bool soft = L.tau > 0.0f;
  const rf_status rs = ts == 32 ? (soft ? launch_solve<32, true>(a, L.num_sms, s) : launch_solve<32, false>(a, L.num_sms, s))
                                : (soft ? launch_solve<16, true>(a, L.num_sms, s) : launch_solve<16, false>(a, L.num_sms, s));
  if (rs != RF_OK) return rs;
  tile_stats_kernel<<<blocks_for(L.n_grids, 256, 64), 256, 0, s>>>(a, ctl.st, L.grid_status, 0);
  return cuda_status(cudaGetLastError());
}

}  // namespace rf
