// rf_sweep.cu -- a2-a5: forward fast sweep, on-device convergence, stencil
// record and residual.
//
// Paper: Sec. 3.2 and App. A (Alg. 1).  One iteration is four directional
// sweeps (columns +x, rows +y, columns -x, rows -y).  Within a sweep every
// line (column or row) is one parallel front: node (s, l) of line step s is
// updated from step s-1 (already updated in this sweep) and from steps s,
// s+1 as they were before the sweep -- the column/row-parallel schedule of
// Sec. 3.2.  The update is the replacement T <- min valid candidate
// (equivalently Alg. 1's min-update whenever the candidate set is monotone),
// so the sweep stops at a fixed point of T = min valid candidate(T).
//
// GB300 mapping.  One persistent cooperative launch runs every sweep of the
// solve.  A sweep's lines are split into bands of R lines, one CTA per band.
// A CTA advances its band K line steps at a time ("block"), recomputing a
// halo of K lines on each side from the values its neighbours published at
// the end of their previous block, so inner lines follow the exact
// line-parallel recurrence and neighbouring CTAs synchronise once per K
// steps instead of once per step.  T ping-pongs between two buffers so the
// "before the sweep" values are never overwritten mid-sweep.  A tile of
// (K+2) x (R+2K+2) times plus the K x (R+2K) metric fields of the block is
// staged in shared memory with coalesced loads (steps are contiguous in
// memory for column sweeps, lines for row sweeps).  Convergence: a CTA ORs
// "some inner node changed" into a per-sweep word; after a bounded grid
// barrier every CTA reads it and stops at the first sweep that changed
// nothing.  Every wait is bounded by the context's timeout.
#include <algorithm>
#include <mutex>

#include "rf_cone.cuh"
#include "rf_ctx.h"
#include "rf_sweep_common.cuh"
#include "rf_sweep_stream.h"
#include "rf_sweep_tiles.h"

namespace rf {

struct SweepArgs {
  int ny, nx;
  float h, eps;
  const float *f;  // 5 planes (projected)
  const uint8_t *src;
  float *Ta;  // caller's T (initial state, final result)
  float *Tb;  // workspace
  int R, K;
  int max_sweeps;
  float tol, rtol;
  unsigned tok_stride;  // progress tokens per sweep
  unsigned *progress;   // [gridDim.x]
  int *changed;         // [max_sweeps]
  LaunchCtl ctl;
};

// Lanes per node in the line-step loop (template parameter NL):
//  NL = 4: lane q of a node evaluates the two-point candidates of stencils
//          2q, 2q+1 and the one-point candidates of neighbours 2q, 2q+1; a
//          two-level shuffle takes the minimum.  Node tables are kTabSize
//          planes of K x EP floats plus K x EP source bytes.
//  NL = 1: one thread evaluates all 16 candidates of its node (no shuffles,
//          each table value and donor time loaded once).  Node tables are
//          K x EP records of kRec floats (the 11 table values and the source
//          flag), read as three float4; the 48-byte record stride puts the
//          8 threads of a quarter-warp on distinct banks.  Only the first
//          ext threads step; the others stage and publish.
// Both use 4 * ext threads, so staging and publishing cost the same.
constexpr int kLanes = 4;
constexpr int kRec = 12;
constexpr int kMaxExt = 128;    // R + 2K <= 128  ->  <= 512 threads
constexpr int kMaxExt1 = 96;    // NL = 1: <= 384 threads (168 registers)
constexpr int kMaxTabPer = 8;   // node tables staged per thread per block (K/4)
constexpr int kMaxOldPer = 12;  // old-T values staged per thread per block

template <int NL>
__host__ __device__ inline size_t sweep_smem_bytes(int R, int K) {
  const int ext = R + 2 * K, W = ext + 2, P = W | 1, EP = ext | 1;
  const size_t tfl = (size_t)(K + 2) * P + (size_t)(K + 1) * P;
  if (NL == 1) return ((size_t)kRec * K * EP + tfl) * sizeof(float);
  return (tfl + (size_t)kTabSize * K * EP) * sizeof(float) + (size_t)K * EP;
}

__host__ __device__ inline int sweep_threads(int R, int K) { return kLanes * (R + 2 * K); }

// Shapes the kernel accepts: K a power of two <= 32, R >= K, R + 2K <= 128
// (96 for NL = 1), and the staged values per thread within the register
// budget.
__host__ inline bool sweep_shape_ok(int R, int K, int NL) {
  if (K < 4 || K > 32 || (K & (K - 1)) || R < K || R + 2 * K > (NL == 1 ? kMaxExt1 : kMaxExt)) return false;
  const int nth = sweep_threads(R, K), W = R + 2 * K + 2;
  return (K * (R + 2 * K) + nth - 1) / nth <= kMaxTabPer && ((K + 2) * W + nth - 1) / nth <= kMaxOldPer;
}

// K line steps of one block, one thread per node (NL = 1).  Thread e owns
// tile line e; at step t it needs the donors of step t-1 of this sweep
// (nw row t) and of steps t, t+1 before the sweep (old rows t+1, t+2).
// Returns whether an inner node changed.
template <int DIR>
__device__ __forceinline__ int steps_one_lane(const float *__restrict__ tb, const float *__restrict__ old, float *nw,
                                              int P, int EP, int K, int R, int ext, int t_end, int l0, int L,
                                              float tol, float rtol) {
  const int e = threadIdx.x, tl = e + 1, l = l0 - K + e;
  const bool valid = (e < ext) && (l >= 0) && (l < L);
  const bool inband = (e >= K) && (e < K + R);
  int changed = 0;
  for (int t = 0; t < t_end; ++t) {
    // only nodes e in [t+1, ext-1-t) can still influence the inner lines
    if (e < ext && e > t && e < ext - 1 - t) {
      float Tn[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const int ds = tile_ds<DIR>(n), dl = tile_dl<DIR>(n);
        Tn[n] = (ds < 0) ? nw[t * P + tl + dl] : old[(t + 1 + ds) * P + tl + dl];
      }
      const float4 *rp = reinterpret_cast<const float4 *>(tb + (size_t)(t * EP + e) * kRec);
      const float4 r0 = rp[0], r1 = rp[1], r2 = rp[2];
      const float tab[kTabSize] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z};
      float cand = kInf;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float l1, l2;
        cand = fminf(cand, two_point(tab, k, Tn[k], Tn[(k + 1) & 7], l1, l2));
      }
#pragma unroll
      for (int n = 0; n < 8; ++n) cand = fminf(cand, one_point(tab, n, Tn[n]));
      float tnew = kInf;
      if (valid) {
        tnew = (r2.w != 0.0f) ? 0.0f : cand;
        if (inband) changed |= node_changed(tnew, old[(t + 1) * P + tl], tol, rtol);
      }
      nw[(t + 1) * P + tl] = tnew;
    }
    __syncthreads();
  }
  return changed;
}

template <int NL>
__global__ void __launch_bounds__(NL == 1 ? 384 : 512) sweep_kernel(SweepArgs a) {
  extern __shared__ float4 smem4[];
  float *smem = reinterpret_cast<float *>(smem4);
  const int R = a.R, K = a.K, ext = R + 2 * K, W = ext + 2, P = W | 1, EP = ext | 1;
  // NL = 1: records first (16-byte aligned), then old and nw
  float *tb = (NL == 1) ? smem : smem + (size_t)(2 * K + 3) * P;  // node tables
  float *old = (NL == 1) ? smem + (size_t)kRec * K * EP : smem;   // (K+2) x P  T before the sweep
  float *nw = old + (size_t)(K + 2) * P;                          // (K+1) x P  T of this sweep
  uint8_t *sm = (uint8_t *)(smem + (size_t)(2 * K + 3) * P + (size_t)kTabSize * K * EP);  // NL = 4: source flags
  const int TS = K * EP;                              // table plane stride
  __shared__ int s_ok;
  __shared__ int s_any;

  const int tid = threadIdx.x, nth = blockDim.x, b = blockIdx.x;
  const int cell = tid / kLanes, q = tid % kLanes;
  const int logK = __ffs(K) - 1;
  const long long plane = (long long)a.ny * a.nx;
  const int n_tab = K * ext, n_old = (K + 2) * W;

  // per-lane table offsets (fixed for the whole launch)
  const int n0 = 2 * q, n1 = 2 * q + 1, n2 = (2 * q + 2) & 7;
  const int offL0 = (TAB_LEN + len_class(n0)) * TS, offL1 = (TAB_LEN + len_class(n1)) * TS,
            offL2 = (TAB_LEN + len_class(n2)) * TS;
  const int offW0 = (TAB_WM + (n0 & 3)) * TS, offW1 = (TAB_WM + (n1 & 3)) * TS, offW2 = (TAB_WM + (n2 & 3)) * TS;
  const float sg0 = n0 < 4 ? 1.0f : -1.0f, sg1 = n1 < 4 ? 1.0f : -1.0f, sg2 = n2 < 4 ? 1.0f : -1.0f;
  const bool xs = (q & 1) != 0;  // stencils 2q, 2q+1 differ along x for q = 1, 3
  const int offLx = (TAB_LEN + (xs ? 0 : 1)) * TS, offInv = (xs ? TAB_IAX : TAB_IAY) * TS, offDet = TAB_DET * TS;

  float *cur = a.Ta, *nxt = a.Tb;
  int sweep = 0;
  int converged = 0;
  bool abort = false;

  while (true) {
    const int dir = sweep & 3;
    const bool col = (dir & 1) == 0;
    const int S = col ? a.nx : a.ny;
    const int L = col ? a.ny : a.nx;
    const int nb = (L + R - 1) / R;
    const int nblk = (S + K - 1) / K;
    const unsigned base = (unsigned)sweep * a.tok_stride;
    int local_changed = 0;
    // tile offsets of this lane's three neighbours 2q, 2q+1, 2q+2
    int nds[3], ndl[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) nb_tile_offset(dir, (2 * q + u) & 7, nds[u], ndl[u]);
    // staging lists of this thread (tile coordinates packed as lo | hi << 8):
    // consecutive threads take consecutive memory (steps for column sweeps,
    // lines for row sweeps)
    int tabidx[kMaxTabPer], oldidx[kMaxOldPer];
#pragma unroll
    for (int j = 0; j < kMaxTabPer; ++j) {
      const int f = tid + j * nth;
      int t = 0, e = 0;
      if (col) { e = f >> logK; t = f & (K - 1); }
      else     { t = f / ext;   e = f - t * ext; }
      tabidx[j] = (f < n_tab) ? (t | (e << 8)) : -1;
    }
#pragma unroll
    for (int j = 0; j < kMaxOldPer; ++j) {
      const int f = tid + j * nth;
      int ts = 0, tl = 0;
      if (col) { tl = f / (K + 2); ts = f - tl * (K + 2); }
      else     { ts = f / W;       tl = f - ts * W; }
      oldidx[j] = (f < n_old) ? (ts | (tl << 8)) : -1;
    }

    if (b < nb && !abort) {
      const int l0 = b * R;
      const int line0 = l0 - K - 1;  // global line of tile column 0
      float rv[kMaxTabPer][5];
      uint8_t sv[kMaxTabPer];
      float ov[kMaxOldPer];
      // issue the (neighbour-independent) loads of the block starting at s0
      auto prefetch = [&](int s0) {
#pragma unroll
        for (int j = 0; j < kMaxTabPer; ++j) {
          const int t = tabidx[j] & 255, e = tabidx[j] >> 8;
          const int s = s0 + t, l = l0 - K + e;
          const bool ok = tabidx[j] >= 0 && s < S && l >= 0 && l < L;
          const long long g = ok ? gidx(dir, s, l, a.ny, a.nx) : 0;
#pragma unroll
          for (int c = 0; c < 5; ++c) rv[j][c] = ok ? __ldg(a.f + c * plane + g) : 1.0f;
          sv[j] = ok ? a.src[g] : (uint8_t)0;
        }
#pragma unroll
        for (int j = 0; j < kMaxOldPer; ++j) {
          const int ts = oldidx[j] & 255, tl = oldidx[j] >> 8;
          const int s = s0 - 1 + ts, l = line0 + tl;
          const bool ok = oldidx[j] >= 0 && s >= 0 && s < S && l >= 0 && l < L;
          ov[j] = ok ? __ldcg(cur + gidx(dir, s, l, a.ny, a.nx)) : kInf;
        }
      };
      prefetch(0);
      for (int kb = 0; kb < nblk; ++kb) {
        const int s0 = kb * K;
        // 1. node tables, source flags and T-before-sweep of this block
#pragma unroll
        for (int j = 0; j < kMaxTabPer; ++j) {
          if (tabidx[j] < 0) continue;
          const int t = tabidx[j] & 255, e = tabidx[j] >> 8;
          float tab[kTabSize];
          node_tab(rv[j][0], rv[j][1], rv[j][2], rv[j][3], rv[j][4], a.h, a.eps, tab);
          if (NL == 1) {
            float4 *d = reinterpret_cast<float4 *>(tb + (size_t)(t * EP + e) * kRec);
            d[0] = make_float4(tab[0], tab[1], tab[2], tab[3]);
            d[1] = make_float4(tab[4], tab[5], tab[6], tab[7]);
            d[2] = make_float4(tab[8], tab[9], tab[10], sv[j] ? 1.0f : 0.0f);
          } else {
#pragma unroll
            for (int c = 0; c < kTabSize; ++c) tb[c * TS + t * EP + e] = tab[c];
            sm[t * EP + e] = sv[j];
          }
        }
#pragma unroll
        for (int j = 0; j < kMaxOldPer; ++j) {
          if (oldidx[j] < 0) continue;
          old[(oldidx[j] & 255) * P + (oldidx[j] >> 8)] = ov[j];
        }
        // 2. neighbours must have published block kb-1 of this sweep
        if (tid == 0) {
          int ok = 1;
          if (kb > 0) {
            if (b > 0) ok &= wait_geq(&a.progress[b - 1], base + kb, a.ctl);
            if (ok && b + 1 < nb) ok &= wait_geq(&a.progress[b + 1], base + kb, a.ctl);
          }
          s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) {
          abort = true;
          break;
        }
        // 3. this sweep's step s0-1 as published by the neighbours (halo
        // lines) and by this CTA (inner lines); edge columns keep old values
        for (int tl = tid; tl < W; tl += nth) {
          const int s = s0 - 1, l = line0 + tl;
          float v = kInf;
          if (s >= 0 && l >= 0 && l < L) {
            const bool halo_ok = (tl >= 1 && tl <= ext);
            v = halo_ok ? __ldcg(nxt + gidx(dir, s, l, a.ny, a.nx)) : __ldcg(cur + gidx(dir, s, l, a.ny, a.nx));
          }
          nw[tl] = v;
        }
        for (int t = tid; t < K; t += nth) {
          nw[(t + 1) * P] = old[(t + 1) * P];
          nw[(t + 1) * P + W - 1] = old[(t + 1) * P + W - 1];
        }
        __syncthreads();
        // 4. K line steps, one parallel front each.  At step t only nodes
        // e in [t+1, ext-1-t) can still influence the inner lines.
        if (NL == 1) {
          const int t_end = min(K, S - s0);
          switch (dir) {
            case 0: local_changed |= steps_one_lane<0>(tb, old, nw, P, EP, K, R, ext, t_end, l0, L, a.tol, a.rtol); break;
            case 1: local_changed |= steps_one_lane<1>(tb, old, nw, P, EP, K, R, ext, t_end, l0, L, a.tol, a.rtol); break;
            case 2: local_changed |= steps_one_lane<2>(tb, old, nw, P, EP, K, R, ext, t_end, l0, L, a.tol, a.rtol); break;
            default: local_changed |= steps_one_lane<3>(tb, old, nw, P, EP, K, R, ext, t_end, l0, L, a.tol, a.rtol); break;
          }
        } else {
          for (int t = 0; t < K; ++t) {
            const int s = s0 + t;
            if (s >= S) break;
            const int e = cell, tl = e + 1, l = l0 - K + e;
            const bool need = (e > t) && (e < ext - 1 - t);
            if (__any_sync(0xffffffffu, need)) {
              const bool live = need && (l >= 0) && (l < L);
              float cand = kInf;
              if (live) {
                float Tq[3];
#pragma unroll
                for (int u = 0; u < 3; ++u)
                  Tq[u] = (nds[u] < 0) ? nw[t * P + tl + ndl[u]] : old[(t + 1 + nds[u]) * P + tl + ndl[u]];
                const float *tc = tb + t * EP + e;
                const float len0 = tc[offL0], len1 = tc[offL1], len2 = tc[offL2];
                const float w0 = sg0 * tc[offW0], w1 = sg1 * tc[offW1], w2 = sg2 * tc[offW2];
                const float lx = tc[offLx], aa = lx * lx, inv = tc[offInv], det = tc[offDet];
                float l1, l2;
                cand = two_point_core(len0, len1, w0, w1, aa, inv, det, Tq[0], Tq[1], l1, l2);
                cand = fminf(cand, two_point_core(len1, len2, w1, w2, aa, inv, det, Tq[1], Tq[2], l1, l2));
                cand = fminf(cand, one_point_core(len0, w0, Tq[0]));
                cand = fminf(cand, one_point_core(len1, w1, Tq[1]));
              }
              cand = fminf(cand, __shfl_xor_sync(0xffffffffu, cand, 1));
              cand = fminf(cand, __shfl_xor_sync(0xffffffffu, cand, 2));
              if (q == 0 && need) {
                float tnew = kInf;
                if (live) {
                  const float told = old[(t + 1) * P + tl];
                  tnew = sm[t * EP + e] ? 0.0f : cand;
                  if (e >= K && e < K + R) {
                    local_changed |= node_changed(tnew, told, a.tol, a.rtol);
                  }
                }
                nw[(t + 1) * P + tl] = tnew;
              }
            }
            __syncthreads();
          }
        }
        // 5. publish the inner lines, prefetch the next block, then release
        const int nwarps = nth >> 5, warp = tid >> 5, lane = tid & 31;
        if (col) {
          for (int e = warp; e < R; e += nwarps) {
            const int l = l0 + e;
            for (int t = lane; t < K; t += 32) {
              const int s = s0 + t;
              if (s < S && l < L) nxt[gidx(dir, s, l, a.ny, a.nx)] = nw[(t + 1) * P + K + 1 + e];
            }
          }
        } else {
          for (int t = warp; t < K; t += nwarps) {
            const int s = s0 + t;
            for (int e = lane; e < R; e += 32) {
              const int l = l0 + e;
              if (s < S && l < L) nxt[gidx(dir, s, l, a.ny, a.nx)] = nw[(t + 1) * P + K + 1 + e];
            }
          }
        }
        if (kb + 1 < nblk) prefetch(s0 + K);
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          st_release_u32(&a.progress[b], base + kb + 1);
        }
      }
    }
    // end of sweep: combine the changed flags, then a bounded grid barrier
    local_changed = __syncthreads_or(local_changed);
    if (tid == 0 && local_changed) atomicOr(&a.changed[sweep], 1);
    if (!grid_sync(a.ctl)) abort = true;
    if (tid == 0) s_any = ld_acquire_s32(&a.changed[sweep]);
    __syncthreads();
    const int any = s_any;
    ++sweep;
    float *tmp = cur;
    cur = nxt;
    nxt = tmp;
    if (abort) break;
    if (!any) {
      converged = 1;
      break;
    }
    if (sweep >= a.max_sweeps) break;
  }
  // the latest values are in `cur`; hand them back in the caller's buffer
  if (cur != a.Ta) {
    for (long long p = (long long)blockIdx.x * nth + tid; p < plane; p += (long long)gridDim.x * nth)
      a.Ta[p] = __ldcg(cur + p);
  }
  if (b == 0 && tid == 0) {
    a.ctl.st->sweeps = sweep;
    a.ctl.st->converged = converged;
    a.ctl.st->cell_updates = (unsigned long long)sweep * (unsigned long long)plane;
    if (!converged && !abort) set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
  }
}

// Initial state: T = 0 on sources; +inf elsewhere (cold) or the guess
// (warm).  Also flags an empty source mask.
__global__ void init_kernel(float *T, const uint8_t *src, long long n, int warm,
                            DevState *st, int *has_src) {
  int any = 0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const bool s = src[p] != 0;
    any |= s;
    if (s) T[p] = 0.0f;
    else if (!warm) T[p] = kInf;
  }
  if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(has_src, 1);
}

__global__ void check_source_kernel(const int *has_src, DevState *st) {
  if (threadIdx.x == 0 && *has_src == 0) set_error(st, RF_ERR_NO_SOURCE);
}

void init_state(float *T, const uint8_t *src, long long n, int warm, DevState *st, int *has_src, int num_sms,
                cudaStream_t s) {
  init_kernel<<<blocks_for(n, 256, num_sms * 8), 256, 0, s>>>(T, src, n, warm, st, has_src);
}

void check_source_flag(const int *has_src, DevState *st, cudaStream_t s) {
  check_source_kernel<<<1, 32, 0, s>>>(has_src, st);
}

struct RecordArgs {
  int ny, nx;
  float h, eps;
  const float *f;
  const uint8_t *src;
  const float *T;
  uint8_t *id;
  float *w1;
  float *dT;
  float *res;  // nullable: per-node residual
  float *max_abs;  // nullable: device float
  DevState *st;
};

// a5: stencil identification + closed-form partials at the converged T
// (record_node_cone: the cone form of the tile-queue and streamed solves,
// one pass over the candidates), with the max |residual| reduced per block.
template <bool RECORD>
__global__ void __launch_bounds__(256) record_kernel(RecordArgs a) {
  const long long n = (long long)a.ny * a.nx;
  float local_max = 0.0f;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p / a.nx), j = (int)(p - (long long)i * a.nx);
    uint8_t id;
    float w1, d[5], r;
    record_node_cone(a.f, n, p, i, j, a.ny, a.nx, a.h, a.eps, a.src[p] != 0, a.T, RECORD, id, w1, d, r);
    if (RECORD) {
      a.id[p] = id;
      a.w1[p] = w1;
#pragma unroll
      for (int c = 0; c < 5; ++c) a.dT[c * n + p] = d[c];
    }
    if (a.res) a.res[p] = r;
    local_max = fmaxf(local_max, fabsf(r));
  }
  // block max -> one atomic per block (non-negative floats order as uints)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
  __shared__ float wmax[8];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = local_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
    atomicMax(&a.st->max_res_bits, __float_as_uint(m));
    if (a.max_abs) atomicMax((unsigned *)a.max_abs, __float_as_uint(m));
  }
}

}  // namespace rf

using namespace rf;

namespace {

struct SweepPlan {
  int R, K, NL, grid, threads;
  size_t smem;
  const void *kernel;
};

template <int NL>
rf_status plan_kernel(rf_ctx *ctx, int R, int K, int maxL, SweepPlan *pl) {
  if (!sweep_shape_ok(R, K, NL)) return RF_ERR_UNSUPPORTED;
  int dev_max_smem = 0;
  cudaDeviceGetAttribute(&dev_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  const int threads = sweep_threads(R, K);
  const size_t smem = sweep_smem_bytes<NL>(R, K);
  if ((long long)smem > dev_max_smem) return RF_ERR_UNSUPPORTED;
  cudaFuncSetAttribute(sweep_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<NL>, threads, smem) != cudaSuccess)
    return RF_ERR_CUDA;
  const int grid = (maxL + R - 1) / R;
  if (per_sm < 1 || grid > per_sm * ctx->num_sms) return RF_ERR_UNSUPPORTED;
  pl->R = R;
  pl->K = K;
  pl->NL = NL;
  pl->grid = grid;
  pl->threads = threads;
  pl->smem = smem;
  pl->kernel = (const void *)sweep_kernel<NL>;
  return RF_OK;
}

// Tiled variants (node tables built per block); lanes = 1 or 4.
rf_status plan_sweep(rf_ctx *ctx, int ny, int nx, const rf_opts *o, int lanes, SweepPlan *pl) {
  int K = (o && o->block > 0) ? o->block : 32;
  int R = (o && o->band > 0) ? o->band : 32;
  const int max_ext = lanes == 1 ? kMaxExt1 : kMaxExt;
  // round the requested shape to one the kernel accepts
  int k2 = 4;
  while (k2 * 2 <= K && k2 < 32) k2 *= 2;
  K = k2;
  if (R < K) R = K;
  while (R + 2 * K > max_ext && K > 4) K /= 2;
  if (R + 2 * K > max_ext) R = max_ext - 2 * K;
  const int maxL = std::max(ny, nx);
  return lanes == 1 ? plan_kernel<1>(ctx, R, K, maxL, pl) : plan_kernel<4>(ctx, R, K, maxL, pl);
}

bool variant_ok(int v) {
  return v == RF_SWEEP_AUTO || v == RF_SWEEP_TILED1 || v == RF_SWEEP_STREAMED || v == RF_SWEEP_TILED4 ||
         v == RF_SWEEP_TILES;
}

}  // namespace

extern "C" rf_status rf_sweep_forward(rf_ctx *ctx, const rf_grid *grid, const float *proj5,
                                      float eps, const uint8_t *src, const rf_opts *opts,
                                      float *T, rf_record *rec, void *stream) {
  if (!ctx || !grid_ok(grid) || !proj5 || !src || !T) return RF_ERR_INVALID_ARG;
  if (!(eps >= 0.0f)) return RF_ERR_INVALID_ARG;
  if (rec && (!rec->id || !rec->w1 || !rec->dT)) return RF_ERR_INVALID_ARG;
  rf_opts o = {0.0f, 64, RF_MODE_COLD, 0, 0, 1e-6f, 0, 0.0f};
  if (opts) o = *opts;
  if (o.max_sweeps < 1 || !(o.tol >= 0.0f) || !(o.rtol >= 0.0f) || (o.mode != RF_MODE_COLD && o.mode != RF_MODE_WARM) ||
      !(o.window >= 0.0f))
    return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ny = grid->ny, nx = grid->nx;
  const long long n = (long long)ny * nx;

  if (!variant_ok(o.variant)) return RF_ERR_INVALID_ARG;

  // tile queue: the default when its workspace can be allocated
  if (o.variant == RF_SWEEP_TILES || o.variant == RF_SWEEP_AUTO) {
    const int ts = rf::tile_side(o.variant == RF_SWEEP_TILES ? o.band : 0);
    const int ncap = rf::tiles_cap(1, n, std::max(ny, nx), ts);
    rf_status rt = ensure(&ctx->tilebuf, &ctx->tilebuf_cap, rf::tile_work_bytes(1, ncap, ts));
    if (rt == RF_OK) rt = ensure(&ctx->tbuf, &ctx->tbuf_cap, (size_t)n);
    if (rt == RF_OK) rt = ensure(&ctx->changed, &ctx->changed_cap, (size_t)o.max_sweeps + 2);
    if (rt != RF_OK && o.variant == RF_SWEEP_TILES) return rt;
    if (rt == RF_OK) {
      cudaMemsetAsync(ctx->changed, 0, sizeof(int) * (o.max_sweeps + 2), s);
      cudaMemsetAsync(&ctx->state->sweeps, 0, sizeof(int) * 2, s);
      cudaMemsetAsync(&ctx->state->bar, 0, sizeof(unsigned long long) + 2 * sizeof(unsigned), s);
      cudaMemsetAsync(&ctx->state->cell_updates, 0, sizeof(unsigned long long), s);
      int *has_src = ctx->changed + o.max_sweeps;
      init_kernel<<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(T, src, n, o.mode == RF_MODE_WARM,
                                                                         ctx->state, has_src);
      check_source_kernel<<<1, 32, 0, s>>>(has_src, ctx->state);
      LaunchCtl ctl;
      ctl.st = ctx->state;
      ctl.abort = ctx->changed + o.max_sweeps + 1;
      ctl.timeout_ns = ctx->timeout_ns;
      const rf::TileWork w = rf::tile_work_carve(ctx->tilebuf, 1, ncap, ts);
      rf::TileLaunch L;
      L.num_sms = ctx->num_sms;
      L.ts = ts;
      L.n_grids = 1;
      L.descs = nullptr;
      L.ny = ny;
      L.nx = nx;
      L.h = grid->h;
      L.max_line = std::max(ny, nx);
      L.total_nodes = n;
      L.ntiles_cap = ncap;
      L.eps = eps;
      L.proj5 = proj5;
      L.src = src;
      L.T = T;
      L.Tb = ctx->tbuf;
      L.warm = o.mode == RF_MODE_WARM;
      L.max_sweeps = o.max_sweeps;
      L.tol = o.tol;
      L.rtol = o.rtol;
      L.window = o.window;
      L.tau = 0.0f;
      L.grid_status = nullptr;
      rt = rf::tiles_launch(L, w, ctl, s);
      if (rt != RF_OK) return rt;
      if (rec) {
        RecordArgs r;
        r.ny = ny;
        r.nx = nx;
        r.h = grid->h;
        r.eps = eps;
        r.f = proj5;
        r.src = src;
        r.T = T;
        r.id = rec->id;
        r.w1 = rec->w1;
        r.dT = rec->dT;
        r.res = nullptr;
        r.max_abs = nullptr;
        r.st = ctx->state;
        cudaMemsetAsync(&ctx->state->max_res_bits, 0, sizeof(unsigned), s);
        record_kernel<true><<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(r);
      }
      return cuda_status(cudaGetLastError());
    }
  }

  // kernel variant: streamed when requested or automatic and it fits,
  // else tiled (one or four threads per node)
  rf::StreamPlan sp;
  SweepPlan pl;
  bool streamed = false;
  rf_status rs = RF_OK;
  if (o.variant == RF_SWEEP_STREAMED || o.variant == RF_SWEEP_AUTO) {
    rs = rf::stream_plan(ctx, ny, nx, o.band, o.block, &sp);
    if (rs == RF_OK) rs = ensure(&ctx->recbuf, &ctx->recbuf_cap, rf::stream_record_floats4(ny, nx));
    if (rs == RF_OK) streamed = true;
    else if (o.variant == RF_SWEEP_STREAMED) return rs;
  }
  if (!streamed) {
    rs = plan_sweep(ctx, ny, nx, &o, o.variant == RF_SWEEP_TILED4 ? 4 : 1, &pl);
    if (rs != RF_OK) return rs;
  }
  const int grid_ctas = streamed ? sp.grid : pl.grid;
  if ((rs = ensure(&ctx->tbuf, &ctx->tbuf_cap, (size_t)n)) != RF_OK) return rs;
  if ((rs = ensure(&ctx->progress, &ctx->progress_cap, (size_t)grid_ctas + 1)) != RF_OK) return rs;
  // changed flags: [0, max_sweeps) per sweep, then has-source, then abort
  if ((rs = ensure(&ctx->changed, &ctx->changed_cap, (size_t)o.max_sweeps + 2)) != RF_OK) return rs;

  // reset the counters this launch uses (status word excluded: it
  // accumulates until rf_ctx_last_stats reads it)
  cudaMemsetAsync(ctx->progress, 0, sizeof(unsigned) * (grid_ctas + 1), s);
  cudaMemsetAsync(ctx->changed, 0, sizeof(int) * (o.max_sweeps + 2), s);
  cudaMemsetAsync(&ctx->state->sweeps, 0, sizeof(int) * 2, s);
  cudaMemsetAsync(&ctx->state->bar, 0, sizeof(unsigned long long) + 2 * sizeof(unsigned), s);
  cudaMemsetAsync(&ctx->state->cell_updates, 0, sizeof(unsigned long long), s);

  int *has_src = ctx->changed + o.max_sweeps;  // last slot
  init_kernel<<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(T, src, n, o.mode == RF_MODE_WARM,
                                                                     ctx->state, has_src);
  check_source_kernel<<<1, 32, 0, s>>>(has_src, ctx->state);

  LaunchCtl ctl;
  ctl.st = ctx->state;
  ctl.abort = ctx->changed + o.max_sweeps + 1;
  ctl.timeout_ns = ctx->timeout_ns;
  if (streamed) {
    if ((rs = rf::stream_records(ny, nx, grid->h, eps, proj5, src, ctx->recbuf, s)) != RF_OK) return rs;
    if ((rs = rf::stream_launch(sp, ny, nx, ctx->recbuf, T, ctx->tbuf, o.max_sweeps, o.tol, o.rtol, ctx->progress,
                                ctx->changed, ctl, s)) != RF_OK)
      return rs;
  } else {
    SweepArgs a;
    a.ny = ny;
    a.nx = nx;
    a.h = grid->h;
    a.eps = eps;
    a.f = proj5;
    a.src = src;
    a.Ta = T;
    a.Tb = ctx->tbuf;
    a.R = pl.R;
    a.K = pl.K;
    a.max_sweeps = o.max_sweeps;
    a.tol = o.tol;
    a.rtol = o.rtol;
    a.tok_stride = (unsigned)((std::max(ny, nx) + pl.K - 1) / pl.K + 1);
    a.progress = ctx->progress;
    a.changed = ctx->changed;
    a.ctl = ctl;
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel(pl.kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, s);
    if (e != cudaSuccess) return RF_ERR_CUDA;
  }

  if (rec) {
    RecordArgs r;
    r.ny = ny;
    r.nx = nx;
    r.h = grid->h;
    r.eps = eps;
    r.f = proj5;
    r.src = src;
    r.T = T;
    r.id = rec->id;
    r.w1 = rec->w1;
    r.dT = rec->dT;
    r.res = nullptr;
    r.max_abs = nullptr;
    r.st = ctx->state;
    cudaMemsetAsync(&ctx->state->max_res_bits, 0, sizeof(unsigned), s);
    record_kernel<true><<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(r);
  }
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_record_stencils(rf_ctx *ctx, const rf_grid *grid, const float *proj5, float eps,
                                        const uint8_t *src, const float *T, rf_record *rec, void *stream) {
  if (!ctx || !grid_ok(grid) || !proj5 || !src || !T || !rec || !rec->id || !rec->w1 || !rec->dT)
    return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const long long n = (long long)grid->ny * grid->nx;
  RecordArgs r;
  r.ny = grid->ny;
  r.nx = grid->nx;
  r.h = grid->h;
  r.eps = eps;
  r.f = proj5;
  r.src = src;
  r.T = T;
  r.id = rec->id;
  r.w1 = rec->w1;
  r.dT = rec->dT;
  r.res = nullptr;
  r.max_abs = nullptr;
  r.st = ctx->state;
  cudaMemsetAsync(&ctx->state->max_res_bits, 0, sizeof(unsigned), s);
  record_kernel<true><<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(r);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_residual(rf_ctx *ctx, const rf_grid *grid, const float *proj5, float eps,
                                 const uint8_t *src, const float *T, float *res, float *max_abs,
                                 void *stream) {
  if (!ctx || !grid_ok(grid) || !proj5 || !src || !T) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const long long n = (long long)grid->ny * grid->nx;
  RecordArgs r;
  r.ny = grid->ny;
  r.nx = grid->nx;
  r.h = grid->h;
  r.eps = eps;
  r.f = proj5;
  r.src = src;
  r.T = T;
  r.id = nullptr;
  r.w1 = nullptr;
  r.dT = nullptr;
  r.res = res;
  r.max_abs = max_abs;
  r.st = ctx->state;
  if (max_abs) cudaMemsetAsync(max_abs, 0, sizeof(float), s);
  cudaMemsetAsync(&ctx->state->max_res_bits, 0, sizeof(unsigned), s);
  record_kernel<false><<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(r);
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// rf_sweep_forward_static: the forward solve without any allocation.
//
// Some callers cannot allocate device memory when they solve: a host
// framework that has already reserved the device's memory for its own
// caching allocator or enforces a memory budget, or a latency-critical loop
// that must not pay cudaMalloc's implicit device-wide synchronisation.  This
// entry point runs the same kernels as rf_sweep_forward, but its scratch --
// the second T buffer of the ping-pong sweeps, the per-band progress tokens,
// the per-sweep change flags and the device status word -- lives in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.  The caller still passes the
// inputs and the output T.
namespace {

constexpr long long kStaticMaxNodes = 1LL << 20;  // ny * nx <= 1,048,576
constexpr int kStaticMaxSweeps = 1024;
constexpr int kStaticMaxBands = 4096;
constexpr int kStaticMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kStaticTOff = 0;
constexpr size_t kStaticProgOff = align256(kStaticTOff + (size_t)kStaticMaxNodes * sizeof(float));
constexpr size_t kStaticChgOff = align256(kStaticProgOff + (size_t)(kStaticMaxBands + 1) * sizeof(unsigned));
constexpr size_t kStaticStateOff = align256(kStaticChgOff + (size_t)(kStaticMaxSweeps + 2) * sizeof(int));
constexpr size_t kStaticBytes = align256(kStaticStateOff + sizeof(rf::DevState));

std::mutex g_static_mu;
void *g_static_addr[kStaticMaxDevices] = {};

}  // namespace

// Scratch of rf_sweep_forward_static (about 4 MiB per device).  In host code
// this name is only a host-side stand-in: kernels receive the device address
// obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_rf_static_scratch[kStaticBytes];

extern "C" rf_status rf_sweep_forward_static(const rf_grid *grid, const float *proj5, float eps,
                                             const uint8_t *src, const rf_opts *opts, float *T,
                                             rf_stats *stats, void *stream) {
  if (!grid_ok(grid) || !proj5 || !src || !T) return RF_ERR_INVALID_ARG;
  if (!(eps >= 0.0f)) return RF_ERR_INVALID_ARG;
  rf_opts o = {0.0f, 64, RF_MODE_COLD, 0, 0, 1e-6f, 0, 0.0f};
  if (opts) o = *opts;
  if (o.max_sweeps < 1 || !(o.tol >= 0.0f) || !(o.rtol >= 0.0f) || (o.mode != RF_MODE_COLD && o.mode != RF_MODE_WARM))
    return RF_ERR_INVALID_ARG;
  const int ny = grid->ny, nx = grid->nx;
  const long long n = (long long)ny * nx;
  // sizes beyond the fixed scratch are rejected before any work is enqueued
  if (n > kStaticMaxNodes || o.max_sweeps > kStaticMaxSweeps) return RF_ERR_INVALID_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RF_ERR_CUDA;
  if (dev < 0 || dev >= kStaticMaxDevices) return RF_ERR_UNSUPPORTED;
  unsigned char *base = nullptr;
  {
    // once per device, with that device current: the device address of the
    // scratch array
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_rf_static_scratch) != cudaSuccess || !p) return RF_ERR_CUDA;
      g_static_addr[dev] = p;
    }
    base = (unsigned char *)g_static_addr[dev];
  }

  rf_ctx planner;  // a stack object: only the device and SM count are used
  planner.device = dev;
  if (cudaDeviceGetAttribute(&planner.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RF_ERR_CUDA;
  // the streamed variant needs a record buffer and the tile queue its queue
  // workspace: neither is available without allocation
  if (o.variant == RF_SWEEP_STREAMED || o.variant == RF_SWEEP_TILES || !variant_ok(o.variant))
    return RF_ERR_INVALID_ARG;
  SweepPlan pl;
  rf_status rs = plan_sweep(&planner, ny, nx, &o, o.variant == RF_SWEEP_TILED4 ? 4 : 1, &pl);
  if (rs != RF_OK) return rs;
  if (pl.grid > kStaticMaxBands) return RF_ERR_INVALID_ARG;

  cudaStream_t s = (cudaStream_t)stream;
  float *tb = (float *)(base + kStaticTOff);
  unsigned *progress = (unsigned *)(base + kStaticProgOff);
  int *changed = (int *)(base + kStaticChgOff);
  DevState *st = (DevState *)(base + kStaticStateOff);
  // the array keeps the previous call's contents: clear what must start at 0
  if (cudaMemsetAsync(progress, 0, sizeof(unsigned) * (pl.grid + 1), s) != cudaSuccess ||
      cudaMemsetAsync(changed, 0, sizeof(int) * (o.max_sweeps + 2), s) != cudaSuccess ||
      cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess)
    return RF_ERR_CUDA;

  int *has_src = changed + o.max_sweeps;
  init_kernel<<<blocks_for(n, 256, planner.num_sms * 8), 256, 0, s>>>(T, src, n, o.mode == RF_MODE_WARM, st,
                                                                        has_src);
  check_source_kernel<<<1, 32, 0, s>>>(has_src, st);

  SweepArgs a;
  a.ny = ny;
  a.nx = nx;
  a.h = grid->h;
  a.eps = eps;
  a.f = proj5;
  a.src = src;
  a.Ta = T;
  a.Tb = tb;
  a.R = pl.R;
  a.K = pl.K;
  a.max_sweeps = o.max_sweeps;
  a.tol = o.tol;
  a.rtol = o.rtol;
  a.tok_stride = (unsigned)((std::max(ny, nx) + pl.K - 1) / pl.K + 1);
  a.progress = progress;
  a.changed = changed;
  a.ctl.st = st;
  a.ctl.abort = changed + o.max_sweeps + 1;
  a.ctl.timeout_ns = 2000000000LL;
  void *args[] = {&a};
  if (cudaLaunchCooperativeKernel(pl.kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, s) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  // asynchronous path: report launch errors of the init kernels here rather
  // than leaving them to whatever call comes next
  if (!stats) return cuda_status(cudaGetLastError());
  DevState h;
  if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RF_ERR_CUDA;
  stats->status = h.status;
  stats->sweeps = h.sweeps;
  stats->converged = h.converged;
  stats->adj_sweeps = 0;
  stats->cell_updates = (int64_t)h.cell_updates;
  stats->max_residual = 0.0f;
  stats->rounds = 0;
  return (rf_status)h.status;
}
