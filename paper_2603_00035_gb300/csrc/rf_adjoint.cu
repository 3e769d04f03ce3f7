// rf_adjoint.cu -- a6-a8: adjoint of the converged discrete system and the
// parameter gradients.
//
// Paper: Sec. 3.3 (Eqs. 4-6) and App. A (Alg. 2).  With every residual
// scaled to unit diagonal, R_q = T_q - f_q(donors), the adjoint system
// J^T lambda = g reads
//     lambda_p = g_p + sum_{children q of p} (dT_q / dT_p) lambda_q,
// where a child q is a neighbour whose recorded update uses p as a donor
// and dT_q/dT_p is its donor weight (w1, 1 - w1, or 1 for a one-point
// update).  The system is triangular in arrival-time order; it is solved
// here by transposed line sweeps: the same band-pipelined persistent launch
// as the forward solve, gathering lambda from children (no atomics), until
// a sweep changes nothing (then lambda = g + W^T lambda holds exactly).
// The final pass writes dL/dtheta_p = lambda_p dT0_p/dtheta_p (Alg. 2 last
// loop; zero at sources and unreached nodes) and the optional lambda.
#include <algorithm>

#include <cub/device/device_radix_sort.cuh>

#include "rf_adjoint.h"
#include "rf_ctx.h"
#include "rf_sweep_common.cuh"

namespace rf {

struct AdjArgs {
  int ny, nx;
  const uint8_t *src;
  const float *T;
  const uint8_t *id;
  const float *w1;
  const float *dT;  // 5 planes
  const float *g;   // dL/dT
  float *La, *Lb;   // lambda ping-pong (La holds the result)
  float *grad;      // 5 planes out
  float *lam_out;   // nullable
  int R, K;
  int max_sweeps;
  unsigned tok_stride;
  unsigned *progress;
  int *changed;
  LaunchCtl ctl;
};

__host__ __device__ inline size_t adj_smem_bytes(int R, int K) {
  const int ext = R + 2 * K, W = ext + 2, P = W | 1, EP = ext | 1;
  // old lambda (K+2)P, new lambda (K+1)P, w1 (K+2)P, g' K*EP floats; ids (K+2)P bytes
  size_t fl = (size_t)(K + 2) * P * 2 + (size_t)(K + 1) * P + (size_t)K * EP;
  return fl * sizeof(float) + (size_t)(K + 2) * P;
}

constexpr int kAdjLanes = 4;  // lanes per node: lane q gathers neighbours 2q, 2q+1

__global__ void __launch_bounds__(1024) adjoint_sweep_kernel(AdjArgs a) {
  extern __shared__ float smem[];
  const int R = a.R, K = a.K, ext = R + 2 * K, W = ext + 2, P = W | 1, EP = ext | 1;
  float *old = smem;                        // (K+2) x P
  float *nw = old + (size_t)(K + 2) * P;    // (K+1) x P
  float *ww = nw + (size_t)(K + 1) * P;     // (K+2) x P  donor weights w1
  float *gg = ww + (size_t)(K + 2) * P;     // K x EP     masked dL/dT
  uint8_t *ids = (uint8_t *)(gg + (size_t)K * EP);  // (K+2) x P
  __shared__ int s_ok, s_any;

  const int tid = threadIdx.x, nth = blockDim.x, b = blockIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  const int cell = tid / kAdjLanes, q = tid % kAdjLanes;
  const long long plane = (long long)a.ny * a.nx;
  float *cur = a.La, *nxt = a.Lb;
  int sweep = 0, converged = 0;
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
    int nds[2], ndl[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) nb_tile_offset(dir, 2 * q + u, nds[u], ndl[u]);
    if (b < nb && !abort) {
      const int l0 = b * R, line0 = l0 - K - 1;
      for (int kb = 0; kb < nblk; ++kb) {
        const int s0 = kb * K;
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
        // stage lambda before the sweep, w1 and ids on (K+2) x W; warps walk
        // the non-contiguous direction, lanes the contiguous one
        {
          const int n_outer = col ? W : K + 2, n_inner = col ? K + 2 : W;
          for (int o = warp; o < n_outer; o += nwarps) {
            for (int in = lane; in < n_inner; in += 32) {
              const int ts = col ? in : o, tl = col ? o : in;
              const int s = s0 - 1 + ts, l = line0 + tl;
              float v = 0.0f, w = 0.0f;
              uint8_t d = 0;
              if (s >= 0 && s < S && l >= 0 && l < L) {
                const long long gi = gidx(dir, s, l, a.ny, a.nx);
                v = __ldcg(cur + gi);
                w = __ldg(a.w1 + gi);
                d = __ldg(a.id + gi);
              }
              old[ts * P + tl] = v;
              ww[ts * P + tl] = w;
              ids[ts * P + tl] = d;
            }
          }
        }
        for (int tl = tid; tl < W; tl += nth) {
          const int s = s0 - 1, l = line0 + tl;
          float v = 0.0f;
          if (s >= 0 && l >= 0 && l < L) {
            const long long gi = gidx(dir, s, l, a.ny, a.nx);
            v = (tl >= 1 && tl <= ext) ? __ldcg(nxt + gi) : __ldcg(cur + gi);
          }
          nw[tl] = v;
        }
        {
          const int n_outer = col ? ext : K, n_inner = col ? K : ext;
          for (int o = warp; o < n_outer; o += nwarps) {
            for (int in = lane; in < n_inner; in += 32) {
              const int t = col ? in : o, e = col ? o : in;
              const int s = s0 + t, l = l0 - K + e;
              float v = 0.0f;
              if (s < S && l >= 0 && l < L) {
                const long long gi = gidx(dir, s, l, a.ny, a.nx);
                v = (__ldg(a.T + gi) < kInf) ? __ldg(a.g + gi) : 0.0f;
              }
              gg[t * EP + e] = v;
            }
          }
        }
        __syncthreads();
        for (int t = tid; t < K; t += nth) {
          nw[(t + 1) * P] = old[(t + 1) * P];
          nw[(t + 1) * P + W - 1] = old[(t + 1) * P + W - 1];
        }
        for (int t = 0; t < K; ++t) {
          const int s = s0 + t;
          if (s >= S) break;
          const int e = cell, tl = e + 1, l = l0 - K + e;
          const bool live = (e < ext) && (l >= 0) && (l < L);
          float part = 0.0f;
          if (live) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int r = t + 1 + nds[u], cidx = tl + ndl[u];
              const float wq = child_weight(ids[r * P + cidx], ww[r * P + cidx], (2 * q + u + 4) & 7);
              if (wq != 0.0f) {
                const float lq = (nds[u] < 0) ? nw[t * P + cidx] : old[r * P + cidx];
                part = fmaf(wq, lq, part);
              }
            }
          }
          // fixed-order tree: ((q0 + q1) + (q2 + q3)), then + g
          part += __shfl_xor_sync(0xffffffffu, part, 1);
          part += __shfl_xor_sync(0xffffffffu, part, 2);
          if (q == 0 && e < ext) {
            float lnew = 0.0f;
            if (live) {
              const float lold = old[(t + 1) * P + tl];
              lnew = gg[t * EP + e] + part;
              if (e >= K && e < K + R) local_changed |= (__float_as_uint(lnew) != __float_as_uint(lold));
            }
            nw[(t + 1) * P + tl] = lnew;
          }
          __syncthreads();
        }
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
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          st_release_u32(&a.progress[b], base + kb + 1);
        }
      }
    }
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
  // a8: parameter gradients and lambda out
  for (long long p = (long long)blockIdx.x * nth + tid; p < plane; p += (long long)gridDim.x * nth) {
    const float lam = __ldcg(cur + p);
    const bool act = a.id[p] != 0 && !a.src[p];
#pragma unroll
    for (int c = 0; c < 5; ++c) a.grad[c * plane + p] = act ? lam * a.dT[c * plane + p] : 0.0f;
    if (a.lam_out) a.lam_out[p] = lam;
  }
  if (b == 0 && tid == 0) {
    a.ctl.st->adj_sweeps = sweep;
    if (!converged && !abort) set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
  }
}


// ---- RF_ADJ_ORDERED: radix sort on T, then a dependency-ordered gather ----
//
// Children always have a strictly larger T than their parents (the
// causality test of the two-point update; F > 0 for the one-point update),
// so processing nodes in decreasing T finishes every child before its
// parents (Alg. 2, "sort nodes by decreasing T").  A CUB radix sort orders
// the nodes; a persistent kernel then hands out the sorted positions in
// warp-sized tickets.  Each lane waits (bounded) until every child named by
// the record has published its multiplier, gathers them in a fixed
// neighbour order (no atomics on lambda), and publishes its own multiplier
// and the epoch of this launch in one 64-bit store (single-copy atomic, no
// fence: the parent reads nothing else of its child).  The latency chain is
// the depth of the stencil DAG, not a sweep count.

__global__ void ordered_keys_kernel(const float *T, unsigned *keys, unsigned *vals, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float t = T[p];
    // ascending key = decreasing T; unreached (+inf) nodes first (key 0)
    keys[p] = (t < kInf) ? ~__float_as_uint(t) : 0u;
    vals[p] = (unsigned)p;
  }
}

struct OrderedArgs {
  int ny, nx;
  long long n;            // ny * nx (plane stride of dT and grad)
  const uint8_t *src;
  const float *T;
  const uint8_t *id;
  const float *w1;
  const float *dT;
  const float *g;
  const unsigned *order;  // node indices by decreasing T
  unsigned long long *state;  // (epoch << 32) | lambda bits
  const unsigned *epoch;      // this launch's tag (device word, bumped before the launch)
  unsigned *ticket;
  float *grad;
  float *lam_out;
  LaunchCtl ctl;
};

__global__ void __launch_bounds__(256) ordered_gather_kernel(OrderedArgs a) {
  const int lane = threadIdx.x & 31;
  const long long n = a.n;
  const unsigned long long tag = (unsigned long long)__ldg(a.epoch) << 32;
  while (true) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(a.ticket, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= n || ld_acquire_s32(a.ctl.abort)) break;
    const long long pos = (long long)base + lane;
    bool done = pos >= n;
    long long p = -1;
    unsigned cmask = 0;  // children among the 8 neighbours
    float cw[8];
    float gsum = 0.0f;
    float dTp[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // partials, loaded before the wait
    bool act = false;
    int pi = 0, pj = 0;
    const int gny = a.ny, gnx = a.nx;
    if (!done) {
      p = a.order[pos];
      pi = (int)(p / gnx);
      pj = (int)(p - (long long)pi * gnx);
      const float tp = a.T[p];
      if (!(tp < kInf)) {
        // unreached: no residual, no children
        st_relaxed_u64(&a.state[p], tag);
        done = true;
      } else {
        gsum = a.g[p];
        act = a.id[p] != 0 && !a.src[p];
#pragma unroll
        for (int c = 0; c < 5; ++c) dTp[c] = act ? a.dT[c * n + p] : 0.0f;
      }
    }
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) {
      cw[nb] = 0.0f;
      const int ii = pi + nb_dy(nb), jj = pj + nb_dx(nb);
      if (!done && ii >= 0 && ii < gny && jj >= 0 && jj < gnx) {
        const long long qn = (long long)ii * gnx + jj;
        cw[nb] = child_weight(a.id[qn], a.w1[qn], (nb + 4) & 7);
        if (cw[nb] != 0.0f) cmask |= 1u << nb;
      }
    }
    const unsigned long long t0 = gtimer();
    unsigned spins = 0;
    while (!__all_sync(0xffffffffu, done)) {
      if (!done) {
        bool ready = true;
        float acc = gsum;
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) {
          if (cmask & (1u << nb)) {
            const long long qn = (long long)(pi + nb_dy(nb)) * gnx + (pj + nb_dx(nb));
            const unsigned long long v = ld_relaxed_u64(&a.state[qn]);
            ready = ready && ((v & 0xffffffff00000000ull) == tag);
            acc = fmaf(cw[nb], __uint_as_float((unsigned)v), acc);
          }
        }
        if (ready) {
          st_relaxed_u64(&a.state[p], tag | __float_as_uint(acc));
#pragma unroll
          for (int c = 0; c < 5; ++c) a.grad[c * n + p] = act ? acc * dTp[c] : 0.0f;
          if (a.lam_out) a.lam_out[p] = acc;
          done = true;
        } else if ((++spins & 63) == 0 &&
                   ((long long)(gtimer() - t0) > a.ctl.timeout_ns || ld_acquire_s32(a.ctl.abort))) {
          // the bound and the abort flag are checked every 64 polls: an
          // extra L2 round trip on every poll doubled the poll period
          raise_timeout(a.ctl);
          done = true;
        }
      }
    }
  }
  // unreached nodes: zero gradient and lambda
}

__global__ void ordered_unreached_kernel(const float *T, float *grad, float *lam, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    if (!(T[p] < kInf)) {
#pragma unroll
      for (int c = 0; c < 5; ++c) grad[c * n + p] = 0.0f;
      if (lam) lam[p] = 0.0f;
    }
  }
}


// ---- RF_ADJ_LEVELS: a DAG-depth pass, then a level-synchronous gather ----
//
// The record's donor edges form a DAG (a donor's T is strictly below its
// child's).  The depth pass gives every reached node its level, the length
// of the longest donor chain from a node without donors (sources: level 0),
//     level_q = 1 + max over donors p of q of level_p,
// by walking the T order upwards with the same ticketed, dependency-polling
// scheme as the ordered gather (a node waits for at most two donors).  A
// child's level exceeds each of its donors' levels, so after a radix sort on
// the level the gather processes whole levels from the deepest to level 0,
// one grid-wide barrier between levels, with plain loads of the children's
// multipliers: no per-node polling.  The multiplier of each node is the same
// fixed-order sum as in the ordered gather, so the two agree bit for bit.

struct LevelArgs {
  int ny, nx;
  long long n;
  const uint8_t *src;
  const float *T;
  const uint8_t *id;
  const float *w1;
  const float *dT;
  const float *g;
  const unsigned *order;      // depth pass: node indices by decreasing T
  unsigned long long *state;  // depth pass: (epoch << 32) | level
  const unsigned *epoch;      // this launch's tag (device word, bumped before the launch)
  unsigned *ticket;
  unsigned *level;            // depth pass output: level of each node (n for unreached nodes)
  unsigned *n_levels;         // depth pass: 1 + the largest level (0: no reached node)
  const unsigned *by_level;   // gather: node indices sorted by level
  const unsigned *start;      // gather: first position of each level in by_level
  unsigned long long *bar;    // gather: arrivals at the level barrier (monotone)
  float *lam;                 // gather: multipliers (internal)
  float *grad;
  float *lam_out;
  LaunchCtl ctl;
};

__device__ __forceinline__ bool in_grid(int i, int j, int ny, int nx) {
  return i >= 0 && i < ny && j >= 0 && j < nx;
}

__global__ void __launch_bounds__(256) level_depth_kernel(LevelArgs a) {
  const int lane = threadIdx.x & 31;
  const long long n = a.n;
  const unsigned long long tag = (unsigned long long)__ldg(a.epoch) << 32;
  unsigned wmax = 0;
  while (true) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(a.ticket, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= n || ld_acquire_s32(a.ctl.abort)) break;
    const long long pos = (long long)base + lane;
    bool done = pos >= n;
    long long q = -1;
    int qi = 0, qj = 0, d0 = -1, d1 = -1;
    if (!done) {
      q = a.order[n - 1 - pos];  // increasing T
      if (!(a.T[q] < kInf)) {
        a.level[q] = (unsigned)n;  // unreached: sorted past every level
        done = true;
      } else {
        qi = (int)(q / a.nx);
        qj = (int)(q - (long long)qi * a.nx);
        const uint8_t idq = a.id[q];
        if (idq & 0x30) d0 = idq & 7;
        if (idq & 0x20) d1 = (d0 + 1) & 7;
        // a record names in-grid donors only; drop any other
        if (d0 >= 0 && !in_grid(qi + nb_dy(d0), qj + nb_dx(d0), a.ny, a.nx)) d0 = -1;
        if (d1 >= 0 && !in_grid(qi + nb_dy(d1), qj + nb_dx(d1), a.ny, a.nx)) d1 = -1;
      }
    }
    const unsigned long long t0 = gtimer();
    unsigned spins = 0;
    while (!__all_sync(0xffffffffu, done)) {
      if (!done) {
        bool ready = true;
        unsigned lv = 0;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int d = u ? d1 : d0;
          if (d >= 0) {
            const long long pn = (long long)(qi + nb_dy(d)) * a.nx + (qj + nb_dx(d));
            const unsigned long long v = ld_relaxed_u64(&a.state[pn]);
            ready = ready && ((v & 0xffffffff00000000ull) == tag);
            lv = max(lv, (unsigned)v + 1u);
          }
        }
        if (ready) {
          st_relaxed_u64(&a.state[q], tag | lv);
          a.level[q] = lv;
          wmax = max(wmax, lv + 1u);
          done = true;
        } else if ((++spins & 63) == 0 &&
                   ((long long)(gtimer() - t0) > a.ctl.timeout_ns || ld_acquire_s32(a.ctl.abort))) {
          raise_timeout(a.ctl);
          done = true;
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  if (lane == 0 && wmax) atomicMax(a.n_levels, wmax);
}

// start[l] = first position of level l in the level-sorted keys, for every
// level present; start[l + 1] = one past its last.  Levels run 0..max
// without gaps (a node of level l > 0 has a donor of level l - 1).
__global__ void level_starts_kernel(const unsigned *keys, unsigned *start, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned k = keys[i];
    if (k >= (unsigned)n) continue;
    if (i == 0 || keys[i - 1] != k) start[k] = (unsigned)i;
    if (i == n - 1 || keys[i + 1] != k) start[k + 1] = (unsigned)(i + 1);
  }
}

// Bounded barrier on a monotone arrival counter, in two halves so that a
// CTA can fetch the next level's static data between them: the k-th
// barrier of the launch waits for k * gridDim.x arrivals (no reset, one
// atomic per CTA).
__device__ __forceinline__ void level_arrive(unsigned long long *bar) {
  __syncthreads();
  // release: the CTA's stores before the __syncthreads become visible to
  // every CTA that acquires the counter past this arrival
  if (threadIdx.x == 0)
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(bar), "l"(1ull) : "memory");
}

__device__ __forceinline__ bool level_wait(unsigned long long *bar, unsigned long long target, const LaunchCtl &c) {
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_acquire_u64(bar) < target) {
      const unsigned long long t0 = gtimer();
      while (ld_acquire_u64(bar) < target) {
        if ((long long)(gtimer() - t0) > c.timeout_ns || ld_acquire_s32(c.abort)) {
          raise_timeout(c);
          ok = 0;
          break;
        }
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// What a node of the level gather needs besides its children's multipliers:
// fetched before the barrier that precedes its level, so that after the
// barrier only the multipliers remain to be loaded.
struct LevelNode {
  long long p;    // -1: no node
  float cw[8];    // child weights in neighbour order (0: not a child)
  float g;
  bool act;       // the node has a gradient (recorded update, not a source)
  float d[5];     // dT0/dtheta
};

__device__ __forceinline__ void level_fetch(const LevelArgs &a, long long i, long long e, LevelNode &v) {
  v.p = -1;
  if (i >= e) return;
  const long long p = a.by_level[i], n = a.n;
  const int pi = (int)(p / a.nx), pj = (int)(p - (long long)pi * a.nx);
  v.p = p;
  v.g = a.g[p];
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) {
    const int ii = pi + nb_dy(nb), jj = pj + nb_dx(nb);
    v.cw[nb] = 0.0f;
    if (ii >= 0 && ii < a.ny && jj >= 0 && jj < a.nx) {
      const long long qn = (long long)ii * a.nx + jj;
      v.cw[nb] = child_weight(a.id[qn], a.w1[qn], (nb + 4) & 7);
    }
  }
  v.act = a.id[p] != 0 && !a.src[p];
#pragma unroll
  for (int c = 0; c < 5; ++c) v.d[c] = a.dT[c * n + p];  // not behind act: one round trip fewer
}

__device__ __forceinline__ void level_finish(const LevelArgs &a, const LevelNode &v) {
  if (v.p < 0) return;
  const long long p = v.p, n = a.n;
  const int pi = (int)(p / a.nx), pj = (int)(p - (long long)pi * a.nx);
  float acc = v.g;
#pragma unroll
  for (int nb = 0; nb < 8; ++nb)
    if (v.cw[nb] != 0.0f)
      acc = fmaf(v.cw[nb], __ldcg(a.lam + (long long)(pi + nb_dy(nb)) * a.nx + (pj + nb_dx(nb))), acc);
  __stcg(a.lam + p, acc);
#pragma unroll
  for (int c = 0; c < 5; ++c) a.grad[c * n + p] = v.act ? acc * v.d[c] : 0.0f;
  if (a.lam_out) a.lam_out[p] = acc;
}

// Level starts held in shared memory for the first kLevelSmem levels.
constexpr int kLevelSmem = 16384;

__global__ void __launch_bounds__(512) level_gather_kernel(LevelArgs a) {
  extern __shared__ unsigned s_start[];
  const long long n = a.n;
  // levels 0 .. nl - 1, counted by the depth pass; none if it gave up
  const long long nl = ld_acquire_s32(a.ctl.abort) ? 0 : min((long long)*a.n_levels, n);
  const long long held = min(nl + 1, (long long)kLevelSmem);
  for (long long k = threadIdx.x; k < held; k += blockDim.x) s_start[k] = a.start[k];
  __syncthreads();
  auto level_start = [&](long long L) -> long long {
    return min((long long)(L < held ? s_start[L] : a.start[L]), n);
  };
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
  unsigned long long step = 0;
  LevelNode v;
  v.p = -1;
  if (nl > 0) level_fetch(a, level_start(nl - 1) + gt, level_start(nl), v);
  for (long long L = nl - 1; L >= 0; --L) {
    level_finish(a, v);
    // a level wider than the grid of threads: the rest without prefetch
    const long long e = level_start(L + 1);
    for (long long i = level_start(L) + gt + gs; i < e; i += gs) {
      LevelNode w;
      level_fetch(a, i, e, w);
      level_finish(a, w);
    }
    if (L == 0) break;
    level_arrive(a.bar);
    level_fetch(a, level_start(L - 1) + gt, level_start(L), v);  // overlaps the barrier
    if (!level_wait(a.bar, (++step) * gridDim.x, a.ctl)) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl.st->adj_sweeps = (int)nl;
}

}  // namespace rf

using namespace rf;

namespace {

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace rf {

// The epoch tagging the per-node state words lives on the device and is
// bumped by a kernel on the launch stream, so a replayed CUDA graph gets a
// new tag on every replay (a tag fixed at capture would find every word
// already final from the previous replay).  The words are cleared on first
// use and when the host's count of launches nears the 32-bit wrap.
__global__ void epoch_bump_kernel(unsigned *e) {
  const unsigned v = *e + 1u;
  *e = v ? v : 1u;
}

rf_status adjoint_next_epoch(rf_ctx *ctx, long long n, cudaStream_t s, const unsigned **epoch) {
  const bool fresh = ctx->adj_state_cap < (size_t)n || !ctx->adj_state;
  rf_status rs;
  if ((rs = ensure(&ctx->adj_state, &ctx->adj_state_cap, (size_t)n)) != RF_OK) return rs;
  if (fresh || ctx->adj_epoch == 0xfffffff0u) {
    if (cudaMemsetAsync(ctx->adj_state, 0, sizeof(unsigned long long) * ctx->adj_state_cap, s) != cudaSuccess ||
        cudaMemsetAsync(&ctx->state->adj_epoch, 0, sizeof(unsigned), s) != cudaSuccess)
      return RF_ERR_CUDA;
    ctx->adj_epoch = 0;
  }
  ++ctx->adj_epoch;
  epoch_bump_kernel<<<1, 1, 0, s>>>(&ctx->state->adj_epoch);
  *epoch = &ctx->state->adj_epoch;
  return cuda_status(cudaGetLastError());
}

// The ordered adjoint of one ny x nx grid.
rf_status adjoint_ordered(rf_ctx *ctx, int ny, int nx, const uint8_t *src, const float *T, const rf_record *rec,
                          const float *dLdT, float *dLdproj5, float *lambda, cudaStream_t s) {
  ctx->last_stream = s;
  const long long n = (long long)ny * nx;
  // scratch: keys in/out, values in/out, ticket, abort flag, CUB temp
  size_t temp_bytes = 0;
  if (cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, (unsigned *)nullptr, (unsigned *)nullptr,
                                      (unsigned *)nullptr, (unsigned *)nullptr, (int)n, 0, 32, s) != cudaSuccess)
    return RF_ERR_CUDA;
  const size_t arr = align_up((size_t)n * sizeof(unsigned));
  const size_t need = 4 * arr + 256 + align_up(temp_bytes);
  rf_status rs;
  if ((rs = ensure((unsigned char **)&ctx->scratch, &ctx->scratch_cap, need)) != RF_OK) return rs;
  unsigned char *base = (unsigned char *)ctx->scratch;
  unsigned *kin = (unsigned *)base, *kout = (unsigned *)(base + arr), *vin = (unsigned *)(base + 2 * arr),
           *vout = (unsigned *)(base + 3 * arr);
  unsigned *ctl_words = (unsigned *)(base + 4 * arr);  // [0] ticket, [1] abort
  void *temp = base + 4 * arr + 256;
  const unsigned *epoch;
  if ((rs = adjoint_next_epoch(ctx, n, s, &epoch)) != RF_OK) return rs;
  if (cudaMemsetAsync(ctl_words, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return RF_ERR_CUDA;

  ordered_keys_kernel<<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(T, kin, vin, n);
  if (cub::DeviceRadixSort::SortPairs(temp, temp_bytes, kin, kout, vin, vout, (int)n, 0, 32, s) != cudaSuccess)
    return RF_ERR_CUDA;

  OrderedArgs a;
  a.ny = ny;
  a.nx = nx;
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
  a.ticket = ctl_words;
  a.grad = dLdproj5;
  a.lam_out = lambda;
  a.ctl.st = ctx->state;
  a.ctl.abort = (int *)(ctl_words + 1);
  a.ctl.timeout_ns = ctx->timeout_ns;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ordered_gather_kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    return RF_ERR_CUDA;
  // every warp that takes a ticket must be resident: a cooperative launch
  // guarantees it.  Full occupancy: with fence-free publishing the gather
  // measured 2.72 / 2.50 / 2.45 / 2.45 ms at 1 / 2 / 3 / 4 CTAs per SM
  // (2048^2 workload); with release stores a small window had been best
  // (4.83 ms at 2 CTAs, 8.41 ms at 4).  A lane-granular hand-out (free
  // lanes taking new positions while others wait) measured slower.
  void *args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void *)ordered_gather_kernel, dim3(per_sm * ctx->num_sms), dim3(256),
                                  args, 0, s) != cudaSuccess)
    return RF_ERR_CUDA;
  ordered_unreached_kernel<<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(T, dLdproj5, lambda, n);
  return cuda_status(cudaGetLastError());
}


// The level-scheduled adjoint of one grid: T order (radix sort), the depth
// pass, a radix sort on the level, the level starts, the level gather.
rf_status adjoint_levels(rf_ctx *ctx, int ny, int nx, const uint8_t *src, const float *T, const rf_record *rec,
                         const float *dLdT, float *dLdproj5, float *lambda, cudaStream_t s) {
  ctx->last_stream = s;
  const long long n = (long long)ny * nx;
  int lbits = 1;  // level keys are <= n
  while (lbits < 32 && ((unsigned long long)n >> lbits) != 0) ++lbits;
  size_t t1 = 0, t2 = 0;
  if (cub::DeviceRadixSort::SortPairs(nullptr, t1, (unsigned *)nullptr, (unsigned *)nullptr, (unsigned *)nullptr,
                                      (unsigned *)nullptr, (int)n, 0, 32, s) != cudaSuccess ||
      cub::DeviceRadixSort::SortPairs(nullptr, t2, (unsigned *)nullptr, (unsigned *)nullptr, (unsigned *)nullptr,
                                      (unsigned *)nullptr, (int)n, 0, lbits, s) != cudaSuccess)
    return RF_ERR_CUDA;
  size_t temp_bytes = std::max(t1, t2);
  const size_t arr = align_up((size_t)n * sizeof(unsigned)), arr1 = align_up((size_t)(n + 1) * sizeof(unsigned));
  const size_t need = 4 * arr + arr1 + 256 + align_up(temp_bytes);
  rf_status rs;
  if ((rs = ensure((unsigned char **)&ctx->scratch, &ctx->scratch_cap, need)) != RF_OK) return rs;
  unsigned char *base = (unsigned char *)ctx->scratch;
  unsigned *kin = (unsigned *)base, *kout = (unsigned *)(base + arr), *vin = (unsigned *)(base + 2 * arr),
           *vout = (unsigned *)(base + 3 * arr), *start = (unsigned *)(base + 4 * arr);
  // control words: [0] ticket, [1] abort, [2] level count, [4..5] barrier counter
  unsigned *ctl_words = (unsigned *)(base + 4 * arr + arr1);
  void *temp = base + 4 * arr + arr1 + 256;
  if ((rs = ensure(&ctx->lbuf, &ctx->lbuf_cap, (size_t)n)) != RF_OK) return rs;
  const unsigned *epoch;
  if ((rs = adjoint_next_epoch(ctx, n, s, &epoch)) != RF_OK) return rs;
  if (cudaMemsetAsync(ctl_words, 0, 6 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(&ctx->state->adj_sweeps, 0, sizeof(int), s) != cudaSuccess)
    return RF_ERR_CUDA;

  ordered_keys_kernel<<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(T, kin, vin, n);
  if (cub::DeviceRadixSort::SortPairs(temp, temp_bytes, kin, kout, vin, vout, (int)n, 0, 32, s) != cudaSuccess)
    return RF_ERR_CUDA;

  LevelArgs a;
  a.ny = ny;
  a.nx = nx;
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
  a.ticket = ctl_words;
  a.level = kin;  // the T keys are consumed
  a.n_levels = ctl_words + 2;
  a.by_level = vout;  // the T order is consumed by the depth pass
  a.start = start;
  a.bar = (unsigned long long *)(ctl_words + 4);
  a.lam = ctx->lbuf;
  a.grad = dLdproj5;
  a.lam_out = lambda;
  a.ctl.st = ctx->state;
  a.ctl.abort = (int *)(ctl_words + 1);
  a.ctl.timeout_ns = ctx->timeout_ns;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, level_depth_kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    return RF_ERR_CUDA;
  // every warp that takes a ticket must be resident: cooperative launch
  void *args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void *)level_depth_kernel, dim3(per_sm * ctx->num_sms), dim3(256), args,
                                  0, s) != cudaSuccess)
    return RF_ERR_CUDA;
  // group the nodes by level (vin still holds 0..n-1: the sort leaves its inputs)
  if (cub::DeviceRadixSort::SortPairs(temp, temp_bytes, kin, kout, vin, vout, (int)n, 0, lbits, s) != cudaSuccess)
    return RF_ERR_CUDA;
  level_starts_kernel<<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(kout, start, n);
  // one CTA of 512 threads per SM: the widest level of a 2048^2 grid (a few
  // thousand nodes) fits in one pass, and the barrier takes one arrival per SM
  const size_t gsmem = kLevelSmem * sizeof(unsigned);
  if (cudaFuncSetAttribute(level_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem) !=
          cudaSuccess ||
      cudaLaunchCooperativeKernel((const void *)level_gather_kernel, dim3(ctx->num_sms), dim3(512), args, gsmem,
                                  s) != cudaSuccess)
    return RF_ERR_CUDA;
  ordered_unreached_kernel<<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(T, dLdproj5, lambda, n);
  return cuda_status(cudaGetLastError());
}

}  // namespace rf

extern "C" rf_status rf_adjoint(rf_ctx *ctx, const rf_grid *grid, const uint8_t *src, const float *T,
                                const rf_record *rec, const float *dLdT, float *dLdproj5, float *lambda,
                                int algo, void *stream) {
  if (!ctx || !grid_ok(grid) || !src || !T || !rec || !rec->id || !rec->w1 || !rec->dT || !dLdT ||
      !dLdproj5)
    return RF_ERR_INVALID_ARG;
  if (algo != RF_ADJ_SWEEP && algo != RF_ADJ_ORDERED && algo != RF_ADJ_LEVELS && algo != RF_ADJ_TILES)
    return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  if (algo == RF_ADJ_TILES)
    return rf::adjoint_tiles(ctx, grid->ny, grid->nx, src, T, rec, dLdT, dLdproj5, lambda, (cudaStream_t)stream);
  if (algo == RF_ADJ_LEVELS)
    return rf::adjoint_levels(ctx, grid->ny, grid->nx, src, T, rec, dLdT, dLdproj5, lambda, (cudaStream_t)stream);
  if (algo == RF_ADJ_ORDERED)
    return rf::adjoint_ordered(ctx, grid->ny, grid->nx, src, T, rec, dLdT, dLdproj5, lambda, (cudaStream_t)stream);
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ny = grid->ny, nx = grid->nx;
  const long long n = (long long)ny * nx;
  const int max_sweeps = 256;

  // plan: same band geometry rules as the forward sweep
  int K = 32, R = 64;
  int dev_max_smem = 0;
  cudaDeviceGetAttribute(&dev_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  int grid_ = 0, threads = 0;
  size_t smem = 0;
  for (int attempt = 0; attempt < 8; ++attempt) {
    threads = kAdjLanes * (R + 2 * K);
    smem = adj_smem_bytes(R, K);
    if (threads > 1024 || (long long)smem > dev_max_smem) return RF_ERR_UNSUPPORTED;
    cudaFuncSetAttribute(adjoint_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_sweep_kernel, threads, smem) !=
        cudaSuccess)
      return RF_ERR_CUDA;
    grid_ = (std::max(ny, nx) + R - 1) / R;
    if (per_sm > 0 && grid_ <= per_sm * ctx->num_sms) break;
    R *= 2;
    grid_ = 0;
  }
  if (!grid_) return RF_ERR_UNSUPPORTED;

  rf_status rs;
  if ((rs = ensure(&ctx->lbuf, &ctx->lbuf_cap, (size_t)(2 * n))) != RF_OK) return rs;
  if ((rs = ensure(&ctx->progress, &ctx->progress_cap, (size_t)grid_ + 1)) != RF_OK) return rs;
  if ((rs = ensure(&ctx->changed, &ctx->changed_cap, (size_t)max_sweeps + 2)) != RF_OK) return rs;
  cudaMemsetAsync(ctx->progress, 0, sizeof(unsigned) * (grid_ + 1), s);
  cudaMemsetAsync(ctx->changed, 0, sizeof(int) * (max_sweeps + 2), s);
  cudaMemsetAsync(&ctx->state->bar, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(&ctx->state->adj_sweeps, 0, sizeof(int), s);
  cudaMemsetAsync(ctx->lbuf, 0, sizeof(float) * n, s);  // lambda starts at 0

  AdjArgs a;
  a.ny = ny;
  a.nx = nx;
  a.src = src;
  a.T = T;
  a.id = rec->id;
  a.w1 = rec->w1;
  a.dT = rec->dT;
  a.g = dLdT;
  a.La = ctx->lbuf;
  a.Lb = ctx->lbuf + n;
  a.grad = dLdproj5;
  a.lam_out = lambda;
  a.R = R;
  a.K = K;
  a.max_sweeps = max_sweeps;
  a.tok_stride = (unsigned)((std::max(ny, nx) + K - 1) / K + 1);
  a.progress = ctx->progress;
  a.changed = ctx->changed;
  a.ctl.st = ctx->state;
  a.ctl.abort = ctx->changed + max_sweeps + 1;
  a.ctl.timeout_ns = ctx->timeout_ns;
  void *args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)adjoint_sweep_kernel, dim3(grid_), dim3(threads),
                                              args, smem, s);
  return e == cudaSuccess ? RF_OK : RF_ERR_CUDA;
}
