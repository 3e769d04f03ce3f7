// rf_sweep_stream.cu -- a2-a4, streamed variant of the forward line sweeps.
//
// Same schedule as the tiled sweep in rf_sweep.cu (Sec. 3.2 column/row
// fronts, bands of R lines per CTA, K-step blocks with recomputed halos,
// replacement update T <- min valid candidate, on-device convergence), with
// two changes aimed at the line-step critical path:
//
// 1. Node records.  Everything a node's 16 candidates need that depends
//    only on the fields is computed once per solve (records_kernel) and
//    kept in HBM, 24 floats per node, in two orientations: row-major for
//    row sweeps and column-major for column sweeps, so that the nodes of
//    one line step are contiguous in both.  During a sweep a single thread
//    per CTA copies the records of each line step into shared memory with
//    the bulk-copy engine (cp.async.bulk + an mbarrier per row), one block
//    ahead of the threads that step, instead of recomputing square roots
//    and divisions for every node in every block of every sweep.
//
// 2. Cone form of the two-point update (rf_cone.cuh): per stencil 12
//    instructions instead of ~30.
//
// Records of a block are stored for the trapezoid of nodes that can still
// influence the band (line step t: tile lines e in [t+1, EXT-1-t)), as six
// planes of float4 so that consecutive threads read consecutive 16 bytes.
#include <algorithm>

#include "rf_cone.cuh"
#include "rf_ctx.h"
#include "rf_sweep_common.cuh"
#include "rf_sweep_stream.h"

namespace rf {

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy helpers (PTX ISA: mbarrier, cp.async.bulk)
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of parity `parity`; false after timeout_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *m, unsigned parity, long long timeout_ns) {
  if (mbar_try_wait(m, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait(m, parity)) {
    if ((long long)(gtimer() - t0) > timeout_ns) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(m))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Records of every node in both orientations.  A 32 x 32 tile of nodes per
// CTA: computed with threads along x (coalesced field loads, row-major
// stores), then transposed through shared memory one plane at a time for
// the column-major stores.
constexpr int kRecTile = 32;
constexpr int kRecRows = 8;  // thread rows; each thread takes 4 nodes

__global__ void __launch_bounds__(kRecTile *kRecRows) records_kernel(const float *f, const uint8_t *src, int ny,
                                                                     int nx, float h, float eps, float4 *rec_row,
                                                                     float4 *rec_col) {
  __shared__ float4 tile[kRecTile][kRecTile + 1];
  const long long n = (long long)ny * nx;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.y * kRecTile, j0 = blockIdx.x * kRecTile;
  constexpr int U = kRecTile / kRecRows;
  float4 q[U][kPlanes] = {};
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int i = i0 + ty + kRecRows * u, j = j0 + tx;
    if (i < ny && j < nx) {
      const long long g = (long long)i * nx + j;
      node_record(f[g], f[n + g], f[2 * n + g], f[3 * n + g], f[4 * n + g], h, eps, src[g] != 0, q[u]);
#pragma unroll
      for (int c = 0; c < kPlanes; ++c) rec_row[c * n + g] = q[u][c];
    }
  }
#pragma unroll
  for (int c = 0; c < kPlanes; ++c) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < U; ++u) tile[ty + kRecRows * u][tx] = q[u][c];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + ty + kRecRows * u, i = i0 + tx;
      if (i < ny && j < nx) rec_col[c * n + (long long)j * ny + i] = tile[tx][ty + kRecRows * u];
    }
  }
}

// ---------------------------------------------------------------------------
// The streamed sweep kernel.  Template parameters: K line steps per block
// and EXT = R + 2K tile lines; R = EXT - 2K.  Threads: 4 * EXT; the first
// EXT step (one node each), thread kProducer issues the record copies, all
// of them stage old T, load the first row and publish.
template <int K, int EXT>
struct StreamShape {
  static constexpr int R = EXT - 2 * K;
  static constexpr int W = EXT + 2;
  static constexpr int P = W | 1;                   // row pitch of old / nw (odd)
  static constexpr int NTR = K * (EXT - 1 - K);     // trapezoid nodes per block
  static constexpr int THREADS = 4 * EXT;
  static constexpr int PRODUCER = ((EXT + 31) / 32) * 32;  // first thread after the steppers
  static constexpr int OLD_PER = ((K + 2) * W + THREADS - 1) / THREADS;
  static constexpr size_t REC_BYTES = (size_t)kPlanes * NTR * sizeof(float4);
  static constexpr size_t MBAR_OFF = REC_BYTES;
  static constexpr size_t ARMS_OFF = MBAR_OFF + (size_t)K * sizeof(uint64_t);
  static constexpr size_t OLD_OFF = ARMS_OFF + (size_t)K * sizeof(int);
  static constexpr size_t NW_OFF = OLD_OFF + (size_t)(K + 2) * P * sizeof(float);
  static constexpr size_t SMEM = NW_OFF + (size_t)(K + 1) * P * sizeof(float);
  static_assert(R >= K, "band must cover the halo");
  static_assert(PRODUCER < THREADS, "a thread must be left to issue copies");
  static_assert(OLD_PER <= 12, "old-T staging exceeds its register budget");
};

// Trapezoid offset of row t: rows u < t hold EXT - 2 - 2u records each.
template <int EXT>
__host__ __device__ constexpr int trap_off(int t) {
  return t * (EXT - 1 - t);
}

// Issue the record copies of row t of the block starting at line step s0
// (one thread).  Row t covers tile lines e in [t+1, EXT-1-t) of step s0+t,
// clipped to the grid; an empty row arms its barrier with zero bytes so
// every row's barrier completes exactly one phase per block.
template <int K, int EXT>
__device__ __forceinline__ void issue_row(const float4 *rec, long long n, float4 *pl, uint64_t *mbar, int *arms,
                                          int t, int s0, int S, int L, int l0, bool rev) {
  const int s = s0 + t;
  const int l_lo = l0 - K + t + 1;
  const int cnt = EXT - 2 - 2 * t;
  const int c_lo = max(l_lo, 0), c_hi = min(l_lo + cnt - 1, L - 1);
  arms[t] += 1;
  if (s >= S || c_lo > c_hi) {
    mbar_arrive_tx(&mbar[t], 0u);
    return;
  }
  const unsigned bytes = (unsigned)(c_hi - c_lo + 1) * (unsigned)sizeof(float4);
  mbar_arrive_tx(&mbar[t], bytes * kPlanes);
  const long long g = (long long)(rev ? S - 1 - s : s) * L + c_lo;
  const int r = trap_off<EXT>(t) + (c_lo - l_lo);
  constexpr int NTR = StreamShape<K, EXT>::NTR;
#pragma unroll
  for (int c = 0; c < kPlanes; ++c) bulk_g2s(pl + c * NTR + r, rec + c * n + g, bytes, &mbar[t]);
}

struct StreamArgs {
  int ny, nx;
  const float4 *rec_row, *rec_col;  // 6 planes each, row-/column-major
  float *Ta, *Tb;
  int max_sweeps;
  float tol, rtol;
  unsigned tok_stride;
  unsigned *progress;
  int *changed;
  LaunchCtl ctl;
};

// K line steps of one block (threads e < EXT; all threads reach every
// barrier).  After the barrier of step t, the producer arms row t of the
// next block through next_row(t).  Returns whether an inner node changed;
// sets bad when a record wait timed out.
template <int DIR, int K, int EXT, class NextRow>
__device__ __forceinline__ int stream_steps(const float4 *__restrict__ pl, const float *__restrict__ old, float *nw,
                                            uint64_t *mbar, unsigned parity, int t_end, int l0, int L, float tol,
                                            float rtol, long long timeout_ns, bool &bad, NextRow next_row) {
  using Sh = StreamShape<K, EXT>;
  constexpr int P = Sh::P, NTR = Sh::NTR;
  const int e = threadIdx.x, tl = e + 1, l = l0 - K + e;
  const bool valid = (e < EXT) && (l >= 0) && (l < L);
  const bool inband = (e >= K) && (e < K + Sh::R);
  int changed = 0;
  for (int t = 0; t < t_end; ++t) {
    if (e < EXT && e > t && e < EXT - 1 - t && !bad) {
      if (!mbar_wait(&mbar[t], parity, timeout_ns)) {
        bad = true;
      } else {
        const int r = trap_off<EXT>(t) + e - t - 1;
        const float4 q0 = pl[r], q1 = pl[NTR + r], q2 = pl[2 * NTR + r];
        const float4 q3 = pl[3 * NTR + r], q4 = pl[4 * NTR + r], q5 = pl[5 * NTR + r];
        float Tn[8];
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) {
          const int ds = tile_ds<DIR>(nb), dl = tile_dl<DIR>(nb);
          Tn[nb] = (ds < 0) ? nw[t * P + tl + dl] : old[(t + 1 + ds) * P + tl + dl];
        }
        const float cand = cone_min(q0, q1, q2, q3, q4, q5, Tn);
        float tnew = kInf;
        if (valid) {
          tnew = (q0.x < 0.0f) ? 0.0f : cand;
          if (inband) changed |= node_changed(tnew, old[(t + 1) * P + tl], tol, rtol);
        }
        nw[(t + 1) * P + tl] = tnew;
      }
    }
    __syncthreads();
    next_row(t);
  }
  return changed;
}

template <int K, int EXT>
__global__ void __launch_bounds__(4 * EXT, 1) sweep_stream_kernel(StreamArgs a) {
  using Sh = StreamShape<K, EXT>;
  constexpr int R = Sh::R, W = Sh::W, P = Sh::P, NTH = Sh::THREADS, OP = Sh::OLD_PER;
  extern __shared__ float4 smem4[];
  unsigned char *sb = reinterpret_cast<unsigned char *>(smem4);
  float4 *pl = smem4;                                                // records, kPlanes x NTR
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sb + Sh::MBAR_OFF);  // one per trapezoid row
  int *arms = reinterpret_cast<int *>(sb + Sh::ARMS_OFF);            // phases armed per row
  float *old = reinterpret_cast<float *>(sb + Sh::OLD_OFF);          // (K+2) x P  T before the sweep
  float *nw = reinterpret_cast<float *>(sb + Sh::NW_OFF);            // (K+1) x P  T of this sweep
  __shared__ int s_ok;
  __shared__ int s_any;

  const int tid = threadIdx.x, b = blockIdx.x;
  const long long plane = (long long)a.ny * a.nx;
  if (tid < K) arms[tid] = 0;
  if (tid == 0) {
    for (int t = 0; t < K; ++t) mbar_init(&mbar[t], 1);
    fence_mbar_init();
  }
  __syncthreads();

  float *cur = a.Ta, *nxt = a.Tb;
  int sweep = 0;
  int converged = 0;
  bool abort = false;
  unsigned blk = 0;  // blocks this CTA has started: parity of the record barriers

  while (true) {
    const int dir = sweep & 3;
    const bool col = (dir & 1) == 0;
    const bool rev = dir >= 2;
    const int S = col ? a.nx : a.ny;
    const int L = col ? a.ny : a.nx;
    const int nb = (L + R - 1) / R;
    const int nblk = (S + K - 1) / K;
    const unsigned base = (unsigned)sweep * a.tok_stride;
    const float4 *rec = col ? a.rec_col : a.rec_row;
    int local_changed = 0;
    // old-T staging list of this thread (ts | tl << 8); consecutive threads
    // take consecutive memory (steps for column sweeps, lines for rows)
    int oldidx[OP];
#pragma unroll
    for (int j = 0; j < OP; ++j) {
      const int f = tid + j * NTH;
      int ts = 0, tl = 0;
      if (col) { tl = f / (K + 2); ts = f - tl * (K + 2); }
      else     { ts = f / W;       tl = f - ts * W; }
      oldidx[j] = (f < (K + 2) * W) ? (ts | (tl << 8)) : -1;
    }

    if (b < nb && !abort) {
      const int l0 = b * R;
      const int line0 = l0 - K - 1;  // global line of tile column 0
      float ov[OP];
      auto prefetch_old = [&](int s0) {
#pragma unroll
        for (int j = 0; j < OP; ++j) {
          const int ts = oldidx[j] & 255, tl = oldidx[j] >> 8;
          const int s = s0 - 1 + ts, l = line0 + tl;
          const bool ok = oldidx[j] >= 0 && s >= 0 && s < S && l >= 0 && l < L;
          ov[j] = ok ? __ldcg(cur + gidx(dir, s, l, a.ny, a.nx)) : kInf;
        }
      };
      // records of block 0
      if (tid == Sh::PRODUCER) {
        fence_proxy_async();
        for (int t = 0; t < K; ++t) issue_row<K, EXT>(rec, plane, pl, mbar, arms, t, 0, S, L, l0, rev);
      }
      prefetch_old(0);
      for (int kb = 0; kb < nblk; ++kb, ++blk) {
        const int s0 = kb * K;
        const int t_end = min(K, S - s0);
        const bool more = kb + 1 < nblk;
        // 1. T before the sweep
#pragma unroll
        for (int j = 0; j < OP; ++j) {
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
        for (int tl = tid; tl < W; tl += NTH) {
          const int s = s0 - 1, l = line0 + tl;
          float v = kInf;
          if (s >= 0 && l >= 0 && l < L) {
            const bool halo_ok = (tl >= 1 && tl <= EXT);
            v = halo_ok ? __ldcg(nxt + gidx(dir, s, l, a.ny, a.nx)) : __ldcg(cur + gidx(dir, s, l, a.ny, a.nx));
          }
          nw[tl] = v;
        }
        for (int t = tid; t < K; t += NTH) {
          nw[(t + 1) * P] = old[(t + 1) * P];
          nw[(t + 1) * P + W - 1] = old[(t + 1) * P + W - 1];
        }
        __syncthreads();
        // 4. K line steps; after step t the producer arms row t of the next
        // block (its previous contents were last read in step t)
        bool bad = false;
        auto next_row = [&](int t) {
          if (tid == Sh::PRODUCER && more) {
            fence_proxy_async();
            issue_row<K, EXT>(rec, plane, pl, mbar, arms, t, s0 + K, S, L, l0, rev);
          }
        };
        const unsigned par = blk & 1u;
        const long long tmo = a.ctl.timeout_ns;
        switch (dir) {
          case 0: local_changed |= stream_steps<0, K, EXT>(pl, old, nw, mbar, par, t_end, l0, L, a.tol, a.rtol, tmo, bad, next_row); break;
          case 1: local_changed |= stream_steps<1, K, EXT>(pl, old, nw, mbar, par, t_end, l0, L, a.tol, a.rtol, tmo, bad, next_row); break;
          case 2: local_changed |= stream_steps<2, K, EXT>(pl, old, nw, mbar, par, t_end, l0, L, a.tol, a.rtol, tmo, bad, next_row); break;
          default: local_changed |= stream_steps<3, K, EXT>(pl, old, nw, mbar, par, t_end, l0, L, a.tol, a.rtol, tmo, bad, next_row); break;
        }
        if (__syncthreads_or(bad)) {
          if (tid == 0) raise_timeout(a.ctl);
          abort = true;
          break;
        }
        // 5. publish: first the block's last row (the only one the next
        // block reads), release it, then the other rows and the next
        // block's old T
        if (more) {
          for (int e = tid; e < R; e += NTH) {
            const int l = l0 + e;
            if (l < L) nxt[gidx(dir, s0 + K - 1, l, a.ny, a.nx)] = nw[K * P + K + 1 + e];
          }
        }
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          st_release_u32(&a.progress[b], base + kb + 1);
        }
        const int t_pub = more ? K - 1 : t_end;
        const int nwarps = NTH >> 5, warp = tid >> 5, lane = tid & 31;
        if (col) {
          for (int e = warp; e < R; e += nwarps) {
            const int l = l0 + e;
            for (int t = lane; t < t_pub; t += 32)
              if (l < L) nxt[gidx(dir, s0 + t, l, a.ny, a.nx)] = nw[(t + 1) * P + K + 1 + e];
          }
        } else {
          for (int t = warp; t < t_pub; t += nwarps) {
            for (int e = lane; e < R; e += 32) {
              const int l = l0 + e;
              if (l < L) nxt[gidx(dir, s0 + t, l, a.ny, a.nx)] = nw[(t + 1) * P + K + 1 + e];
            }
          }
        }
        if (more) prefetch_old(s0 + K);
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
  // record copies still in flight (only after an abort): wait for them
  // before the CTA's shared memory goes away.  The bound is fixed (1 s, far
  // above a copy's microseconds) so that a short or zero context timeout
  // cannot skip it.
  if (tid == Sh::PRODUCER) {
    for (int t = 0; t < K; ++t)
      if (arms[t] > 0) mbar_wait(&mbar[t], (unsigned)(arms[t] - 1) & 1u, 1000000000LL);
  }
  __syncthreads();
  // the latest values are in `cur`; hand them back in the caller's buffer
  if (cur != a.Ta) {
    for (long long p = (long long)blockIdx.x * NTH + tid; p < plane; p += (long long)gridDim.x * NTH)
      a.Ta[p] = __ldcg(cur + p);
  }
  if (b == 0 && tid == 0) {
    a.ctl.st->sweeps = sweep;
    a.ctl.st->converged = converged;
    a.ctl.st->cell_updates = (unsigned long long)sweep * (unsigned long long)plane;
    if (!converged && !abort) set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
  }
}

}  // namespace rf

using namespace rf;

namespace {

template <int K, int EXT>
rf_status plan_one(rf_ctx *ctx, int maxL, rf::StreamPlan *pl) {
  using Sh = StreamShape<K, EXT>;
  int dev_max_smem = 0;
  cudaDeviceGetAttribute(&dev_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  if ((long long)Sh::SMEM > dev_max_smem) return RF_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(sweep_stream_kernel<K, EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Sh::SMEM) != cudaSuccess)
    return RF_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_stream_kernel<K, EXT>, Sh::THREADS, Sh::SMEM) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  const int grid = (maxL + Sh::R - 1) / Sh::R;
  if (per_sm < 1 || grid > per_sm * ctx->num_sms) return RF_ERR_UNSUPPORTED;
  pl->R = Sh::R;
  pl->K = K;
  pl->grid = grid;
  pl->threads = Sh::THREADS;
  pl->smem = Sh::SMEM;
  pl->kernel = (const void *)sweep_stream_kernel<K, EXT>;
  return RF_OK;
}

}  // namespace

namespace rf {

// Shapes with a compiled kernel: (R, K) = (32, 32), (64, 16), (32, 16), (16, 16).
rf_status stream_plan(rf_ctx *ctx, int ny, int nx, int R, int K, StreamPlan *pl) {
  if (R <= 0) R = 32;
  if (K <= 0) K = 32;
  const int maxL = std::max(ny, nx);
  if (K >= 32 && R <= 32) return plan_one<32, 96>(ctx, maxL, pl);
  if (R >= 64) return plan_one<16, 96>(ctx, maxL, pl);
  if (R >= 32) return plan_one<16, 64>(ctx, maxL, pl);
  return plan_one<16, 48>(ctx, maxL, pl);
}

size_t stream_record_floats4(int ny, int nx) { return (size_t)2 * kPlanes * (size_t)ny * (size_t)nx; }

rf_status stream_records(int ny, int nx, float h, float eps, const float *proj5, const uint8_t *src, float4 *recbuf,
                         cudaStream_t s) {
  const long long n = (long long)ny * nx;
  dim3 block(kRecTile, kRecRows), grid((nx + kRecTile - 1) / kRecTile, (ny + kRecTile - 1) / kRecTile);
  records_kernel<<<grid, block, 0, s>>>(proj5, src, ny, nx, h, eps, recbuf, recbuf + (size_t)kPlanes * n);
  return cuda_status(cudaGetLastError());
}

rf_status stream_launch(const StreamPlan &pl, int ny, int nx, const float4 *recbuf, float *T, float *Tb,
                        int max_sweeps, float tol, float rtol, unsigned *progress, int *changed, const LaunchCtl &ctl,
                        cudaStream_t s) {
  const long long n = (long long)ny * nx;
  StreamArgs a;
  a.ny = ny;
  a.nx = nx;
  a.rec_row = recbuf;
  a.rec_col = recbuf + (size_t)kPlanes * n;
  a.Ta = T;
  a.Tb = Tb;
  a.max_sweeps = max_sweeps;
  a.tol = tol;
  a.rtol = rtol;
  a.tok_stride = (unsigned)((std::max(ny, nx) + pl.K - 1) / pl.K + 1);
  a.progress = progress;
  a.changed = changed;
  a.ctl = ctl;
  void *args[] = {&a};
  return cuda_status(
      cudaLaunchCooperativeKernel(pl.kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, s));
}

}  // namespace rf
