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

// Weight with which child q (record id, w1) passes lambda to the neighbour in
// direction `back` (the direction from q to that neighbour); 0 if none.
__device__ __forceinline__ float child_weight(uint8_t id, float w1, int back) {
  const int k = id & 7;
  if (id & 0x10) return (k == back) ? 1.0f : 0.0f;
  if (id & 0x20) return (k == back) ? w1 : ((((k + 1) & 7) == back) ? 1.0f - w1 : 0.0f);
  return 0.0f;
}

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
        const int rows = K + 2;
        for (int f = tid; f < rows * W; f += nth) {
          int ts, tl;
          if (col) { tl = f / rows; ts = f - tl * rows; }
          else     { ts = f / W;    tl = f - ts * W; }
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
        for (int tl = tid; tl < W; tl += nth) {
          const int s = s0 - 1, l = line0 + tl;
          float v = 0.0f;
          if (s >= 0 && l >= 0 && l < L) {
            const long long gi = gidx(dir, s, l, a.ny, a.nx);
            v = (tl >= 1 && tl <= ext) ? __ldcg(nxt + gi) : __ldcg(cur + gi);
          }
          nw[tl] = v;
        }
        for (int f = tid; f < K * ext; f += nth) {
          int t, e;
          if (col) { e = f / K; t = f - e * K; }
          else     { t = f / ext; e = f - t * ext; }
          const int s = s0 + t, l = l0 - K + e;
          float v = 0.0f;
          if (s < S && l >= 0 && l < L) {
            const long long gi = gidx(dir, s, l, a.ny, a.nx);
            v = (__ldg(a.T + gi) < kInf) ? __ldg(a.g + gi) : 0.0f;
          }
          gg[t * EP + e] = v;
        }
        __syncthreads();
        for (int t = tid; t < K; t += nth) {
          nw[(t + 1) * P] = old[(t + 1) * P];
          nw[(t + 1) * P + W - 1] = old[(t + 1) * P + W - 1];
        }
        for (int t = 0; t < K; ++t) {
          const int s = s0 + t;
          if (s >= S) break;
          if (tid < ext) {
            const int e = tid, tl = e + 1, l = l0 - K + e;
            float lnew = 0.0f;
            if (l >= 0 && l < L) {
              const float lold = old[(t + 1) * P + tl];
              float acc = gg[t * EP + e];
#pragma unroll
              for (int n = 0; n < 8; ++n) {
                int ds, dl;
                nb_tile_offset(dir, n, ds, dl);
                const int r = t + 1 + ds, cidx = tl + dl;
                const float wq = child_weight(ids[r * P + cidx], ww[r * P + cidx], (n + 4) & 7);
                if (wq != 0.0f) {
                  const float lq = (ds < 0) ? nw[t * P + cidx] : old[r * P + cidx];
                  acc = fmaf(wq, lq, acc);
                }
              }
              lnew = acc;
              if (e >= K && e < K + R) local_changed |= (__float_as_uint(lnew) != __float_as_uint(lold));
            }
            nw[(t + 1) * P + tl] = lnew;
          }
          __syncthreads();
        }
        for (int f = tid; f < K * R; f += nth) {
          int t, e;
          if (col) { e = f / K; t = f - e * K; }
          else     { t = f / R; e = f - t * R; }
          const int s = s0 + t, l = l0 + e;
          if (s < S && l < L) nxt[gidx(dir, s, l, a.ny, a.nx)] = nw[(t + 1) * P + K + 1 + e];
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

}  // namespace rf

using namespace rf;

extern "C" rf_status rf_adjoint(rf_ctx *ctx, const rf_grid *grid, const uint8_t *src, const float *T,
                                const rf_record *rec, const float *dLdT, float *dLdproj5, float *lambda,
                                int algo, void *stream) {
  if (!ctx || !grid_ok(grid) || !src || !T || !rec || !rec->id || !rec->w1 || !rec->dT || !dLdT ||
      !dLdproj5)
    return RF_ERR_INVALID_ARG;
  if (algo != RF_ADJ_SWEEP) return RF_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
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
    threads = ((R + 2 * K + 31) / 32) * 32;
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
  cudaMemsetAsync(&ctx->state->bar_count, 0, sizeof(unsigned) * 2, s);
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
