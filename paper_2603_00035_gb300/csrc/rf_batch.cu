// rf_batch.cu -- a10: many grids of uneven size and source count solved
// forward + record + adjoint.
//
// Two paths.  The default (variant AUTO or TILES) puts every grid's tiles in
// one tile queue (rf_sweep_tiles.cu), so a large grid spreads over all SMs
// while small ones finish in a few rounds, then records the stencils of all
// grids in one pass and runs the tiled adjoint over the packed grids
// (rf_adjoint_tiles.cu: 16 x 16 tiles handed out a few grids at a time; a
// node's children are in its own grid).  The line-sweep variants use the
// single persistent launch below.
//
// Paper: the batched solves of Sec. 3.4 ("batched approach proves
// essential"), with the same discrete system as rf_sweep_forward / rf_adjoint
// (Sec. 3.2, Alg. 1; Sec. 3.3, Alg. 2).
//
// GB300 mapping.  CTAs take whole grids from an atomic work counter (the
// caller orders the descriptors largest first, so long solves start early).
// A CTA owns its grid alone, so there are no waits between CTAs at all, and
// its SM's L1 sees every write to the grid (T and lambda are updated in
// place).  A sweep keeps three lines in shared memory -- this sweep's step
// s-1 and the pre-sweep steps s, s+1 -- and prefetches step s+2 and the
// fields of step s+1 into registers while step s is computed; each thread
// owns up to kBCells nodes of the front.  After the forward converges the
// CTA records the stencils of its grid and, when dL/dT is given, runs the
// transposed sweeps for lambda with the same rolling lines, then writes the
// parameter gradients.
#include <algorithm>

#include "rf_adjoint.h"
#include "rf_cone.cuh"
#include "rf_ctx.h"
#include "rf_sweep_common.cuh"
#include "rf_sweep_tiles.h"

namespace rf {

constexpr int kBThreads = 512;
constexpr int kBCells = 2;  // front nodes per thread: lines up to 1024

struct BatchArgs {
  const rf_batch_desc *descs;
  int n_grids;
  long long total;  // plane stride of the packed arrays
  int max_line;
  const float *f;  // 5 planes
  float eps;
  const uint8_t *src;
  float *T;
  uint8_t *id;
  float *w1;
  float *dT;  // 5 planes
  const float *g;  // nullable: no adjoint
  float *lam;      // lambda (in place), workspace
  float *grad;     // 5 planes
  int max_sweeps, max_adj_sweeps, warm;
  float tol, rtol;
  int *gstat;  // nullable: [3 * n_grids] status, sweeps, adjoint sweeps
  unsigned *counter;
  DevState *st;
};

__host__ __device__ inline size_t batch_smem_bytes(int max_line) {
  const size_t W = (size_t)max_line + 2;
  return 5 * W * sizeof(float) + 4 * W * sizeof(float) + 4 * W;
}

__global__ void __launch_bounds__(kBThreads, 1) batch_kernel(BatchArgs a) {
  extern __shared__ float smem[];
  const int W = a.max_line + 2;
  float *rows[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) rows[r] = smem + (size_t)r * W;
  float *wrow[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) wrow[r] = smem + (size_t)(5 + r) * W;
  uint8_t *irow[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) irow[r] = (uint8_t *)(smem + (size_t)9 * W) + (size_t)r * W;
  __shared__ int s_grid;
  const int tid = threadIdx.x, nth = blockDim.x;

  while (true) {
    if (tid == 0) s_grid = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int gi = s_grid;
    __syncthreads();
    if (gi >= a.n_grids) break;
    const rf_batch_desc d = a.descs[gi];
    const int ny = d.ny, nx = d.nx;
    const long long n = (long long)ny * nx;
    const float h = d.h;
    if (ny < 1 || nx < 1 || ny > a.max_line || nx > a.max_line || !(h > 0.0f)) {
      if (tid == 0 && a.gstat) a.gstat[3 * gi] = RF_ERR_INVALID_ARG;
      continue;
    }
    float *Tg = a.T + d.offset;
    const float *fg = a.f + d.offset;
    const uint8_t *sg = a.src + d.offset;

    // ---- init (a2) -------------------------------------------------------
    int any_src = 0;
    for (long long p = tid; p < n; p += nth) {
      const bool s = sg[p] != 0;
      any_src |= s;
      if (s) Tg[p] = 0.0f;
      else if (!a.warm) Tg[p] = kInf;
    }
    any_src = __syncthreads_or(any_src);

    // ---- forward line sweeps (a3, a4) --------------------------------------
    int sweep = 0, converged = 0;
    while (any_src) {
      const int dir = sweep & 3;
      const bool col = (dir & 1) == 0;
      const int S = col ? nx : ny, L = col ? ny : nx;
      float *P = rows[0], *C = rows[1], *N = rows[2], *O = rows[3], *X = rows[4];
      for (int l = tid; l < W; l += nth) {
        const int gl = l - 1;
        const bool in = gl >= 0 && gl < L;
        P[l] = kInf;
        O[l] = kInf;
        X[l] = kInf;
        C[l] = in ? Tg[gidx(dir, 0, gl, ny, nx)] : kInf;
        N[l] = (in && S > 1) ? Tg[gidx(dir, 1, gl, ny, nx)] : kInf;
      }
      float fv[kBCells][5];
      uint8_t sv[kBCells];
#pragma unroll
      for (int k = 0; k < kBCells; ++k) {
        const int l = tid + k * nth;
        const bool ok = l < L;
        const long long gp = ok ? gidx(dir, 0, l, ny, nx) : 0;
#pragma unroll
        for (int c = 0; c < 5; ++c) fv[k][c] = ok ? fg[c * a.total + gp] : 1.0f;
        sv[k] = ok ? sg[gp] : 0;
      }
      __syncthreads();
      int changed = 0;
      for (int s = 0; s < S; ++s) {
        // prefetch step s+1's fields and the pre-sweep values of step s+2
        float fn[kBCells][5], xo[kBCells];
        uint8_t sn[kBCells];
#pragma unroll
        for (int k = 0; k < kBCells; ++k) {
          const int l = tid + k * nth;
          const bool ok1 = l < L && s + 1 < S;
          const long long g1 = ok1 ? gidx(dir, s + 1, l, ny, nx) : 0;
#pragma unroll
          for (int c = 0; c < 5; ++c) fn[k][c] = ok1 ? fg[c * a.total + g1] : 1.0f;
          sn[k] = ok1 ? sg[g1] : 0;
          const bool ok2 = l < L && s + 2 < S;
          xo[k] = ok2 ? Tg[gidx(dir, s + 2, l, ny, nx)] : kInf;
        }
        // step s: every node of the line from P (step s-1, this sweep),
        // C (step s) and N (step s+1), both as before the sweep
#pragma unroll
        for (int k = 0; k < kBCells; ++k) {
          const int l = tid + k * nth;
          if (l < L) {
            const float told = C[l + 1];
            float tnew;
            if (sv[k]) {
              tnew = 0.0f;
            } else {
              float Tn[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                int ds, dl;
                nb_tile_offset(dir, q, ds, dl);
                const float *row = ds < 0 ? P : (ds == 0 ? C : N);
                Tn[q] = row[l + 1 + dl];
              }
              float tab[kTabSize];
              node_tab(fv[k][0], fv[k][1], fv[k][2], fv[k][3], fv[k][4], h, a.eps, tab);
              tnew = winner(tab, Tn).value;
            }
            O[l + 1] = tnew;
            changed |= node_changed(tnew, told, a.tol, a.rtol);
            Tg[gidx(dir, s, l, ny, nx)] = tnew;
          }
        }
#pragma unroll
        for (int k = 0; k < kBCells; ++k) {
          const int l = tid + k * nth;
          if (l < L) X[l + 1] = xo[k];
#pragma unroll
          for (int c = 0; c < 5; ++c) fv[k][c] = fn[k][c];
          sv[k] = sn[k];
        }
        __syncthreads();
        // (P, C, N, O, X) <- (O, N, X, P, C)
        float *t0 = P, *t1 = C;
        P = O;
        C = N;
        N = X;
        O = t0;
        X = t1;
      }
      changed = __syncthreads_or(changed);
      ++sweep;
      if (!changed) {
        converged = 1;
        break;
      }
      if (sweep >= a.max_sweeps) break;
    }

    // ---- record (a5) --------------------------------------------------------
    for (long long p = tid; p < n; p += nth) {
      const int i = (int)(p / nx), j = (int)(p - (long long)i * nx);
      uint8_t id;
      float w1, dd[5], r;
      record_node_cone(fg, a.total, p, i, j, ny, nx, h, a.eps, sg[p] != 0, Tg, true, id, w1, dd, r);
      a.id[d.offset + p] = id;
      a.w1[d.offset + p] = w1;
#pragma unroll
      for (int c = 0; c < 5; ++c) a.dT[c * a.total + d.offset + p] = dd[c];
    }
    __syncthreads();

    // ---- adjoint (a7, a8): transposed line sweeps, in place -------------------
    int asweep = 0, aconv = 1;
    if (a.g) {
      float *Lg = a.lam + d.offset;
      const uint8_t *ig = a.id + d.offset;
      const float *wg = a.w1 + d.offset;
      const float *gg = a.g + d.offset;
      for (long long p = tid; p < n; p += nth) Lg[p] = 0.0f;
      __syncthreads();
      aconv = 0;
      while (true) {
        const int dir = asweep & 3;
        const bool col = (dir & 1) == 0;
        const int S = col ? nx : ny, L = col ? ny : nx;
        float *P = rows[0], *C = rows[1], *N = rows[2], *O = rows[3], *X = rows[4];
        float *WP = wrow[0], *WC = wrow[1], *WN = wrow[2], *WX = wrow[3];
        uint8_t *IP = irow[0], *IC = irow[1], *IN = irow[2], *IX = irow[3];
        for (int l = tid; l < W; l += nth) {
          const int gl = l - 1;
          const bool in = gl >= 0 && gl < L;
          P[l] = 0.0f;
          O[l] = 0.0f;
          X[l] = 0.0f;
          WP[l] = 0.0f;
          IP[l] = 0;
          WX[l] = 0.0f;
          IX[l] = 0;
          const long long g0 = in ? gidx(dir, 0, gl, ny, nx) : 0;
          const long long g1 = (in && S > 1) ? gidx(dir, 1, gl, ny, nx) : 0;
          C[l] = in ? Lg[g0] : 0.0f;
          WC[l] = in ? wg[g0] : 0.0f;
          IC[l] = in ? ig[g0] : 0;
          N[l] = (in && S > 1) ? Lg[g1] : 0.0f;
          WN[l] = (in && S > 1) ? wg[g1] : 0.0f;
          IN[l] = (in && S > 1) ? ig[g1] : 0;
        }
        float gv[kBCells];
#pragma unroll
        for (int k = 0; k < kBCells; ++k) {
          const int l = tid + k * nth;
          const long long gp = l < L ? gidx(dir, 0, l, ny, nx) : 0;
          gv[k] = (l < L && Tg[gp] < kInf) ? gg[gp] : 0.0f;
        }
        __syncthreads();
        int changed = 0;
        for (int s = 0; s < S; ++s) {
          float gn[kBCells], xl[kBCells], xw[kBCells];
          uint8_t xi[kBCells];
#pragma unroll
          for (int k = 0; k < kBCells; ++k) {
            const int l = tid + k * nth;
            const bool ok1 = l < L && s + 1 < S;
            const long long g1 = ok1 ? gidx(dir, s + 1, l, ny, nx) : 0;
            gn[k] = (ok1 && Tg[g1] < kInf) ? gg[g1] : 0.0f;
            const bool ok2 = l < L && s + 2 < S;
            const long long g2 = ok2 ? gidx(dir, s + 2, l, ny, nx) : 0;
            xl[k] = ok2 ? Lg[g2] : 0.0f;
            xw[k] = ok2 ? wg[g2] : 0.0f;
            xi[k] = ok2 ? ig[g2] : 0;
          }
#pragma unroll
          for (int k = 0; k < kBCells; ++k) {
            const int l = tid + k * nth;
            if (l < L) {
              const float lold = C[l + 1];
              float acc = gv[k];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                int ds, dl;
                nb_tile_offset(dir, q, ds, dl);
                const int c = l + 1 + dl;
                const float wq = child_weight(ds < 0 ? IP[c] : (ds == 0 ? IC[c] : IN[c]),
                                              ds < 0 ? WP[c] : (ds == 0 ? WC[c] : WN[c]), (q + 4) & 7);
                if (wq != 0.0f) acc = fmaf(wq, ds < 0 ? P[c] : (ds == 0 ? C[c] : N[c]), acc);
              }
              O[l + 1] = acc;
              changed |= (__float_as_uint(acc) != __float_as_uint(lold));
              Lg[gidx(dir, s, l, ny, nx)] = acc;
            }
          }
#pragma unroll
          for (int k = 0; k < kBCells; ++k) {
            const int l = tid + k * nth;
            if (l < L) {
              X[l + 1] = xl[k];
              WX[l + 1] = xw[k];
              IX[l + 1] = xi[k];
            }
            gv[k] = gn[k];
          }
          __syncthreads();
          float *t0 = P, *t1 = C;
          P = O;
          C = N;
          N = X;
          O = t0;
          X = t1;
          float *u0 = WP;
          WP = WC;
          WC = WN;
          WN = WX;
          WX = u0;
          uint8_t *v0 = IP;
          IP = IC;
          IC = IN;
          IN = IX;
          IX = v0;
        }
        changed = __syncthreads_or(changed);
        ++asweep;
        if (!changed) {
          aconv = 1;
          break;
        }
        if (asweep >= a.max_adj_sweeps) break;
      }
      // a8: parameter gradients
      for (long long p = tid; p < n; p += nth) {
        const bool act = ig[p] != 0 && !sg[p];
        const float lam = Lg[p];
#pragma unroll
        for (int c = 0; c < 5; ++c)
          a.grad[c * a.total + d.offset + p] = act ? lam * a.dT[c * a.total + d.offset + p] : 0.0f;
      }
    }
    if (tid == 0) {
      const int stc = !any_src ? RF_ERR_NO_SOURCE : (!converged || !aconv) ? RF_ERR_NOT_CONVERGED : RF_OK;
      if (a.gstat) {
        a.gstat[3 * gi] = stc;
        a.gstat[3 * gi + 1] = sweep;
        a.gstat[3 * gi + 2] = asweep;
      }
      if (stc != RF_OK) set_error(a.st, stc);
      atomicAdd(&a.st->cell_updates, (unsigned long long)sweep * (unsigned long long)n);
    }
    __syncthreads();
  }
}

// a5 for packed grids (blockIdx.y = grid): stencil ids, donor weights and
// partials of every node at the converged T (cone form, as the tile queue
// that solved them), and the max residual.
__global__ void __launch_bounds__(256) batch_record_kernel(const TGrid *grids, long long total, const float *f,
                                                           float eps, const uint8_t *src, const float *T,
                                                           uint8_t *id, float *w1, float *dT, DevState *st) {
  const TGrid g = grids[blockIdx.y];
  const long long n = (long long)g.ny * g.nx;
  float local_max = 0.0f;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / g.nx), j = (int)(q - (long long)i * g.nx);
    const long long p = g.node_off + q;
    uint8_t idv;
    float w1v, d[5], r;
    record_node_cone(f + g.node_off, total, q, i, j, g.ny, g.nx, g.h, eps, src[p] != 0, T + g.node_off, true, idv,
                w1v, d, r);
    id[p] = idv;
    w1[p] = w1v;
#pragma unroll
    for (int c = 0; c < 5; ++c) dT[c * total + p] = d[c];
    local_max = fmaxf(local_max, fabsf(r));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&st->max_res_bits, __float_as_uint(local_max));
}

// Adjoint column of the per-grid status (the tiled adjoint has no sweeps).
__global__ void batch_adj_status_kernel(int *gstat, int n_grids) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_grids; g += gridDim.x * blockDim.x)
    gstat[3 * g + 2] = 0;
}

}  // namespace rf

using namespace rf;

namespace {

// The tile-queue path of rf_batch_solve (see the file comment).
rf_status batch_tiles(rf_ctx *ctx, const rf_batch_desc *descs, int n_grids, int64_t total_nodes, int32_t max_line,
                      const float *proj5, float eps, const uint8_t *src, const rf_opts &o, float *T,
                      rf_record *rec, const float *dLdT, float *dLdproj5, int32_t *grid_status, cudaStream_t s) {
  const int ts = rf::tile_side(o.variant == RF_SWEEP_TILES ? o.band : 0);
  const int ncap = rf::tiles_cap(n_grids, total_nodes, max_line, ts);
  rf_status rs;
  if ((rs = ensure(&ctx->tilebuf, &ctx->tilebuf_cap, rf::tile_work_bytes(n_grids, ncap, ts))) != RF_OK) return rs;
  if ((rs = ensure(&ctx->tbuf, &ctx->tbuf_cap, (size_t)total_nodes)) != RF_OK) return rs;
  if ((rs = ensure(&ctx->changed, &ctx->changed_cap, (size_t)o.max_sweeps + 2)) != RF_OK) return rs;
  cudaMemsetAsync(ctx->changed, 0, sizeof(int) * (o.max_sweeps + 2), s);
  cudaMemsetAsync(&ctx->state->sweeps, 0, sizeof(int) * 2, s);
  cudaMemsetAsync(&ctx->state->bar, 0, sizeof(unsigned long long) + 2 * sizeof(unsigned), s);
  cudaMemsetAsync(&ctx->state->cell_updates, 0, sizeof(unsigned long long), s);
  int *has_src = ctx->changed + o.max_sweeps;  // per-grid sources are checked by the seed kernel
  rf::init_state(T, src, total_nodes, o.mode == RF_MODE_WARM, ctx->state, has_src, ctx->num_sms, s);
  LaunchCtl ctl;
  ctl.st = ctx->state;
  ctl.abort = ctx->changed + o.max_sweeps + 1;
  ctl.timeout_ns = ctx->timeout_ns;
  const rf::TileWork w = rf::tile_work_carve(ctx->tilebuf, n_grids, ncap, ts);
  rf::TileLaunch L;
  L.num_sms = ctx->num_sms;
  L.ts = ts;
  L.n_grids = n_grids;
  L.descs = descs;
  L.ny = L.nx = 0;
  L.h = 0.0f;
  L.max_line = max_line;
  L.total_nodes = total_nodes;
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
  L.grid_status = grid_status;
  if ((rs = rf::tiles_launch(L, w, ctl, s)) != RF_OK) return rs;
  cudaMemsetAsync(&ctx->state->max_res_bits, 0, sizeof(unsigned), s);
  const long long per_grid = std::max<long long>(1, total_nodes / n_grids);
  const int gx = std::max(1, std::min(blocks_for(per_grid, 256, ctx->num_sms * 8), 65535));
  batch_record_kernel<<<dim3(gx, n_grids), 256, 0, s>>>(w.grids, total_nodes, proj5, eps, src, T, rec->id, rec->w1,
                                                        rec->dT, ctx->state);
  if ((rs = cuda_status(cudaGetLastError())) != RF_OK) return rs;
  if (grid_status) batch_adj_status_kernel<<<blocks_for(n_grids, 256, 64), 256, 0, s>>>(grid_status, n_grids);
  if (!dLdT) return cuda_status(cudaGetLastError());
  return rf::adjoint_tiles_packed(ctx, total_nodes, w.grids, n_grids, max_line, src, T, rec, dLdT, dLdproj5, nullptr,
                                  s);
}

}  // namespace

extern "C" rf_status rf_batch_solve(rf_ctx *ctx, const rf_batch_desc *descs, int n_grids, int64_t total_nodes,
                                    int32_t max_line, const float *proj5, float eps, const uint8_t *src,
                                    const rf_opts *opts, float *T, rf_record *rec, const float *dLdT,
                                    float *dLdproj5, int32_t *grid_status, void *stream) {
  if (!ctx || !descs || n_grids < 1 || total_nodes < 1 || !proj5 || !src || !T || !rec || !rec->id || !rec->w1 ||
      !rec->dT)
    return RF_ERR_INVALID_ARG;
  if (max_line < 1 || !(eps >= 0.0f)) return RF_ERR_INVALID_ARG;
  if (dLdT && !dLdproj5) return RF_ERR_INVALID_ARG;
  rf_opts o = {0.0f, 64, RF_MODE_COLD, 0, 0, 1e-6f, 0, 0.0f};
  if (opts) o = *opts;
  if (o.max_sweeps < 1 || !(o.tol >= 0.0f) || !(o.rtol >= 0.0f) || (o.mode != RF_MODE_COLD && o.mode != RF_MODE_WARM) ||
      !(o.window >= 0.0f))
    return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  if (o.variant == RF_SWEEP_AUTO || o.variant == RF_SWEEP_TILES) {
    // launch-grid limits of the per-grid kernels and the 32-bit sort
    if (n_grids > 65535 || total_nodes >= (1LL << 31)) return RF_ERR_INVALID_ARG;
    return batch_tiles(ctx, descs, n_grids, total_nodes, max_line, proj5, eps, src, o, T, rec, dLdT, dLdproj5,
                       grid_status, s);
  }
  // the persistent kernel keeps whole lines of a grid in shared memory
  if (max_line > kBThreads * kBCells) return RF_ERR_INVALID_ARG;
  rf_status rs;
  if (dLdT && (rs = ensure(&ctx->lbuf, &ctx->lbuf_cap, (size_t)total_nodes)) != RF_OK) return rs;
  if ((rs = ensure(&ctx->changed, &ctx->changed_cap, (size_t)2)) != RF_OK) return rs;
  const size_t smem = batch_smem_bytes(max_line);
  if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return RF_ERR_UNSUPPORTED;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBThreads, smem) != cudaSuccess ||
      per_sm < 1)
    return RF_ERR_UNSUPPORTED;
  cudaMemsetAsync(ctx->changed, 0, sizeof(int), s);  // work counter
  cudaMemsetAsync(&ctx->state->cell_updates, 0, sizeof(unsigned long long), s);
  BatchArgs a;
  a.descs = descs;
  a.n_grids = n_grids;
  a.total = total_nodes;
  a.max_line = max_line;
  a.f = proj5;
  a.eps = eps;
  a.src = src;
  a.T = T;
  a.id = rec->id;
  a.w1 = rec->w1;
  a.dT = rec->dT;
  a.g = dLdT;
  a.lam = ctx->lbuf;
  a.grad = dLdproj5;
  a.max_sweeps = o.max_sweeps;
  a.max_adj_sweeps = 4 * o.max_sweeps;
  a.warm = o.mode == RF_MODE_WARM;
  a.tol = o.tol;
  a.rtol = o.rtol;
  a.gstat = grid_status;
  a.counter = (unsigned *)ctx->changed;
  a.st = ctx->state;
  const int grid = std::min(per_sm * ctx->num_sms, n_grids);
  batch_kernel<<<grid, kBThreads, smem, s>>>(a);
  return cuda_status(cudaGetLastError());
}
