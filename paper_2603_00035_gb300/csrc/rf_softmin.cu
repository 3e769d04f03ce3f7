// rf_softmin.cu -- NEXT-4: the soft-min relaxation of the stencil selection.
//
// Sec. 3.3 ("Stencil Boundaries and Non-Smoothness") names soft-min
// relaxations as an alternative to the hard minimum over the stencils,
// without a formula.  The reading implemented here: every one of a node's 8
// stencils k (donors k, k+1) has the value of the minimum of its segment --
// the two-point candidate when it is valid (App. A), else the smaller
// one-point candidate of its finite endpoints -- and the node takes
//     T = -tau log sum_k exp(-c_k / tau) = c_min - tau log sum_k exp(-(c_k - c_min) / tau),
// a smooth minimum that tends to the hard one as tau -> 0 (a sum over the
// individual candidates would jump wherever a two-point update turns valid
// next to the one-point update it equals).  The relaxed system is solved by
// Jacobi iterations over the whole grid in one persistent launch; its
// stencil record holds, per node, the derivative of T with respect to each
// neighbour (the softmax weights times the candidates' donor weights) and to
// the five parameters; the adjoint iterates lambda = g + W^T lambda.
//
// A soft value lies up to tau log 8 below its candidate minimum, so a large
// tau can pull a node below its own donors and the values then run to -inf
// (no finite fixed point): a non-source node going negative ends the solve
// with RF_ERR_NOT_CONVERGED.
#include <algorithm>

#include "rf_ctx.h"
#include "rf_sweep_common.cuh"
#include "rf_sweep_tiles.h"

namespace rf {

// Stencil values of a node (tab: node table; Tn: neighbour times), and for
// each the candidate behind it: from[k] = 8 + k two-point, n one-point via
// neighbour n, -1 none; l1, l2 of the two-point candidates.
struct SoftCands {
  float v[8];
  int from[8];
  float l1[8], l2[8];
};

__device__ __forceinline__ void soft_cands(const float tab[kTabSize], const float Tn[8], SoftCands &c) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int a = k, b = (k + 1) & 7;
    float l1, l2;
    const float t2 = two_point(tab, k, Tn[a], Tn[b], l1, l2);
    c.l1[k] = l1;
    c.l2[k] = l2;
    if (t2 < kInf) {
      c.v[k] = t2;
      c.from[k] = 8 + k;
    } else {
      const float oa = one_point(tab, a, Tn[a]), ob = one_point(tab, b, Tn[b]);
      c.v[k] = fminf(oa, ob);
      c.from[k] = (oa < kInf || ob < kInf) ? (oa <= ob ? a : b) : -1;
    }
  }
}

// Soft minimum of the stencil values; p[k] = softmax weights (sum 1).
__device__ __forceinline__ float soft_min(const float v[8], float tau, float p[8]) {
  float cmin = kInf;
#pragma unroll
  for (int k = 0; k < 8; ++k) cmin = fminf(cmin, v[k]);
  if (!(cmin < kInf)) {
#pragma unroll
    for (int k = 0; k < 8; ++k) p[k] = 0.0f;
    return kInf;
  }
  if (!(tau > 0.0f)) {
    bool set = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      p[k] = (!set && v[k] == cmin) ? 1.0f : 0.0f;
      set |= v[k] == cmin;
    }
    return cmin;
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    p[k] = (v[k] < kInf) ? expf((cmin - v[k]) / tau) : 0.0f;
    s += p[k];
  }
  const float inv = 1.0f / s;
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] *= inv;
  return cmin - tau * logf(s);
}

__device__ __forceinline__ void gather8(const float *T, int i, int j, int ny, int nx, float Tn[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int ii = i + nb_dy(q), jj = j + nb_dx(q);
    Tn[q] = (ii >= 0 && ii < ny && jj >= 0 && jj < nx) ? __ldcg(T + (long long)ii * nx + jj) : kInf;
  }
}

struct SoftArgs {
  int ny, nx;
  float h, eps, tau;
  const float *f;
  const uint8_t *src;
  float *Ta, *Tb;  // Ta = caller's T (initial state), Tb = workspace
  int max_iter;
  float tol, rtol;
  int *changed;    // [3] change flags by iteration mod 3, [3] a value went negative
  LaunchCtl ctl;
};

// Jacobi iterations of T = softmin(stencil values(T)) until an iteration
// changes no node by more than tol + rtol |T|; one grid barrier per
// iteration.
__global__ void __launch_bounds__(256) softmin_solve_kernel(SoftArgs a) {
  const long long n = (long long)a.ny * a.nx;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float *cur = a.Ta, *nxt = a.Tb;
  int it = 0;
  bool converged = false, abort = false;
  for (; it < a.max_iter; ++it) {
    int changed = 0, negative = 0;
    for (long long p = g0; p < n; p += stride) {
      const float told = __ldcg(cur + p);
      float tnew = told;
      if (!a.src[p]) {
        const int i = (int)(p / a.nx), j = (int)(p - (long long)i * a.nx);
        float Tn[8], tab[kTabSize], pk[8];
        gather8(cur, i, j, a.ny, a.nx, Tn);
        node_tab(__ldg(a.f + p), __ldg(a.f + n + p), __ldg(a.f + 2 * n + p), __ldg(a.f + 3 * n + p),
                 __ldg(a.f + 4 * n + p), a.h, a.eps, tab);
        SoftCands c;
        soft_cands(tab, Tn, c);
        tnew = soft_min(c.v, a.tau, pk);
        changed |= node_changed(tnew, told, a.tol, a.rtol);
        negative |= tnew < 0.0f;
      }
      __stcg(nxt + p, tnew);
    }
    // the slot of iteration it + 1 last held iteration it - 2's flag, which
    // every CTA read before the barrier of iteration it - 1
    if (blockIdx.x == 0 && threadIdx.x == 0) a.changed[(it + 1) % 3] = 0;
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&a.changed[it % 3], 1);
    if (__syncthreads_or(negative) && threadIdx.x == 0) atomicOr(&a.changed[3], 1);
    if (!grid_sync(a.ctl)) {
      abort = true;
      break;
    }
    float *t = cur;
    cur = nxt;
    nxt = t;
    if (ld_acquire_s32(&a.changed[3])) break;  // values below 0: no finite fixed point
    if (!ld_acquire_s32(&a.changed[it % 3])) {
      converged = true;
      ++it;
      break;
    }
  }
  // hand the latest values back in the caller's buffer
  if (!abort && cur != a.Ta)
    for (long long p = g0; p < n; p += stride) a.Ta[p] = __ldcg(cur + p);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl.st->sweeps = it;
    a.ctl.st->converged = converged ? 1 : 0;
    a.ctl.st->cell_updates = (unsigned long long)it * (unsigned long long)n;
    if (!converged && !abort) set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
  }
}

// Record of the relaxed system at T: wnb[nb * n + p] = dT_p / dT_(neighbour
// nb), dT[c * n + p] = dT_p / d(L11, L21, L22, wx, wy).  For a candidate with
// barycentric weights (w1, 1 - w1) the characteristic displacement is
// v = w1 m1 + (1 - w1) m2 (v = m_n for a one-point candidate) and
//   dc/dw = -v,  dc/dM = v v^T / (2 |v|_M),  dc/dL = 2 (dc/dM) L;
// the node's derivatives are the softmax-weighted sums over its stencils.
__global__ void __launch_bounds__(256) softmin_record_kernel(int ny, int nx, float h, float eps, float tau,
                                                             const float *f, const uint8_t *src, const float *T,
                                                             float *wnb, float *dT) {
  const long long n = (long long)ny * nx;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float d[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const float t0 = T[p];
    if (!src[p] && t0 < kInf) {
      const int i = (int)(p / nx), j = (int)(p - (long long)i * nx);
      float Tn[8], tab[kTabSize], pk[8];
      gather8(T, i, j, ny, nx, Tn);
      const float l11 = f[p], l21 = f[n + p], l22 = f[2 * n + p];
      node_tab(l11, l21, l22, f[3 * n + p], f[4 * n + p], h, eps, tab);
      SoftCands c;
      soft_cands(tab, Tn, c);
      soft_min(c.v, tau, pk);
      const float m11 = fmaf(l11, l11, eps), m12 = l11 * l21, m22 = fmaf(l21, l21, fmaf(l22, l22, eps));
      float D11 = 0.f, D12 = 0.f, D22 = 0.f, vwx = 0.f, vwy = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (!(pk[k] > 0.0f) || c.from[k] < 0) continue;
        float vx, vy;
        if (c.from[k] >= 8) {
          const int k2 = (k + 1) & 7;
          const float sum = c.l1[k] + c.l2[k];
          const float w1 = sum > 0.0f ? c.l1[k] / sum : 0.5f;
          w[k] += pk[k] * w1;
          w[k2] += pk[k] * (1.0f - w1);
          vx = h * (w1 * (float)nb_dx(k) + (1.0f - w1) * (float)nb_dx(k2));
          vy = h * (w1 * (float)nb_dy(k) + (1.0f - w1) * (float)nb_dy(k2));
        } else {
          const int nb = c.from[k];
          w[nb] += pk[k];
          vx = h * (float)nb_dx(nb);
          vy = h * (float)nb_dy(nb);
        }
        const float vm = sqrtf(vx * (m11 * vx + m12 * vy) + vy * (m12 * vx + m22 * vy));
        const float s = pk[k] * 0.5f / vm;
        D11 = fmaf(s * vx, vx, D11);
        D12 = fmaf(s * vx, vy, D12);
        D22 = fmaf(s * vy, vy, D22);
        vwx = fmaf(pk[k], vx, vwx);
        vwy = fmaf(pk[k], vy, vwy);
      }
      d[0] = 2.0f * (D11 * l11 + D12 * l21);
      d[1] = 2.0f * (D12 * l11 + D22 * l21);
      d[2] = 2.0f * D22 * l22;
      d[3] = -vwx;
      d[4] = -vwy;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) wnb[k * n + p] = w[k];
#pragma unroll
    for (int c = 0; c < 5; ++c) dT[c * n + p] = d[c];
  }
}

struct SoftAdjArgs {
  int ny, nx;
  const uint8_t *src;
  const float *T, *wnb, *dT, *g;
  float *La, *Lb;   // lambda ping-pong (La zeroed by the host)
  float *grad, *lam_out;
  int max_iter;
  int *flags;       // [3] change flags by iteration mod 3
  LaunchCtl ctl;
};

// lambda_p = g_p + sum over neighbours q of wnb_q(q -> p) lambda_q, iterated
// until no multiplier changes by more than 1e-7 relative between two grid
// barriers, then dL/dtheta_p = lambda_p dT_p.  Block Jacobi: between two
// grid barriers each 16 x 16 tile runs kSoftInner Jacobi steps in shared
// memory with its halo held at the previous iterate, so one barrier moves
// information across a tile instead of one node (the relaxed weights do
// not form a DAG -- a node also weighs neighbours that are not later than
// itself -- so the multipliers are a fixed point, not a back-substitution).
constexpr int kSoftTile = 16;
constexpr int kSoftInner = 16;

__global__ void __launch_bounds__(kSoftTile * kSoftTile) softmin_adjoint_kernel(SoftAdjArgs a) {
  constexpr int TS = kSoftTile, HW = TS + 2;
  __shared__ float lam[2][HW][HW + 1];
  const long long n = (long long)a.ny * a.nx;
  const int t = threadIdx.x, li = t / TS, lj = t - (t / TS) * TS;
  const int tiles_x = (a.nx + TS - 1) / TS, tiles = ((a.ny + TS - 1) / TS) * tiles_x;
  float *cur = a.La, *nxt = a.Lb;
  int it = 0;
  bool converged = false, abort = false;
  for (; it < a.max_iter; ++it) {
    int changed = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      const int i0 = (tile / tiles_x) * TS, j0 = (tile % tiles_x) * TS;
      // the tile and its halo at the previous iterate (0 outside the grid)
      for (int k = t; k < HW * HW; k += TS * TS) {
        const int r = k / HW, c = k - (k / HW) * HW, i = i0 + r - 1, j = j0 + c - 1;
        const float v = (i >= 0 && i < a.ny && j >= 0 && j < a.nx) ? __ldcg(cur + (long long)i * a.nx + j) : 0.0f;
        lam[0][r][c] = v;
        lam[1][r][c] = v;
      }
      // this thread's node: g and the weights of its neighbours toward it
      const int i = i0 + li, j = j0 + lj;
      const bool in = i < a.ny && j < a.nx;
      const long long p = in ? (long long)i * a.nx + j : 0;
      const bool live = in && a.T[p] < kInf;
      float gp = 0.0f, w[8];
#pragma unroll
      for (int nb = 0; nb < 8; ++nb) {
        w[nb] = 0.0f;
        const int ii = i + nb_dy(nb), jj = j + nb_dx(nb);
        if (live && ii >= 0 && ii < a.ny && jj >= 0 && jj < a.nx)
          w[nb] = a.wnb[(long long)((nb + 4) & 7) * n + (long long)ii * a.nx + jj];
      }
      if (live) gp = a.g[p];
      __syncthreads();
      int b = 0;
      for (int k = 0; k < kSoftInner; ++k) {
        float acc = 0.0f;
        if (live) {
          acc = gp;
#pragma unroll
          for (int nb = 0; nb < 8; ++nb)
            if (w[nb] != 0.0f) acc = fmaf(w[nb], lam[b][li + 1 + nb_dy(nb)][lj + 1 + nb_dx(nb)], acc);
        }
        lam[b ^ 1][li + 1][lj + 1] = acc;
        b ^= 1;
        __syncthreads();
      }
      if (in) {
        const float acc = lam[b][li + 1][lj + 1];
        changed |= node_changed(acc, __ldcg(cur + p), 0.0f, 1e-7f);
        __stcg(nxt + p, acc);
      }
      __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[(it + 1) % 3] = 0;
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&a.flags[it % 3], 1);
    if (!grid_sync(a.ctl)) {
      abort = true;
      break;
    }
    float *tmp = cur;
    cur = nxt;
    nxt = tmp;
    if (!ld_acquire_s32(&a.flags[it % 3])) {
      converged = true;
      ++it;
      break;
    }
  }
  if (!abort) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
      const float lp = __ldcg(cur + p);
      const bool act = a.T[p] < kInf && !a.src[p];
#pragma unroll
      for (int c = 0; c < 5; ++c) a.grad[c * n + p] = act ? lp * a.dT[c * n + p] : 0.0f;
      if (a.lam_out) a.lam_out[p] = lp;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl.st->adj_sweeps = it;
    if (!converged && !abort) set_error(a.ctl.st, RF_ERR_NOT_CONVERGED);
  }
}

}  // namespace rf

using namespace rf;

namespace {

int coop_grid(rf_ctx *ctx, const void *kernel, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
    return 0;
  return per_sm * ctx->num_sms;
}

}  // namespace

extern "C" rf_status rf_softmin_forward(rf_ctx *ctx, const rf_grid *grid, const float *proj5, float eps,
                                        const uint8_t *src, float tau, const rf_opts *opts, float *T,
                                        void *stream) {
  if (!ctx || !grid_ok(grid) || !proj5 || !src || !T || !(eps >= 0.0f) || !(tau >= 0.0f) || !(tau < kInf))
    return RF_ERR_INVALID_ARG;
  rf_opts o = {0.0f, 64, RF_MODE_COLD, 0, 0, 1e-6f, 0, 0.0f};
  if (opts) o = *opts;
  if (o.max_sweeps < 1 || !(o.tol >= 0.0f) || !(o.rtol >= 0.0f) || (o.mode != RF_MODE_COLD && o.mode != RF_MODE_WARM))
    return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ny = grid->ny, nx = grid->nx;
  const long long n = (long long)ny * nx;
  rf_status rs;
  if (o.variant == RF_SWEEP_AUTO || o.variant == RF_SWEEP_TILES) {
    // the tile queue (rf_sweep_tiles.cu) with the soft-min update: Jacobi
    // inside 16 x 16 tiles, rounds over the tiles the front reaches
    const int ts = tile_side(o.variant == RF_SWEEP_TILES ? o.band : 0);
    const int ncap = tiles_cap(1, n, std::max(ny, nx), ts);
    if ((rs = ensure(&ctx->tilebuf, &ctx->tilebuf_cap, tile_work_bytes(1, ncap, ts))) != RF_OK) return rs;
    if ((rs = ensure(&ctx->tbuf, &ctx->tbuf_cap, (size_t)n)) != RF_OK) return rs;
    if ((rs = ensure(&ctx->changed, &ctx->changed_cap, (size_t)o.max_sweeps + 2)) != RF_OK) return rs;
    cudaMemsetAsync(ctx->changed, 0, sizeof(int) * (o.max_sweeps + 2), s);
    cudaMemsetAsync(&ctx->state->sweeps, 0, sizeof(int) * 2, s);
    cudaMemsetAsync(&ctx->state->bar, 0, sizeof(unsigned long long) + 2 * sizeof(unsigned), s);
    cudaMemsetAsync(&ctx->state->cell_updates, 0, sizeof(unsigned long long), s);
    int *has_src = ctx->changed + o.max_sweeps;
    init_state(T, src, n, o.mode == RF_MODE_WARM, ctx->state, has_src, ctx->num_sms, s);
    check_source_flag(has_src, ctx->state, s);
    LaunchCtl ctl;
    ctl.st = ctx->state;
    ctl.abort = ctx->changed + o.max_sweeps + 1;
    ctl.timeout_ns = ctx->timeout_ns;
    const TileWork w = tile_work_carve(ctx->tilebuf, 1, ncap, ts);
    TileLaunch L;
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
    L.tau = tau;
    L.grid_status = nullptr;
    return tiles_launch(L, w, ctl, s);
  }
  // the line-sweep variants select Jacobi iterations over the whole grid
  if ((rs = ensure(&ctx->tbuf, &ctx->tbuf_cap, (size_t)n)) != RF_OK) return rs;
  if ((rs = ensure(&ctx->changed, &ctx->changed_cap, (size_t)8)) != RF_OK) return rs;
  cudaMemsetAsync(ctx->changed, 0, sizeof(int) * 8, s);
  cudaMemsetAsync(&ctx->state->sweeps, 0, sizeof(int) * 2, s);
  cudaMemsetAsync(&ctx->state->bar, 0, sizeof(unsigned long long) + 2 * sizeof(unsigned), s);
  int *has_src = ctx->changed + 4;
  init_state(T, src, n, o.mode == RF_MODE_WARM, ctx->state, has_src, ctx->num_sms, s);
  check_source_flag(has_src, ctx->state, s);
  SoftArgs a;
  a.ny = ny;
  a.nx = nx;
  a.h = grid->h;
  a.eps = eps;
  a.tau = tau;
  a.f = proj5;
  a.src = src;
  a.Ta = T;
  a.Tb = ctx->tbuf;
  // Jacobi moves information one node per iteration: max_sweeps lengths of
  // the longer side
  a.max_iter = o.max_sweeps * std::max(ny, nx);
  a.tol = o.tol;
  a.rtol = o.rtol;
  a.changed = ctx->changed;
  a.ctl.st = ctx->state;
  a.ctl.abort = ctx->changed + 5;
  a.ctl.timeout_ns = ctx->timeout_ns;
  const int g = coop_grid(ctx, (const void *)softmin_solve_kernel, 256);
  if (!g) return RF_ERR_UNSUPPORTED;
  void *args[] = {&a};
  return cuda_status(
      cudaLaunchCooperativeKernel((const void *)softmin_solve_kernel, dim3(g), dim3(256), args, 0, s));
}

extern "C" rf_status rf_softmin_record(rf_ctx *ctx, const rf_grid *grid, const float *proj5, float eps,
                                       const uint8_t *src, const float *T, float tau, float *wnb, float *dT,
                                       void *stream) {
  if (!ctx || !grid_ok(grid) || !proj5 || !src || !T || !wnb || !dT || !(eps >= 0.0f) || !(tau >= 0.0f))
    return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const long long n = (long long)grid->ny * grid->nx;
  softmin_record_kernel<<<blocks_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(grid->ny, grid->nx, grid->h, eps, tau,
                                                                             proj5, src, T, wnb, dT);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_softmin_adjoint(rf_ctx *ctx, const rf_grid *grid, const uint8_t *src, const float *T,
                                        const float *wnb, const float *dT, const float *dLdT, float *dLdproj5,
                                        float *lambda, void *stream) {
  if (!ctx || !grid_ok(grid) || !src || !T || !wnb || !dT || !dLdT || !dLdproj5) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ny = grid->ny, nx = grid->nx;
  const long long n = (long long)ny * nx;
  rf_status rs;
  if ((rs = ensure(&ctx->lbuf, &ctx->lbuf_cap, (size_t)(2 * n))) != RF_OK) return rs;
  if ((rs = ensure(&ctx->changed, &ctx->changed_cap, (size_t)8)) != RF_OK) return rs;
  cudaMemsetAsync(ctx->changed, 0, sizeof(int) * 8, s);
  cudaMemsetAsync(&ctx->state->adj_sweeps, 0, sizeof(int), s);
  cudaMemsetAsync(&ctx->state->bar, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(ctx->lbuf, 0, sizeof(float) * n, s);
  SoftAdjArgs a;
  a.ny = ny;
  a.nx = nx;
  a.src = src;
  a.T = T;
  a.wnb = wnb;
  a.dT = dT;
  a.g = dLdT;
  a.La = ctx->lbuf;
  a.Lb = ctx->lbuf + n;
  a.grad = dLdproj5;
  a.lam_out = lambda;
  a.max_iter = 64 * std::max(ny, nx);
  a.flags = ctx->changed;
  a.ctl.st = ctx->state;
  a.ctl.abort = ctx->changed + 5;
  a.ctl.timeout_ns = ctx->timeout_ns;
  const int g = coop_grid(ctx, (const void *)softmin_adjoint_kernel, kSoftTile * kSoftTile);
  if (!g) return RF_ERR_UNSUPPORTED;
  void *args[] = {&a};
  return cuda_status(cudaLaunchCooperativeKernel((const void *)softmin_adjoint_kernel, dim3(g),
                                                 dim3(kSoftTile * kSoftTile), args, 0, s));
}
