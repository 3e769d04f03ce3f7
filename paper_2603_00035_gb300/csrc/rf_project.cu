// rf_project.cu -- a1 feasibility projection and a9 its backward.
// Paper: App. B "Feasibility Projections" (|b|_{G^-1} via the closed-form
// 2x2 inverse); factor form M = L L^T + eps I, w scaled to
// |w|_{M^-1} <= 1 - delta.  Elementwise and HBM-bound: 20 B read + 8 B
// (+1 B clip) written per node forward; 40 B read + 20 B written backward.
#include "rf_ctx.h"

namespace rf {

struct ProjArgs {
  long long n;
  const float *raw;  // 5 planes
  float *proj;       // 5 planes
  uint8_t *clip;
  float eps, c;      // c = 1 - delta
  DevState *st;
};

__global__ void __launch_bounds__(256) project_kernel(ProjArgs a) {
  const long long n = a.n;
  bool bad = false;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float l11 = __ldg(a.raw + p), l21 = __ldg(a.raw + n + p),
                l22 = __ldg(a.raw + 2 * n + p), wx = __ldg(a.raw + 3 * n + p),
                wy = __ldg(a.raw + 4 * n + p);
    bad |= !(isfinite(l11) && isfinite(l21) && isfinite(l22) && isfinite(wx) &&
             isfinite(wy));
    const float m11 = fmaf(l11, l11, a.eps), m12 = l11 * l21,
                m22 = fmaf(l21, l21, fmaf(l22, l22, a.eps));
    const float q = l11 * l22;
    const float det = fmaf(q, q, a.eps * (l11 * l11 + l21 * l21 + l22 * l22 + a.eps));
    const float n2 = (wx * wx * m22 - 2.0f * wx * wy * m12 + wy * wy * m11) / det;
    const float nn = sqrtf(n2);
    const bool clipped = nn > a.c;
    const float s = clipped ? a.c / nn : 1.0f;
    if (a.proj != a.raw) {
      a.proj[p] = l11;
      a.proj[n + p] = l21;
      a.proj[2 * n + p] = l22;
    }
    a.proj[3 * n + p] = wx * s;
    a.proj[4 * n + p] = wy * s;
    a.clip[p] = clipped ? 1 : 0;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_error(a.st, RF_ERR_NONFINITE_INPUT);
}

struct ProjBwdArgs {
  long long n;
  const float *raw;
  const uint8_t *clip;
  const float *gin;  // 5 planes, dL/d(L, w_out)
  float *gout;       // 5 planes, dL/d(raw)
  float eps, c;
};

__global__ void __launch_bounds__(256) project_backward_kernel(ProjBwdArgs a) {
  const long long n = a.n;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    float g11 = a.gin[p], g21 = a.gin[n + p], g22 = a.gin[2 * n + p];
    float gx = a.gin[3 * n + p], gy = a.gin[4 * n + p];
    if (a.clip[p]) {
      const float l11 = __ldg(a.raw + p), l21 = __ldg(a.raw + n + p),
                  l22 = __ldg(a.raw + 2 * n + p), wx = __ldg(a.raw + 3 * n + p),
                  wy = __ldg(a.raw + 4 * n + p);
      const float m11 = fmaf(l11, l11, a.eps), m12 = l11 * l21,
                  m22 = fmaf(l21, l21, fmaf(l22, l22, a.eps));
      const float q = l11 * l22;
      const float det = fmaf(q, q, a.eps * (l11 * l11 + l21 * l21 + l22 * l22 + a.eps));
      // P w with P = M^-1
      const float pwx = (m22 * wx - m12 * wy) / det;
      const float pwy = (m11 * wy - m12 * wx) / det;
      const float n2 = wx * pwx + wy * pwy;
      const float nn = sqrtf(n2);
      const float wg = wx * gx + wy * gy;
      const float ox = (a.c / nn) * (gx - pwx * wg / n2);
      const float oy = (a.c / nn) * (gy - pwy * wg / n2);
      const float s = a.c * wg / (2.0f * nn * n2);
      const float D11 = s * pwx * pwx, D12 = s * pwx * pwy, D22 = s * pwy * pwy;
      g11 += 2.0f * (D11 * l11 + D12 * l21);
      g21 += 2.0f * (D12 * l11 + D22 * l21);
      g22 += 2.0f * D22 * l22;
      gx = ox;
      gy = oy;
    }
    a.gout[p] = g11;
    a.gout[n + p] = g21;
    a.gout[2 * n + p] = g22;
    a.gout[3 * n + p] = gx;
    a.gout[4 * n + p] = gy;
  }
}

}  // namespace rf

using namespace rf;

extern "C" rf_status rf_project(rf_ctx *ctx, const rf_grid *grid, const float *raw5,
                                float eps, float delta, float *proj5, uint8_t *clip,
                                void *stream) {
  if (!ctx || !grid_ok(grid) || !raw5 || !proj5 || !clip) return RF_ERR_INVALID_ARG;
  if (!(eps >= 0.0f) || !(delta > 0.0f && delta < 1.0f)) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  ProjArgs a;
  a.n = (long long)grid->ny * grid->nx;
  a.raw = raw5;
  a.proj = proj5;
  a.clip = clip;
  a.eps = eps;
  a.c = 1.0f - delta;
  a.st = ctx->state;
  project_kernel<<<blocks_for(a.n, 256, ctx->num_sms * 8), 256, 0, s>>>(a);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_project_backward(rf_ctx *ctx, const rf_grid *grid,
                                         const float *raw5, const uint8_t *clip,
                                         float eps, float delta, const float *dproj5,
                                         float *draw5, void *stream) {
  if (!ctx || !grid_ok(grid) || !raw5 || !clip || !dproj5 || !draw5)
    return RF_ERR_INVALID_ARG;
  if (!(eps >= 0.0f) || !(delta > 0.0f && delta < 1.0f)) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  ProjBwdArgs a;
  a.n = (long long)grid->ny * grid->nx;
  a.raw = raw5;
  a.clip = clip;
  a.gin = dproj5;
  a.gout = draw5;
  a.eps = eps;
  a.c = 1.0f - delta;
  project_backward_kernel<<<blocks_for(a.n, 256, ctx->num_sms * 8), 256, 0, s>>>(a);
  return cuda_status(cudaGetLastError());
}
