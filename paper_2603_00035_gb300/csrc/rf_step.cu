// rf_step.cu -- whole steps of the inverse-problem hot path on host buffers
// (a1 projection, a2-a4 forward solve, a5 record, a6-a8 adjoint, a9
// projection backward; Sec. 3 and Alg. 1-2), pipelined across steps.
//
// Step i: its inputs (raw fields, sources, dL/dT) are copied to one of two
// device input sets on the context's input-copy stream; the five kernels run
// on the caller's stream once that copy is done; T and dL/draw go to one of
// two device output sets and are copied back on the output-copy stream.  So
// step i + 1's input copy and step i - 1's output copy overlap step i's
// compute.  A set is refilled only after the step that last used it has
// read its inputs (input set) or had its results copied out (output set).
// The intermediates (projected fields, clip mask, record, dL/dproj) are one
// set: the computes run one after another on the caller's stream.
#include <algorithm>

#include "rf_ctx.h"

using rf::ensure;
using rf::grid_ok;

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct StepBufs {
  float *raw[2];
  uint8_t *src[2];
  float *g[2];
  float *T[2];
  float *graw[2];
  float *proj, *gproj, *w1, *dT;
  uint8_t *clip, *id;
};

// Carve the step buffers for n nodes out of base (or, with base NULL,
// return the bytes needed).
size_t carve(unsigned char *base, size_t n, StepBufs *b) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base ? base + off : nullptr;
    off += up256(bytes);
    return p;
  };
  for (int k = 0; k < 2; ++k) {
    b->raw[k] = (float *)take(5 * n * sizeof(float));
    b->src[k] = (uint8_t *)take(n);
    b->g[k] = (float *)take(n * sizeof(float));
    b->T[k] = (float *)take(n * sizeof(float));
    b->graw[k] = (float *)take(5 * n * sizeof(float));
  }
  b->proj = (float *)take(5 * n * sizeof(float));
  b->gproj = (float *)take(5 * n * sizeof(float));
  b->w1 = (float *)take(n * sizeof(float));
  b->dT = (float *)take(5 * n * sizeof(float));
  b->clip = (uint8_t *)take(n);
  b->id = (uint8_t *)take(n);
  return off;
}

rf_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? RF_OK : RF_ERR_CUDA; }

}  // namespace

extern "C" rf_status rf_step_host(rf_ctx *ctx, const rf_grid *grid, int n_steps, const float *const *raw5_h,
                                  const uint8_t *const *src_h, const float *const *dLdT_h, float eps, float delta,
                                  const rf_opts *opts, int algo, float *const *T_h, float *const *dLdraw_h,
                                  void *stream) {
  if (!ctx || !grid_ok(grid) || n_steps < 0 || (n_steps > 0 && (!raw5_h || !src_h || !dLdT_h || !T_h || !dLdraw_h)))
    return RF_ERR_INVALID_ARG;
  for (int i = 0; i < n_steps; ++i)
    if (!raw5_h[i] || !src_h[i] || !dLdT_h[i] || !T_h[i] || !dLdraw_h[i]) return RF_ERR_INVALID_ARG;
  if (algo != RF_ADJ_SWEEP && algo != RF_ADJ_ORDERED && algo != RF_ADJ_LEVELS && algo != RF_ADJ_TILES)
    return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  if (n_steps == 0) return RF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)grid->ny * grid->nx;

  StepBufs b;
  const size_t need = carve(nullptr, n, &b);
  rf_status rs;
  if ((rs = ensure(&ctx->stepbuf, &ctx->stepbuf_cap, need)) != RF_OK) return rs;
  carve(ctx->stepbuf, n, &b);
  if (!ctx->step_in && (rs = cuda_ok(cudaStreamCreateWithFlags(&ctx->step_in, cudaStreamNonBlocking))) != RF_OK)
    return rs;
  if (!ctx->step_out && (rs = cuda_ok(cudaStreamCreateWithFlags(&ctx->step_out, cudaStreamNonBlocking))) != RF_OK)
    return rs;
  for (cudaEvent_t &e : ctx->step_ev)
    if (!e && (rs = cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming))) != RF_OK) return rs;
  cudaEvent_t *ev_in = ctx->step_ev, *ev_done = ctx->step_ev + 2, *ev_out = ctx->step_ev + 4;
  // the copy streams start after what the caller queued before this call
  cudaEvent_t start = ev_done[0];
  if ((rs = cuda_ok(cudaEventRecord(start, s))) != RF_OK) return rs;
  if ((rs = cuda_ok(cudaStreamWaitEvent(ctx->step_in, start, 0))) != RF_OK) return rs;
  if ((rs = cuda_ok(cudaStreamWaitEvent(ctx->step_out, start, 0))) != RF_OK) return rs;

  rf_record rec;
  rec.id = b.id;
  rec.w1 = b.w1;
  rec.dT = b.dT;
  for (int i = 0; i < n_steps; ++i) {
    const int k = i & 1;
    // inputs of step i into set k, once step i - 2 has read them
    if (i >= 2 && (rs = cuda_ok(cudaStreamWaitEvent(ctx->step_in, ev_done[k], 0))) != RF_OK) return rs;
    if ((rs = cuda_ok(cudaMemcpyAsync(b.raw[k], raw5_h[i], 5 * n * sizeof(float), cudaMemcpyHostToDevice,
                                      ctx->step_in))) != RF_OK ||
        (rs = cuda_ok(cudaMemcpyAsync(b.src[k], src_h[i], n, cudaMemcpyHostToDevice, ctx->step_in))) != RF_OK ||
        (rs = cuda_ok(cudaMemcpyAsync(b.g[k], dLdT_h[i], n * sizeof(float), cudaMemcpyHostToDevice,
                                      ctx->step_in))) != RF_OK ||
        (rs = cuda_ok(cudaEventRecord(ev_in[k], ctx->step_in))) != RF_OK)
      return rs;
    // compute on the caller's stream: its inputs copied, the output set free
    if ((rs = cuda_ok(cudaStreamWaitEvent(s, ev_in[k], 0))) != RF_OK) return rs;
    if (i >= 2 && (rs = cuda_ok(cudaStreamWaitEvent(s, ev_out[k], 0))) != RF_OK) return rs;
    if ((rs = rf_project(ctx, grid, b.raw[k], eps, delta, b.proj, b.clip, stream)) != RF_OK) return rs;
    if ((rs = rf_sweep_forward(ctx, grid, b.proj, eps, b.src[k], opts, b.T[k], nullptr, stream)) != RF_OK)
      return rs;
    if ((rs = rf_record_stencils(ctx, grid, b.proj, eps, b.src[k], b.T[k], &rec, stream)) != RF_OK) return rs;
    if ((rs = rf_adjoint(ctx, grid, b.src[k], b.T[k], &rec, b.g[k], b.gproj, nullptr, algo, stream)) != RF_OK)
      return rs;
    if ((rs = rf_project_backward(ctx, grid, b.raw[k], b.clip, eps, delta, b.gproj, b.graw[k], stream)) != RF_OK)
      return rs;
    if ((rs = cuda_ok(cudaEventRecord(ev_done[k], s))) != RF_OK) return rs;
    // results of step i out of set k
    if ((rs = cuda_ok(cudaStreamWaitEvent(ctx->step_out, ev_done[k], 0))) != RF_OK ||
        (rs = cuda_ok(cudaMemcpyAsync(T_h[i], b.T[k], n * sizeof(float), cudaMemcpyDeviceToHost,
                                      ctx->step_out))) != RF_OK ||
        (rs = cuda_ok(cudaMemcpyAsync(dLdraw_h[i], b.graw[k], 5 * n * sizeof(float), cudaMemcpyDeviceToHost,
                                      ctx->step_out))) != RF_OK ||
        (rs = cuda_ok(cudaEventRecord(ev_out[k], ctx->step_out))) != RF_OK)
      return rs;
  }
  // the caller's stream continues after the last result copy; the host
  // buffers are complete when this returns
  if ((rs = cuda_ok(cudaStreamWaitEvent(s, ev_out[(n_steps - 1) & 1], 0))) != RF_OK) return rs;
  ctx->last_stream = s;
  return cuda_ok(cudaStreamSynchronize(s));
}
