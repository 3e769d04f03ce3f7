// rf_ctx.cu -- context lifetime, statistics and status strings.
#include <cstring>

#include "rf_ctx.h"

extern "C" rf_status rf_ctx_create(rf_ctx **out, int device) {
  if (!out) return RF_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return RF_ERR_CUDA;
  rf_ctx *c = new rf_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc((void **)&c->state, sizeof(rf::DevState)) != cudaSuccess) {
    delete c;
    return RF_ERR_NO_MEMORY;
  }
  if (cudaMemset(c->state, 0, sizeof(rf::DevState)) != cudaSuccess) {
    cudaFree(c->state);
    delete c;
    return RF_ERR_CUDA;
  }
  *out = c;
  return RF_OK;
}

extern "C" rf_status rf_ctx_destroy(rf_ctx *c) {
  if (!c) return RF_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->state);
  cudaFree(c->progress);
  cudaFree(c->changed);
  cudaFree(c->tbuf);
  cudaFree(c->lbuf);
  cudaFree(c->scratch);
  cudaFree(c->adj_state);
  cudaFree(c->recbuf);
  cudaFree(c->tvbuf);
  cudaFree(c->tilebuf);
  cudaFree(c->stepbuf);
  cudaFree(c->wpack);
  if (c->step_in) cudaStreamDestroy(c->step_in);
  if (c->step_out) cudaStreamDestroy(c->step_out);
  for (cudaEvent_t e : c->step_ev)
    if (e) cudaEventDestroy(e);
  delete c;
  return RF_OK;
}

extern "C" rf_status rf_ctx_set_timeout(rf_ctx *c, int64_t timeout_ns) {
  if (!c || timeout_ns < 0) return RF_ERR_INVALID_ARG;
  c->timeout_ns = (long long)timeout_ns;
  return RF_OK;
}

extern "C" rf_status rf_ctx_set_adjoint_park(rf_ctx *c, int64_t park_ns) {
  if (!c || park_ns < 0) return RF_ERR_INVALID_ARG;
  c->adj_park_ns = (long long)park_ns;
  return RF_OK;
}

extern "C" rf_status rf_ctx_last_stats(rf_ctx *c, rf_stats *out) {
  if (!c || !out) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return RF_ERR_CUDA;
  if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) return RF_ERR_CUDA;
  rf::DevState s;
  if (cudaMemcpy(&s, c->state, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RF_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  out->status = s.status;
  out->sweeps = s.sweeps;
  out->converged = s.converged;
  out->adj_sweeps = s.adj_sweeps;
  out->cell_updates = (int64_t)s.cell_updates;
  float mr;
  std::memcpy(&mr, &s.max_res_bits, sizeof(mr));
  out->max_residual = mr;
  out->rounds = (int32_t)s.rounds;
  // the status word reports errors since the previous call: clear it
  int zero = 0;
  if (cudaMemcpy(&c->state->status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return RF_ERR_CUDA;
  return (rf_status)s.status;
}

extern "C" const char *rf_status_string(rf_status s) {
  switch (s) {
    case RF_OK: return "RF_OK";
    case RF_ERR_INVALID_ARG: return "RF_ERR_INVALID_ARG";
    case RF_ERR_CUDA: return "RF_ERR_CUDA";
    case RF_ERR_NOT_CONVERGED: return "RF_ERR_NOT_CONVERGED";
    case RF_ERR_TIMEOUT: return "RF_ERR_TIMEOUT";
    case RF_ERR_NONFINITE_INPUT: return "RF_ERR_NONFINITE_INPUT";
    case RF_ERR_NO_SOURCE: return "RF_ERR_NO_SOURCE";
    case RF_ERR_NO_MEMORY: return "RF_ERR_NO_MEMORY";
    case RF_ERR_UNSUPPORTED: return "RF_ERR_UNSUPPORTED";
  }
  return "RF_ERR_UNKNOWN";
}
