// rf_encoder.cu -- the head of the covariate encoder (Sec. 5, "Encoder
// Architecture"): the global pathway's per-grid baseline (G0, b0) and the
// fully-convolutional pathway's per-node residuals combine as
// G = G0 + alpha G_local, b = b0 + alpha b_local, written as the five
// (g11, g12, g22, b1, b2) planes the App. B projection reads; and the
// adjoint of that map (the residual gradient scaled by alpha, the baseline
// gradient summed over each grid's nodes).  Memory-bound: 20 B read + 20 B
// written per node forward, the same backward.
#include <cuda_bf16.h>

#include "rf_ctx.h"

namespace rf {

__device__ __forceinline__ uint16_t f2bf(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }

// one thread per node: gb[b][c][p] = base[b][c] + alpha local[b][p][c]
__global__ void __launch_bounds__(256) combine_kernel(const float *local, int B, long long HW, int C,
                                                      const float *base, int Cb, float alpha, float *gb) {
  const long long n = (long long)B * HW;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long b = q / HW, p = q - b * HW;
    const float *lp = local + q * C;
#pragma unroll
    for (int c = 0; c < 5; ++c) gb[(b * 5 + c) * HW + p] = fmaf(alpha, lp[c], base[b * Cb + c]);
  }
}

// residual gradient: dlocal[b][p][c] = alpha dgb[b][c][p] (c < 5), 0 else
__global__ void __launch_bounds__(256) combine_local_bwd_kernel(const float *dgb, int B, long long HW, int C,
                                                                float alpha, uint16_t *dlocal) {
  const long long n = (long long)B * HW;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long b = q / HW, p = q - b * HW;
    for (int c = 0; c < C; ++c) dlocal[q * C + c] = c < 5 ? f2bf(alpha * dgb[(b * 5 + c) * HW + p]) : (uint16_t)0;
  }
}

// baseline gradient: one CTA per (grid, channel), fixed-order reduction
__global__ void __launch_bounds__(256) combine_base_bwd_kernel(const float *dgb, long long HW, int Cb,
                                                               uint16_t *dbase) {
  __shared__ float red[8];
  const int b = blockIdx.x / Cb, c = blockIdx.x - b * Cb;
  float acc = 0.0f;
  if (c < 5) {
    const float *src = dgb + ((long long)b * 5 + c) * HW;
    for (long long p = threadIdx.x; p < HW; p += blockDim.x) acc += src[p];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    dbase[(long long)b * Cb + c] = f2bf(t);
  }
}

}  // namespace rf

using namespace rf;

extern "C" rf_status rf_encoder_combine(rf_ctx *ctx, const float *local, int B, int H, int W, int C,
                                        const float *base, int Cb, float alpha, float *gb, void *stream) {
  if (!ctx || !local || !base || !gb || B < 1 || H < 1 || W < 1 || C < 5 || Cb < 5) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const long long HW = (long long)H * W;
  combine_kernel<<<blocks_for((long long)B * HW, 256, ctx->num_sms * 8), 256, 0, s>>>(local, B, HW, C, base, Cb,
                                                                                       alpha, gb);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_encoder_combine_backward(rf_ctx *ctx, const float *dgb, int B, int H, int W, int C, int Cb,
                                                 float alpha, uint16_t *dlocal, uint16_t *dbase, void *stream) {
  if (!ctx || !dgb || !dlocal || !dbase || B < 1 || H < 1 || W < 1 || C < 5 || Cb < 5) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const long long HW = (long long)H * W;
  combine_local_bwd_kernel<<<blocks_for((long long)B * HW, 256, ctx->num_sms * 8), 256, 0, s>>>(dgb, B, HW, C,
                                                                                                 alpha, dlocal);
  if (cudaGetLastError() != cudaSuccess) return RF_ERR_CUDA;
  combine_base_bwd_kernel<<<B * Cb, 256, 0, s>>>(dgb, HW, Cb, dbase);
  return cuda_status(cudaGetLastError());
}
