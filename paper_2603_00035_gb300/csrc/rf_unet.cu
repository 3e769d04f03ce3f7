// rf_unet.cu -- kernels of the learned warm start (a11, a12): a small
// U-Net in BF16 with FP32 accumulation, trained on the solver's own
// outputs.  The paper has no network for this (it is the build's learned
// initial guess for the replacement sweeps of rf_sweep_forward).
//
// 3x3 "same" convolutions as implicit GEMMs on the tensor cores
// (mma.sync m16n8k16, BF16 inputs, FP32 accumulators):
//   forward  y[p, co] = sum_{tap, ci} x[p + off(tap), ci] W[co, tap, ci]
//            GEMM M = pixels, N = Cout, K = 9 Cin; the 3x3 gather comes from
//            a haloed input patch in shared memory (no im2col buffer);
//   dgrad    the same kernel on W' [ci, tap', co] = W[co, 8 - tap, ci];
//   wgrad    dW[co, tap, ci] = sum_p dy[p, co] x[p + off(tap), ci]
//            GEMM M = Cout, N = 9 Cin, K = pixels, split over pixel rows
//            with FP32 atomic accumulation.
// Activations are NHWC BF16 with channels a multiple of 16.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "rf_ctx.h"

namespace rf {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---- forward / dgrad ---------------------------------------------------------
// CTA: 8 x 16 output pixels of one image, 32 output channels, 4 warps; warp
// w owns pixel rows 2w, 2w+1 (two m16 tiles) x 32 channels (four n8 tiles).
// K loop: input channels in chunks of 16; per chunk the 10 x 18 halo patch
// (zero outside the image) and the [9 taps][32 co][16 ci] weights go to
// shared memory with a 24-element pitch (48 B: conflict-free ldmatrix).
constexpr int kCvTH = 8, kCvTW = 16, kCvBN = 32, kCvPitch = 24;

struct ConvArgs {
  const bf16 *x;  // [B][H][W][Cin]
  const bf16 *w;  // [Cout][9][Cin]
  const float *bias;  // [Cout] or null
  bf16 *y;        // [B][H][W][Cout]
  float *y32;     // optional FP32 copy of the output
  int B, H, W, Cin, Cout, relu;
};

__global__ void __launch_bounds__(128) conv3x3_fwd_kernel(ConvArgs a) {
  __shared__ __align__(16) bf16 xs[(kCvTH + 2) * (kCvTW + 2) * kCvPitch];
  __shared__ __align__(16) bf16 ws[9 * kCvBN * kCvPitch];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = (a.W + kCvTW - 1) / kCvTW;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int x0 = tx * kCvTW, y0 = ty * kCvTH;
  const int co0 = blockIdx.y * kCvBN;
  const int b = blockIdx.z;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;

  for (int c0 = 0; c0 < a.Cin; c0 += 16) {
    // halo patch: 10 x 18 pixels x 16 channels, as 8-channel (16 B) vectors
    for (int v = tid; v < (kCvTH + 2) * (kCvTW + 2) * 2; v += 128) {
      const int pix = v >> 1, half = v & 1;
      const int py = pix / (kCvTW + 2), px = pix - py * (kCvTW + 2);
      const int gy = y0 + py - 1, gx = x0 + px - 1;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
        val = *reinterpret_cast<const uint4 *>(a.x + (((long long)b * a.H + gy) * a.W + gx) * a.Cin + c0 + half * 8);
      *reinterpret_cast<uint4 *>(xs + pix * kCvPitch + half * 8) = val;
    }
    // weights: [9][32 co][16 ci]
    for (int v = tid; v < 9 * kCvBN * 2; v += 128) {
      const int half = v & 1, r = v >> 1;
      const int tap = r / kCvBN, co = r - tap * kCvBN;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (co0 + co < a.Cout)
        val = *reinterpret_cast<const uint4 *>(a.w + ((long long)(co0 + co) * 9 + tap) * a.Cin + c0 + half * 8);
      *reinterpret_cast<uint4 *>(ws + (tap * kCvBN + co) * kCvPitch + half * 8) = val;
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap - ky * 3;
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // m16 tile = one output pixel row (16 pixels); lanes 0-15 address
        // rows (pixels) 0-15 at channel 0, lanes 16-31 the same at channel 8
        const int prow = 2 * warp + mt;
        const int pcol = lane & 15;
        const bf16 *src = xs + ((prow + ky) * (kCvTW + 2) + pcol + kx) * kCvPitch + (lane >> 4) * 8;
        ldsm_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], src);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        // two n8 tiles: matrices (n 0-7, k 0-7), (n 0-7, k 8-15),
        // (n 8-15, k 0-7), (n 8-15, k 8-15)
        const int n = np * 16 + (lane & 7) + ((lane >> 4) << 3);
        const int kh = (lane >> 3) & 1;
        uint32_t b0, b1, b2, b3;
        ldsm_x4(b0, b1, b2, b3, ws + (tap * kCvBN + n) * kCvPitch + kh * 8);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_bf16(acc[mt][2 * np], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
          mma_bf16(acc[mt][2 * np + 1], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b2, b3);
        }
      }
    }
    __syncthreads();
  }
  // epilogue: bias, ReLU, BF16 (and optional FP32) NHWC stores
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int gy = y0 + 2 * warp + mt;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int co = co0 + nt * 8 + 2 * t4;
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int gx = x0 + g + hf * 8;
        if (gy < a.H && gx < a.W && co < a.Cout) {
          float v0 = acc[mt][nt][2 * hf], v1 = acc[mt][nt][2 * hf + 1];
          if (a.bias) {
            v0 += a.bias[co];
            v1 += a.bias[co + 1];
          }
          if (a.relu) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
          }
          const long long o = (((long long)b * a.H + gy) * a.W + gx) * a.Cout + co;
          *reinterpret_cast<__nv_bfloat162 *>(a.y + o) = __floats2bfloat162_rn(v0, v1);
          if (a.y32) {
            a.y32[o] = v0;
            a.y32[o + 1] = v1;
          }
        }
      }
    }
  }
}


// ---- wgrad ------------------------------------------------------------------
// CTA: 32 output channels x 16 input channels x 9 taps for one image and
// kWgRows pixel rows; 3 warps, warp ky owns taps (ky, 0..2) -> 3 x (2 m16 x
// 2 n8) accumulator tiles.  Per 16-pixel row segment: dy [16 px][32 co] and
// the 3 x 18 halo of x [px][16 ci] go to shared memory; both operands are
// read with ldmatrix.trans (A = dy^T: m = co, k = px; B: k = px, n = ci).
constexpr int kWgRows = 8, kDyPitch = 40;

struct WgradArgs {
  const bf16 *x;   // [B][H][W][Cin]
  const bf16 *dy;  // [B][H][W][Cout]
  float *dw;       // [Cout][9][Cin], accumulated
  int B, H, W, Cin, Cout;
};

__global__ void __launch_bounds__(96) conv3x3_wgrad_kernel(WgradArgs a) {
  __shared__ __align__(16) bf16 ds[16 * kDyPitch];
  __shared__ __align__(16) bf16 xs[3 * 18 * kCvPitch];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int co0 = blockIdx.x * 32, ci0 = blockIdx.y * 16;
  const int rows_per = (a.H + kWgRows - 1) / kWgRows;
  const int b = blockIdx.z / rows_per, ry0 = (blockIdx.z - b * rows_per) * kWgRows;
  float acc[3][2][2][4];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l) acc[i][j][k][l] = 0.0f;

  for (int y = ry0; y < min(ry0 + kWgRows, a.H); ++y) {
    for (int x0 = 0; x0 < a.W; x0 += 16) {
      // dy segment: 16 px x 32 co (4 x 16 B per pixel)
      for (int v = tid; v < 16 * 4; v += 96) {
        const int px = v >> 2, q = v & 3;
        const int gx = x0 + px;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (gx < a.W && co0 + q * 8 < a.Cout)
          val = *reinterpret_cast<const uint4 *>(a.dy + (((long long)b * a.H + y) * a.W + gx) * a.Cout + co0 + q * 8);
        *reinterpret_cast<uint4 *>(ds + px * kDyPitch + q * 8) = val;
      }
      // x halo: rows y-1..y+1, px x0-1 .. x0+16, 16 ci (2 x 16 B)
      for (int v = tid; v < 3 * 18 * 2; v += 96) {
        const int half = v & 1, r = v >> 1;
        const int ry = r / 18, px = r - ry * 18;
        const int gy = y + ry - 1, gx = x0 + px - 1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
          val = *reinterpret_cast<const uint4 *>(a.x + (((long long)b * a.H + gy) * a.W + gx) * a.Cin + ci0 + half * 8);
        *reinterpret_cast<uint4 *>(xs + (ry * 18 + px) * kCvPitch + half * 8) = val;
      }
      __syncthreads();
      const int j = lane >> 3, r = lane & 7;
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int px = r + ((j >> 1) << 3), co = mt * 16 + ((j & 1) << 3);
        ldsm_x4_t(af[mt][0], af[mt][1], af[mt][2], af[mt][3], ds + px * kDyPitch + co);
      }
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        // B rows: pixels (r + 8 (j&1)) shifted by kx in halo row `warp` (= ky)
        const int px = r + ((j & 1) << 3) + kx, ci = (j >> 1) << 3;
        uint32_t b0, b1, b2, b3;
        ldsm_x4_t(b0, b1, b2, b3, xs + (warp * 18 + px) * kCvPitch + ci);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_bf16(acc[kx][mt][0], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
          mma_bf16(acc[kx][mt][1], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b2, b3);
        }
      }
      __syncthreads();
    }
  }
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int kx = 0; kx < 3; ++kx) {
    const int tap = warp * 3 + kx;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int co = co0 + mt * 16 + g + hf * 8, ci = ci0 + nt * 8 + 2 * t4;
          if (co < a.Cout) {
            float *d = a.dw + ((long long)co * 9 + tap) * a.Cin + ci;
            atomicAdd(d, acc[kx][mt][nt][2 * hf]);
            atomicAdd(d + 1, acc[kx][mt][nt][2 * hf + 1]);
          }
        }
  }
}

// dbias[co] += sum over pixels of dy[p, co]
__global__ void __launch_bounds__(256) bias_grad_kernel(const bf16 *dy, long long npix, int C, float *db) {
  const int co = blockIdx.y * 32 + (threadIdx.x & 31);
  float s = 0.0f;
  if (co < C)
    for (long long p = blockIdx.x * 8 + (threadIdx.x >> 5); p < npix; p += (long long)gridDim.x * 8)
      s += __bfloat162float(dy[p * C + co]);
  __shared__ float red[8][33];
  red[threadIdx.x >> 5][threadIdx.x & 31] = s;
  __syncthreads();
  if (threadIdx.x < 32 && co < C) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    atomicAdd(db + co, t);
  }
}

// W'[ci][tap'][co] = W[co][8 - tap'][ci]: the weights of the data gradient
__global__ void flip_weights_kernel(const bf16 *w, bf16 *wt, int Cin, int Cout) {
  const long long n = (long long)Cout * 9 * Cin;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(i % Cin);
    const int tap = (int)((i / Cin) % 9);
    const int co = (int)(i / ((long long)Cin * 9));
    wt[((long long)ci * 9 + (8 - tap)) * Cout + co] = w[i];
  }
}

// ---- memory-bound pieces (NHWC BF16) ------------------------------------------
#define RF_GRID_STRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// 2x2 max pool (H, W even); arg = position 0..3 of the max in its window
__global__ void maxpool2_fwd_kernel(const bf16 *x, bf16 *y, uint8_t *arg, int B, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  const long long n = (long long)B * Ho * Wo * C;
  RF_GRID_STRIDE(i, n) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), b = (int)(q / ((long long)Wo * Ho));
    float best = -3.0e38f;
    int bi = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float v = __bfloat162float(x[(((long long)b * H + 2 * yo + (k >> 1)) * W + 2 * xo + (k & 1)) * C + c]);
      if (v > best) {
        best = v;
        bi = k;
      }
    }
    y[i] = __float2bfloat16(best);
    arg[i] = (uint8_t)bi;
  }
}

__global__ void maxpool2_bwd_kernel(const bf16 *dy, const uint8_t *arg, bf16 *dx, int B, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  const long long n = (long long)B * Ho * Wo * C;
  RF_GRID_STRIDE(i, n) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), b = (int)(q / ((long long)Wo * Ho));
    const bf16 z = __float2bfloat16(0.0f);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      dx[(((long long)b * H + 2 * yo + (k >> 1)) * W + 2 * xo + (k & 1)) * C + c] = (arg[i] == k) ? dy[i] : z;
  }
}

// nearest 2x upsampling and its adjoint (sum of the 4 children)
__global__ void upsample2_fwd_kernel(const bf16 *x, bf16 *y, int B, int H, int W, int C) {
  const long long n = (long long)B * (2 * H) * (2 * W) * C;
  RF_GRID_STRIDE(i, n) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xo = (int)(q % (2 * W)), yo = (int)((q / (2 * W)) % (2 * H)), b = (int)(q / (4LL * W * H));
    y[i] = x[(((long long)b * H + yo / 2) * W + xo / 2) * C + c];
  }
}

__global__ void upsample2_bwd_kernel(const bf16 *dy, bf16 *dx, int B, int H, int W, int C) {
  const long long n = (long long)B * H * W * C;
  RF_GRID_STRIDE(i, n) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xi = (int)(q % W), yi = (int)((q / W) % H), b = (int)(q / ((long long)W * H));
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      s += __bfloat162float(dy[(((long long)b * 2 * H + 2 * yi + (k >> 1)) * 2 * W + 2 * xi + (k & 1)) * C + c]);
    dx[i] = __float2bfloat16(s);
  }
}

// y[..., 0:Ca] = a, y[..., Ca:Ca+Cb] = b; the backward splits (dir = 1)
__global__ void concat_kernel(bf16 *a, bf16 *b, bf16 *y, long long npix, int Ca, int Cb, int split) {
  const int C = Ca + Cb;
  RF_GRID_STRIDE(i, npix * C) {
    const int c = (int)(i % C);
    const long long p = i / C;
    bf16 *src = (c < Ca) ? a + p * Ca + c : b + p * Cb + (c - Ca);
    if (split) *src = y[i];
    else y[i] = *src;
  }
}

// dy *= (y > 0)
__global__ void relu_bwd_kernel(bf16 *dy, const bf16 *y, long long n) {
  RF_GRID_STRIDE(i, n) {
    if (!(__bfloat162float(y[i]) > 0.0f)) dy[i] = __float2bfloat16(0.0f);
  }
}

// masked MSE on channel 0 of an FP32 prediction [npix][C]: loss = sum m (p -
// t)^2 / sum m; dp (BF16, [npix][C], zero outside channel 0) = 2 m (p - t) / sum m
__global__ void mse_kernel(const float *pred, int C, const float *target, const float *mask, long long npix,
                           float inv_count, bf16 *dpred, float *loss) {
  float s = 0.0f;
  RF_GRID_STRIDE(p, npix) {
    const float m = mask ? mask[p] : 1.0f;
    const float d = (pred[p * C] - target[p]) * m;
    s += d * d;
    dpred[p * C] = __float2bfloat16(2.0f * d * inv_count);
    for (int c = 1; c < C; ++c) dpred[p * C + c] = __float2bfloat16(0.0f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_count);
}

// FP32 -> BF16 (master weights -> kernel weights)
__global__ void cast_bf16_kernel(const float *x, bf16 *y, long long n) {
  RF_GRID_STRIDE(i, n) y[i] = __float2bfloat16(x[i]);
}

// Network input: planes [B][Cp][H][W] (FP32) -> NHWC BF16 with C channels
// (the first Cp filled, the rest zero)
__global__ void pack_input_kernel(const float *planes, int Cp, bf16 *y, int B, int H, int W, int C) {
  const long long n = (long long)B * H * W * C;
  RF_GRID_STRIDE(i, n) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const long long hw = q % ((long long)H * W);
    const int b = (int)(q / ((long long)H * W));
    y[i] = __float2bfloat16(c < Cp ? planes[((long long)b * Cp + c) * H * W + hw] : 0.0f);
  }
}

// y += x (BF16, accumulated in FP32)
__global__ void add_bf16_kernel(bf16 *y, const bf16 *x, long long n) {
  RF_GRID_STRIDE(i, n) y[i] = __float2bfloat16(__bfloat162float(y[i]) + __bfloat162float(x[i]));
}

// Nearest-source features of image b at pixel (i, j): distance to the
// nearest source and the displacement to it, in domain units (h per pixel);
// out [B][3][H][W].  Sources of image b: src_ij[src_off[b] .. src_off[b+1]).
__global__ void source_features_kernel(int B, int H, int W, float h, const int *src_ij, const int *src_off,
                                       float *out) {
  const long long n = (long long)B * H * W;
  RF_GRID_STRIDE(q, n) {
    const int j = (int)(q % W), i = (int)((q / W) % H), b = (int)(q / ((long long)H * W));
    float best = 3.0e38f, bx = 0.0f, by = 0.0f;
    for (int k = src_off[b]; k < src_off[b + 1]; ++k) {
      const float dy = (float)(i - src_ij[2 * k]) * h, dx = (float)(j - src_ij[2 * k + 1]) * h;
      const float d = dx * dx + dy * dy;
      if (d < best) {
        best = d;
        bx = dx;
        by = dy;
      }
    }
    const long long hw = (long long)H * W, o = (long long)b * 3 * hw + (long long)i * W + j;
    out[o] = best < 3.0e38f ? sqrtf(best) : 0.0f;
    out[o + hw] = bx;
    out[o + 2 * hw] = by;
  }
}

// Box average of FP32 planes [P][H][W] by an integer factor f -> [P][H/f][W/f]
__global__ void box_down_kernel(const float *x, float *y, int P, int H, int W, int f) {
  const int Ho = H / f, Wo = W / f;
  const long long n = (long long)P * Ho * Wo;
  RF_GRID_STRIDE(q, n) {
    const int jo = (int)(q % Wo), io = (int)((q / Wo) % Ho), p = (int)(q / ((long long)Wo * Ho));
    float s = 0.0f;
    for (int a = 0; a < f; ++a)
      for (int c = 0; c < f; ++c) s += x[((long long)p * H + io * f + a) * W + jo * f + c];
    y[q] = s / (float)(f * f);
  }
}

// Bilinear resampling of FP32 planes [P][Hi][Wi] -> [P][Ho][Wo], node-aligned
// (corner nodes map to corner nodes), scaled by `scale`.
__global__ void bilinear_kernel(const float *x, float *y, int P, int Hi, int Wi, int Ho, int Wo, float scale) {
  const long long n = (long long)P * Ho * Wo;
  const float ry = Ho > 1 ? (float)(Hi - 1) / (float)(Ho - 1) : 0.0f;
  const float rx = Wo > 1 ? (float)(Wi - 1) / (float)(Wo - 1) : 0.0f;
  RF_GRID_STRIDE(q, n) {
    const int jo = (int)(q % Wo), io = (int)((q / Wo) % Ho), p = (int)(q / ((long long)Wo * Ho));
    const float fy = io * ry, fx = jo * rx;
    const int y0 = min((int)fy, Hi - 1), x0 = min((int)fx, Wi - 1);
    const int y1 = min(y0 + 1, Hi - 1), x1 = min(x0 + 1, Wi - 1);
    const float ty = fy - y0, tx = fx - x0;
    const float *b = x + (long long)p * Hi * Wi;
    const float v = (1 - ty) * ((1 - tx) * b[(long long)y0 * Wi + x0] + tx * b[(long long)y0 * Wi + x1]) +
                    ty * ((1 - tx) * b[(long long)y1 * Wi + x0] + tx * b[(long long)y1 * Wi + x1]);
    y[q] = scale * v;
  }
}

}  // namespace rf

using namespace rf;

namespace {

inline bool ch_ok(int c) { return c >= 16 && c % 16 == 0; }
inline int ew_blocks(rf_ctx *ctx, long long n) { return blocks_for(n, 256, ctx->num_sms * 16); }
inline rf_status begin(rf_ctx *ctx, void *stream) {
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  ctx->last_stream = (cudaStream_t)stream;
  return RF_OK;
}

}  // namespace

extern "C" rf_status rf_unet_conv3x3(rf_ctx *ctx, const uint16_t *x, int B, int H, int W, int Cin, const uint16_t *w,
                                     const float *bias, int Cout, int relu, uint16_t *y, float *y32, void *stream) {
  if (!ctx || !x || !w || !y || B < 1 || H < 1 || W < 1 || !ch_ok(Cin) || !ch_ok(Cout)) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  ConvArgs a;
  a.x = (const bf16 *)x;
  a.w = (const bf16 *)w;
  a.bias = bias;
  a.y = (bf16 *)y;
  a.y32 = y32;
  a.B = B;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  a.relu = relu;
  const int tiles = ((W + kCvTW - 1) / kCvTW) * ((H + kCvTH - 1) / kCvTH);
  if (B > 65535) return RF_ERR_INVALID_ARG;
  dim3 grid(tiles, (Cout + kCvBN - 1) / kCvBN, B);
  conv3x3_fwd_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(a);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_conv3x3_wgrad(rf_ctx *ctx, const uint16_t *x, const uint16_t *dy, int B, int H, int W,
                                           int Cin, int Cout, float *dw, void *stream) {
  if (!ctx || !x || !dy || !dw || B < 1 || H < 1 || W < 1 || !ch_ok(Cin) || !ch_ok(Cout)) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  WgradArgs a;
  a.x = (const bf16 *)x;
  a.dy = (const bf16 *)dy;
  a.dw = dw;
  a.B = B;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  const long long zdim = (long long)B * ((H + kWgRows - 1) / kWgRows);
  if (zdim > 65535) return RF_ERR_INVALID_ARG;
  dim3 grid((Cout + 31) / 32, Cin / 16, (unsigned)zdim);
  conv3x3_wgrad_kernel<<<grid, 96, 0, (cudaStream_t)stream>>>(a);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_bias_grad(rf_ctx *ctx, const uint16_t *dy, int64_t npix, int C, float *db, void *stream) {
  if (!ctx || !dy || !db || npix < 1 || C < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  dim3 grid((unsigned)std::min<long long>((npix + 7) / 8, 2048), (C + 31) / 32);
  bias_grad_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const bf16 *)dy, npix, C, db);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_flip_weights(rf_ctx *ctx, const uint16_t *w, int Cin, int Cout, uint16_t *wt,
                                          void *stream) {
  if (!ctx || !w || !wt || Cin < 1 || Cout < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  const long long n = (long long)Cout * 9 * Cin;
  flip_weights_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)w, (bf16 *)wt, Cin, Cout);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_maxpool2(rf_ctx *ctx, const uint16_t *x, int B, int H, int W, int C, uint16_t *y,
                                      uint8_t *arg, void *stream) {
  if (!ctx || !x || !y || !arg || B < 1 || H < 2 || W < 2 || (H & 1) || (W & 1) || C < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  const long long n = (long long)B * (H / 2) * (W / 2) * C;
  maxpool2_fwd_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, (bf16 *)y, arg, B, H, W,
                                                                             C);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_maxpool2_backward(rf_ctx *ctx, const uint16_t *dy, const uint8_t *arg, int B, int H,
                                               int W, int C, uint16_t *dx, void *stream) {
  if (!ctx || !dy || !arg || !dx || B < 1 || H < 2 || W < 2 || (H & 1) || (W & 1) || C < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  const long long n = (long long)B * (H / 2) * (W / 2) * C;
  maxpool2_bwd_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)dy, arg, (bf16 *)dx, B, H,
                                                                             W, C);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_upsample2(rf_ctx *ctx, const uint16_t *x, int B, int H, int W, int C, uint16_t *y,
                                       void *stream) {
  if (!ctx || !x || !y || B < 1 || H < 1 || W < 1 || C < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  const long long n = 4LL * B * H * W * C;
  upsample2_fwd_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, (bf16 *)y, B, H, W, C);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_upsample2_backward(rf_ctx *ctx, const uint16_t *dy, int B, int H, int W, int C,
                                                uint16_t *dx, void *stream) {
  if (!ctx || !dy || !dx || B < 1 || H < 1 || W < 1 || C < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  const long long n = (long long)B * H * W * C;
  upsample2_bwd_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)dy, (bf16 *)dx, B, H, W,
                                                                              C);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_concat(rf_ctx *ctx, uint16_t *a, int Ca, uint16_t *b, int Cb, int64_t npix, uint16_t *y,
                                    int split, void *stream) {
  if (!ctx || !a || !b || !y || Ca < 1 || Cb < 1 || npix < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  concat_kernel<<<ew_blocks(ctx, npix * (Ca + Cb)), 256, 0, (cudaStream_t)stream>>>((bf16 *)a, (bf16 *)b, (bf16 *)y,
                                                                                     npix, Ca, Cb, split);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_relu_backward(rf_ctx *ctx, uint16_t *dy, const uint16_t *y, int64_t n, void *stream) {
  if (!ctx || !dy || !y || n < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  relu_bwd_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>((bf16 *)dy, (const bf16 *)y, n);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_mse(rf_ctx *ctx, const float *pred32, int C, const float *target, const float *mask,
                                 int64_t npix, float count, uint16_t *dpred, float *loss, void *stream) {
  if (!ctx || !pred32 || !target || !dpred || !loss || C < 1 || npix < 1 || !(count > 0.0f)) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  mse_kernel<<<ew_blocks(ctx, npix), 256, 0, (cudaStream_t)stream>>>(pred32, C, target, mask, npix, 1.0f / count,
                                                                       (bf16 *)dpred, loss);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_cast_bf16(rf_ctx *ctx, const float *x, uint16_t *y, int64_t n, void *stream) {
  if (!ctx || !x || !y || n < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  cast_bf16_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>(x, (bf16 *)y, n);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_pack_input(rf_ctx *ctx, const float *planes, int Cp, int B, int H, int W, int C,
                                        uint16_t *y, void *stream) {
  if (!ctx || !planes || !y || Cp < 1 || Cp > C || B < 1 || H < 1 || W < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  const long long n = (long long)B * H * W * C;
  pack_input_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>(planes, Cp, (bf16 *)y, B, H, W, C);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_add(rf_ctx *ctx, uint16_t *y, const uint16_t *x, int64_t n, void *stream) {
  if (!ctx || !y || !x || n < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  add_bf16_kernel<<<ew_blocks(ctx, n), 256, 0, (cudaStream_t)stream>>>((bf16 *)y, (const bf16 *)x, n);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_source_features(rf_ctx *ctx, int B, int H, int W, float h, const int32_t *src_ij,
                                             const int32_t *src_off, float *out, void *stream) {
  if (!ctx || !src_ij || !src_off || !out || B < 1 || H < 1 || W < 1 || !(h > 0.0f)) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  source_features_kernel<<<ew_blocks(ctx, (long long)B * H * W), 256, 0, (cudaStream_t)stream>>>(B, H, W, h, src_ij,
                                                                                                  src_off, out);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_box_down(rf_ctx *ctx, const float *x, int P, int H, int W, int f, float *y,
                                      void *stream) {
  if (!ctx || !x || !y || P < 1 || f < 1 || H < f || W < f || H % f || W % f) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  box_down_kernel<<<ew_blocks(ctx, (long long)P * (H / f) * (W / f)), 256, 0, (cudaStream_t)stream>>>(x, y, P, H, W,
                                                                                                      f);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_unet_bilinear(rf_ctx *ctx, const float *x, int P, int Hi, int Wi, int Ho, int Wo, float scale,
                                      float *y, void *stream) {
  if (!ctx || !x || !y || P < 1 || Hi < 1 || Wi < 1 || Ho < 1 || Wo < 1) return RF_ERR_INVALID_ARG;
  rf_status rs = begin(ctx, stream);
  if (rs != RF_OK) return rs;
  bilinear_kernel<<<ew_blocks(ctx, (long long)P * Ho * Wo), 256, 0, (cudaStream_t)stream>>>(x, y, P, Hi, Wi, Ho, Wo,
                                                                                             scale);
  return cuda_status(cudaGetLastError());
}
