// rf_unet_wgrad_tc.cu -- the warm-start network's weight gradient on the
// fifth-generation tensor cores.
//
// dw[co][tap][ci] += sum over pixels p of dy[p][co] * x[p + tap offset][ci]:
// for each of the 9 taps a GEMM with M = output channels, N = input
// channels and K = pixels.  A CTA owns 128 output channels (rows beyond
// Cout are zero), N input channels (32, or 16 when Cin is not a multiple of
// 32) and a range of image rows; its 9 accumulators (9 x N FP32 columns)
// live in tensor memory for the whole range.  K advances in chunks of one
// 64-pixel row segment.
//
// Both operands are used as they lie in memory (NHWC: channels contiguous
// per pixel), in the MN-major no-swizzle canonical layout: a core matrix is
// 8 pixels (K) x 8 channels (MN), 16 bytes per pixel row, 128 contiguous
// bytes; core matrices adjacent along K are 128 bytes apart (leading byte
// offset), along MN one channel plane apart (stride byte offset).
// * A (dy): 16 planes of 8 output channels, each [64 px][8 ch];
// * B (x): for rows y-1, y, y+1, N/8 planes of 8 input channels, each
//   [66 px][8 ch] (pixels x0-1 .. x0+64); the operand of tap (ky, kx)
//   starts kx pixels (16 kx bytes) into row ky's planes, so the 9 taps
//   share one staged copy.
// Chunks arrive in a ring of 3 stages by cp.async (zero-filled outside the
// image); one thread issues each chunk's 9 x 4 MMAs (K = 16) and commits
// them to the stage's mbarrier, which the threads wait on (bounded by the
// context timeout) before the stage is refilled.  The epilogue reads the
// accumulators with tcgen05.ld (warp w: TMEM lanes 32w .. 32w+31 = output
// channels) and adds them to dw.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "rf_ctx.h"

namespace rf {
namespace wtc {

using bf16 = __nv_bfloat16;

constexpr int kM = 128;          // output channels per CTA (MMA M)
constexpr int kSeg = 64;         // pixels per chunk (4 MMA K-steps)
constexpr int kHalo = kSeg + 2;  // staged x pixels per row
constexpr int kThreads = 128;
constexpr int kStages = 3;
constexpr unsigned kAPlane = kSeg * 16;   // one 8-channel plane of dy
constexpr unsigned kBPlane = kHalo * 16;  // one 8-channel plane of an x row

__host__ __device__ constexpr unsigned a_bytes() { return (kM / 8) * kAPlane; }
__host__ __device__ constexpr unsigned b_bytes(int N) { return 3u * (unsigned)(N / 8) * kBPlane; }
__host__ __device__ constexpr unsigned stage_bytes(int N) { return a_bytes() + b_bytes(N); }
__host__ __device__ constexpr size_t smem_bytes(int N) { return (size_t)kStages * stage_bytes(N) + kStages * 8 + 16; }

__device__ __forceinline__ unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), version 1 (46-47),
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// kind::f16 instruction descriptor: D FP32, A and B BF16, both MN-major
// (bits 15 and 16), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_mn(int N, int M) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *m, unsigned parity, long long timeout_ns) {
  if (mbar_try_wait(m, parity)) return true;
  const unsigned long long t0 = gtimer_ns();
  while (!mbar_try_wait(m, parity))
    if ((long long)(gtimer_ns() - t0) > timeout_ns) return false;
  return true;
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *m) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(m))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros
__device__ __forceinline__ void cp_async16(void *dst, const void *src, unsigned src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

struct Args {
  const bf16 *x;   // [B][H][W][Cin]
  const bf16 *dy;  // [B][H][W][Cout]
  float *dw;       // [Cout][9][Cin], accumulated
  int B, H, W, Cin, Cout;
  int rows_per;    // image rows (of all B x H) per CTA
  DevState *st;
  long long timeout_ns;
};

template <int N>
__device__ __forceinline__ void stage_chunk(const Args &a, unsigned char *st, int co0, int ci0, int row, int seg) {
  constexpr int NP = N / 8;
  const int b = row / a.H, y = row - b * a.H, x0 = seg * kSeg;
  const int tid = threadIdx.x;
  unsigned char *As = st;
  unsigned char *Bs = st + a_bytes();
  // A: dy [64 px][128 co] as 16 planes [px][8 co]
  for (int f = tid; f < (kM / 8) * kSeg; f += kThreads) {
    const int q = f / kSeg, px = f - q * kSeg;
    const int gx = x0 + px, co = co0 + 8 * q;
    const bool ok = gx < a.W && co < a.Cout;
    const bf16 *src = ok ? a.dy + (((long long)b * a.H + y) * a.W + gx) * a.Cout + co : a.dy;
    cp_async16(As + q * kAPlane + px * 16, src, ok ? 16u : 0u);
  }
  // B: x rows y-1 .. y+1, pixels x0-1 .. x0+64, as 3 x NP planes [px][8 ci]
  for (int f = tid; f < 3 * NP * kHalo; f += kThreads) {
    const int rq = f / kHalo, px = f - rq * kHalo;
    const int r = rq / NP, q = rq - r * NP;
    const int gy = y + r - 1, gx = x0 - 1 + px;
    const bool ok = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
    const bf16 *src = ok ? a.x + (((long long)b * a.H + gy) * a.W + gx) * a.Cin + ci0 + 8 * q : a.x;
    cp_async16(Bs + (r * NP + q) * kBPlane + px * 16, src, ok ? 16u : 0u);
  }
}

template <int N>
__global__ void __launch_bounds__(kThreads, 1) wgrad_tc_kernel(Args a) {
  extern __shared__ __align__(128) unsigned char sm[];
  constexpr int NP = N / 8;
  constexpr unsigned kCols = (9 * N <= 256) ? 256u : 512u;  // TMEM: a power of two >= 9 N
  constexpr uint32_t idesc = idesc_mn(N, kM);
  constexpr unsigned SB = stage_bytes(N);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + kStages * SB);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + kStages);
  __shared__ int s_late;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int co0 = blockIdx.x * kM, ci0 = blockIdx.y * N;
  const int rows = a.B * a.H;
  const int r0 = blockIdx.z * a.rows_per, r1 = min(rows, r0 + a.rows_per);
  const int nseg = (a.W + kSeg - 1) / kSeg;
  const int nc = r1 > r0 ? (r1 - r0) * nseg : 0;

  if (warp == 0) tmem_alloc(tslot, kCols);
  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(mbar + k, 1);
    fence_mbar_init();
    s_late = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  for (int c = 0; c < 2; ++c) {
    if (c < nc) stage_chunk<N>(a, sm + c * SB, co0, ci0, r0 + c / nseg, c % nseg);
    cp_async_commit();
  }
  int c = 0;
  for (; c < nc; ++c) {
    cp_async_wait<1>();  // chunk c has landed (all groups but the newest)
    fence_proxy_async();  // the tensor cores read shared memory through the async proxy
    __syncthreads();
    if (s_late) break;
    const int s = c % kStages;
    if (tid == 0) {
      fence_after();
      const unsigned abase = saddr(sm + s * SB), bbase = abase + a_bytes();
      for (int t = 0; t < 9; ++t) {
        const int ky = t / 3, kx = t - 3 * ky;
#pragma unroll
        for (int ks = 0; ks < kSeg / 16; ++ks) {
          const uint64_t ad = smem_desc(abase + ks * 256, 128, kAPlane);
          const uint64_t bd = smem_desc(bbase + ky * NP * kBPlane + (16 * ks + kx) * 16, 128, kBPlane);
          mma_bf16(tmem + (uint32_t)(t * N), ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
        }
      }
      mma_commit(mbar + s);
    }
    // refill the stage of chunk c - 1 with chunk c + 2 once its MMAs are done
    if (c >= 1) {
      const int cp = c - 1;
      if (!mbar_wait(mbar + cp % kStages, (unsigned)(cp / kStages) & 1u, a.timeout_ns)) atomicExch(&s_late, 1);
    }
    if (c + 2 < nc && !s_late)
      stage_chunk<N>(a, sm + ((c + 2) % kStages) * SB, co0, ci0, r0 + (c + 2) / nseg, (c + 2) % nseg);
    cp_async_commit();
  }
  cp_async_wait<0>();
  __syncthreads();
  bool ok = !s_late;
  if (nc > 0) {
    // the last chunk's commit covers every MMA issued before it
    const int cl = (ok ? nc : c) - 1;
    if (cl >= 0 && !mbar_wait(mbar + cl % kStages, (unsigned)(cl / kStages) & 1u, a.timeout_ns)) ok = false;
  }
  if (!ok && tid == 0) set_error(a.st, RF_ERR_TIMEOUT);
  ok = __syncthreads_and(ok);
  fence_after();
  if (ok && nc > 0) {
    const int co = co0 + warp * 32 + lane;
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
#pragma unroll
      for (int cb = 0; cb < N; cb += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * N + cb), r);
        if (co < a.Cout) {
          float *d = a.dw + ((long long)co * 9 + t) * a.Cin + ci0 + cb;
#pragma unroll
          for (int j = 0; j < 16; ++j) atomicAdd(d + j, __uint_as_float(r[j]));
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

}  // namespace wtc
}  // namespace rf

using namespace rf;

extern "C" rf_status rf_unet_conv3x3_wgrad_tc(rf_ctx *ctx, const uint16_t *x, const uint16_t *dy, int B, int H,
                                              int W, int Cin, int Cout, float *dw, void *stream) {
  if (!ctx || !x || !dy || !dw || B < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 || Cout < 16 || Cout % 16)
    return RF_ERR_INVALID_ARG;
  if ((((uintptr_t)x) | ((uintptr_t)dy)) & 15) return RF_ERR_INVALID_ARG;  // 16-byte copies
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  wtc::Args a;
  a.x = (const wtc::bf16 *)x;
  a.dy = (const wtc::bf16 *)dy;
  a.dw = dw;
  a.B = B;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  a.st = ctx->state;
  a.timeout_ns = ctx->timeout_ns;
  const int N = (Cin % 32 == 0) ? 32 : 16;
  const int co_tiles = (Cout + wtc::kM - 1) / wtc::kM, ci_tiles = Cin / N;
  // about two CTAs per SM over the pixel rows (at least one row each)
  const long long rows = (long long)B * H;
  const long long want = std::max<long long>(1, (2LL * ctx->num_sms + co_tiles * ci_tiles - 1) / (co_tiles * ci_tiles));
  a.rows_per = (int)std::max<long long>(1, (rows + want - 1) / want);
  const long long groups = (rows + a.rows_per - 1) / a.rows_per;
  if (groups > 65535) return RF_ERR_INVALID_ARG;
  dim3 grid(co_tiles, ci_tiles, (unsigned)groups);
  cudaError_t e;
  if (N == 32) {
    const size_t smem = wtc::smem_bytes(32);
    e = cudaFuncSetAttribute(wtc::wgrad_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      wtc::wgrad_tc_kernel<32><<<grid, wtc::kThreads, smem, s>>>(a);
      e = cudaGetLastError();
    }
  } else {
    const size_t smem = wtc::smem_bytes(16);
    e = cudaFuncSetAttribute(wtc::wgrad_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      wtc::wgrad_tc_kernel<16><<<grid, wtc::kThreads, smem, s>>>(a);
      e = cudaGetLastError();
    }
  }
  return e == cudaSuccess ? RF_OK : RF_ERR_CUDA;
}
