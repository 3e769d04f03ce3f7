// rf_unet_tc.cu -- the warm-start network's 3x3 convolution on the fifth-
// generation tensor cores: tcgen05.mma with BF16 operands in shared memory
// and the FP32 accumulator in tensor memory (TMEM).
//
// Implicit GEMM per CTA: D[128 pixels][N out-channels] = sum over the 9 taps
// and the input channels of A_tap[128][Cin] * B_tap[N][Cin]^T, where the 128
// pixels are an 8 x 16 output tile and A_tap is the input patch shifted by
// the tap.  Input channels are processed in chunks of CC (16 or 32).
//
// Shared-memory operands use the no-swizzle K-major canonical layout: a
// core matrix is 8 rows x 8 BF16 (16 bytes per row, 128 contiguous bytes).
// * A: three copies of the 10 x 16 input patch, one per column tap kx
//   (columns kx .. kx+15 of the 18-wide halo patch), stored
//   [kx][c8][row 0..9][col 0..15][8 channels].  For tap (ky, kx) the
//   matrix starts at row ky of copy kx; its 128 rows (8 rows x 16 columns
//   of pixels) are 16 consecutive core matrices 128 bytes apart (stride
//   byte offset 128, a patch row being 2 core matrices), and the second 8
//   channels of an MMA's K = 16 sit one channel plane (10 x 16 x 16 B =
//   2560 B) further (leading byte offset).
// * B: the chunk's weights [tap][c8][n][8 channels]: N rows 16 bytes apart
//   (stride byte offset 128 per 8 rows), next 8 channels one c8 plane
//   (N x 16 B) further.
// One thread issues the 9 x CC/16 MMAs of a chunk and commits them to an
// mbarrier; all threads wait (bounded) before the chunk's buffers are
// rewritten.  The epilogue reads the accumulator with tcgen05.ld (warp w
// owns TMEM lanes 32w .. 32w+31 = pixels 32w ..), adds the bias, applies
// ReLU and stores BF16 (and optionally FP32).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "rf_ctx.h"

namespace rf {
namespace tc {

using bf16 = __nv_bfloat16;

constexpr int kTH = 8, kTW = 16;  // output tile 8 x 16 = 128 pixels = MMA M
constexpr int kPH = kTH + 2;      // patch rows
constexpr int kThreads = 128;     // 4 warps: one per 32 TMEM lanes
constexpr unsigned kPlaneBytes = kPH * kTW * 16;  // one 8-channel plane of a patch copy

__device__ __forceinline__ unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (PTX ISA, tcgen05 matrix descriptors):
// start address >> 4 in bits 0-13, leading byte offset >> 4 in 16-29,
// stride byte offset >> 4 in 32-45, descriptor version 1 in 46-47, base
// offset 0, layout type 0 (no swizzle) in 61-63.
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor for kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28, dense, no negation.
__host__ __device__ constexpr uint32_t idesc_bf16(int N, int M) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
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
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
  const bf16 *x;      // [B][H][W][Cin]
  const bf16 *w;      // [Cout][9][Cin]
  const float *bias;  // [Cout] or null
  bf16 *wpack;        // Cout * 9 * Cin scratch for the packed weights (persistent kernel)
  bf16 *y;            // [B][H][W][Cout]
  float *y32;         // optional FP32 copy
  int B, H, W, Cin, Cout, relu, CC;
  DevState *st;
  long long timeout_ns;
};

__host__ __device__ inline size_t tc_smem_bytes(int CC, int N) {
  const size_t a = (size_t)3 * (CC / 8) * kPlaneBytes, b = (size_t)9 * (CC / 8) * N * 16;
  return a + b + 16;  // + mbarrier and TMEM slot
}

template <int N>
__global__ void __launch_bounds__(kThreads, 2) conv3x3_tc_kernel(TcArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  constexpr unsigned kCols = N < 32 ? 32 : N;  // TMEM columns: a power of two >= 32
  const int CC = a.CC, c8n = CC / 8;
  const unsigned a_copy = (unsigned)c8n * kPlaneBytes;
  bf16 *As = reinterpret_cast<bf16 *>(sm);
  bf16 *Bs = reinterpret_cast<bf16 *>(sm + 3 * a_copy);
  const unsigned b_bytes = 9u * c8n * N * 16;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 3 * a_copy + b_bytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  __shared__ int s_late;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = (a.W + kTW - 1) / kTW;
  const int tx0 = (blockIdx.x % tiles_x) * kTW, ty0 = (blockIdx.x / tiles_x) * kTH;
  const int n0 = blockIdx.y * N, b = blockIdx.z;
  const int H = a.H, W = a.W, Cin = a.Cin, Cout = a.Cout;

  if (warp == 0) tmem_alloc(tslot, kCols);
  if (tid == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
    s_late = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = idesc_bf16(N, 128);

  unsigned phase = 0;
  for (int c0 = 0; c0 < Cin && !s_late; c0 += CC) {
    // A: patch copies [kx][c8][row][col][8 ch] from x (zero outside the image)
    const int na = 3 * c8n * kPH * kTW;
    for (int f = tid; f < na; f += kThreads) {
      const int col = f % kTW;
      int r = f / kTW;
      const int row = r % kPH;
      r /= kPH;
      const int c8 = r % c8n, kx = r / c8n;
      const int gy = ty0 + row - 1, gx = tx0 + col + kx - 1;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gy >= 0 && gy < H && gx >= 0 && gx < W)
        v = *reinterpret_cast<const uint4 *>(a.x + (((long long)b * H + gy) * W + gx) * Cin + c0 + c8 * 8);
      *reinterpret_cast<uint4 *>(As + ((size_t)((kx * c8n + c8) * kPH + row) * kTW + col) * 8) = v;
    }
    // B: weights [tap][c8][n][8 ch] of output channels n0 .. n0+N-1
    const int nb = 9 * c8n * N;
    for (int f = tid; f < nb; f += kThreads) {
      const int n = f % N;
      int r = f / N;
      const int c8 = r % c8n, t = r / c8n;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (n0 + n < Cout) v = *reinterpret_cast<const uint4 *>(a.w + ((long long)(n0 + n) * 9 + t) * Cin + c0 + c8 * 8);
      *reinterpret_cast<uint4 *>(Bs + ((size_t)(t * c8n + c8) * N + n) * 8) = v;
    }
    fence_proxy_async();  // the tensor cores read shared memory through the async proxy
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const unsigned abase = saddr(As), bbase = saddr(Bs);
      for (int t = 0; t < 9; ++t) {
        const int ky = t / 3, kx = t % 3;
        for (int ks = 0; ks < CC / 16; ++ks) {
          const unsigned aaddr = abase + kx * a_copy + (2 * ks) * kPlaneBytes + ky * (kTW * 16);
          const unsigned baddr = bbase + (unsigned)((t * c8n + 2 * ks) * N * 16);
          mma_bf16(tmem, smem_desc(aaddr, kPlaneBytes, 128), smem_desc(baddr, N * 16, 128), idesc,
                   (c0 > 0 || t > 0 || ks > 0) ? 1u : 0u);
        }
      }
      mma_commit(mbar);
      // wait (bounded) for the chunk's MMAs: they read the buffers the next
      // chunk rewrites, and the epilogue reads their result
      if (!mbar_wait(mbar, phase, a.timeout_ns)) s_late = 1;
    }
    phase ^= 1u;
    __syncthreads();
    fence_after();
  }
  if (s_late) {
    // the chunk's MMAs did not report completion within the bound: record
    // it, then wait once more (bounded) before the accumulator is freed
    if (tid == 0) {
      set_error(a.st, RF_ERR_TIMEOUT);
      mbar_wait(mbar, phase ^ 1u, a.timeout_ns);
    }
    __syncthreads();
  } else {
    // epilogue: pixel m = 32 warp + lane of the tile, accumulator row m
    const int m = warp * 32 + lane, gy = ty0 + m / kTW, gx = tx0 + m % kTW;
    const bool in = gy < H && gx < W;
    const long long obase = (((long long)b * H + gy) * W + gx) * Cout + n0;
#pragma unroll
    for (int cb = 0; cb < N; cb += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, r);
      if (in && n0 + cb < Cout) {  // Cout is a multiple of 16: all 16 columns are in range
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] = __uint_as_float(r[j]) + (a.bias ? a.bias[n0 + cb + j] : 0.0f);
          if (a.relu) v[j] = fmaxf(v[j], 0.0f);
        }
        uint4 pk[2];
        __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
        for (int j = 0; j < 8; ++j) h2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        uint4 *dst = reinterpret_cast<uint4 *>(a.y + obase + cb);
        dst[0] = pk[0];
        dst[1] = pk[1];
        if (a.y32) {
          float4 *d32 = reinterpret_cast<float4 *>(a.y32 + obase + cb);
#pragma unroll
          for (int j = 0; j < 4; ++j) d32[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------------------
// Pipelined form: the operand tiles arrive by tensor copies
// (cp.async.bulk.tensor) into a ring of STAGES buffers, 16 input channels
// per stage, while the tensor cores consume earlier stages.
//  * warp 0 (producer): per stage, lane 0 arms the stage's "full" barrier
//    with the stage's bytes, then 6 lanes copy the A planes (3 column taps
//    x 2 channel planes, box 8 ch x 16 cols x 10 rows from the NHWC input,
//    zero-filled outside the image) and 18 lanes the B planes (9 taps x 2
//    channel planes, box 8 ch x N out-channels); it reuses a stage once
//    the MMAs that read it have committed to its "empty" barrier;
//  * warp 1, lane 0 (MMA issuer): waits for a stage, issues its 9 MMAs
//    (one per tap, K = 16), commits them to the stage's empty barrier, and
//    after the last stage commits to the "done" barrier;
//  * all 4 warps: epilogue from TMEM as in conv3x3_tc_kernel.
// Every wait is bounded by the context timeout; a timeout records
// RF_ERR_TIMEOUT and the CTA drains what it issued before freeing TMEM.
constexpr int kStages = 4;

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *m) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(saddr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(m))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *m) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          saddr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(m))
      : "memory");
}

// One contiguous copy (cp.async.bulk, not tensor-mapped): both addresses
// 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(m))
               : "memory");
}

struct TmaArgs {
  const bf16 *wpack;  // persistent kernel: the weights in stage order (pack_w_kernel)
  const float *bias;
  bf16 *y;
  float *y32;
  int B, H, W, Cin, Cout, relu;
  DevState *st;
  long long timeout_ns;
};

__host__ __device__ constexpr unsigned stage_a_bytes() { return 3u * 2u * kPlaneBytes; }
__host__ __device__ constexpr unsigned stage_b_bytes(int N) { return 9u * 2u * (unsigned)N * 16u; }
__host__ __device__ constexpr size_t tma_smem_bytes(int N) {
  return (size_t)kStages * (stage_a_bytes() + stage_b_bytes(N)) + (2 * kStages + 1) * 8 + 16;
}

template <int N>
__global__ void __launch_bounds__(kThreads, 1)
    conv3x3_tma_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap,
                       TmaArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  constexpr unsigned kCols = N < 32 ? 32 : N;
  constexpr unsigned SA = stage_a_bytes(), SB = stage_b_bytes(N), SS = SA + SB;
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + kStages * SS);
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  __shared__ int s_late;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = (a.W + kTW - 1) / kTW;
  const int tx0 = (blockIdx.x % tiles_x) * kTW, ty0 = (blockIdx.x / tiles_x) * kTH;
  const int n0 = blockIdx.y * N, b = blockIdx.z;
  const int nchunks = a.Cin / 16;

  if (warp == 0) tmem_alloc(tslot, kCols);
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
    s_late = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  int issued = 0;  // producer: chunks whose copies were issued

  if (warp == 0) {
    for (int i = 0; i < nchunks; ++i) {
      const int st = i % kStages;
      const unsigned u = (unsigned)(i / kStages);
      int ok = 1;
      if (lane == 0 && i >= kStages) ok = mbar_wait(&empty[st], (u - 1u) & 1u, a.timeout_ns);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) s_late = 1;
        break;
      }
      unsigned char *sa = sm + st * SS, *sb = sa + SA;
      if (lane == 0) mbar_arrive_tx(&full[st], SA + SB);
      __syncwarp();
      const int c8_0 = i * 2;  // first 8-channel plane of this chunk
      if (lane < 6) {
        const int kx = lane >> 1, c8 = lane & 1;
        tma_load_4d(sa + (kx * 2 + c8) * kPlaneBytes, &xmap, (c8_0 + c8) * 8, tx0 + kx - 1, ty0 - 1, b, &full[st]);
      } else if (lane < 24) {
        const int j = lane - 6, t = j >> 1, c8 = j & 1;
        tma_load_3d(sb + (t * 2 + c8) * N * 16, &wmap, (c8_0 + c8) * 8, t, n0, &full[st]);
      }
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(N, 128);
    int i = 0;
    for (; i < nchunks; ++i) {
      const int st = i % kStages;
      const unsigned u = (unsigned)(i / kStages);
      if (!mbar_wait(&full[st], u & 1u, a.timeout_ns)) {
        s_late = 1;
        break;
      }
      fence_after();
      const unsigned abase = saddr(sm + st * SS), bbase = abase + SA;
      for (int t = 0; t < 9; ++t) {
        const int ky = t / 3, kx = t % 3;
        // A: copy kx = planes (kx, c8 0) and (kx, c8 1), 2560 B apart; row ky
        const unsigned aaddr = abase + (kx * 2) * kPlaneBytes + ky * (kTW * 16);
        const unsigned baddr = bbase + (unsigned)(t * 2 * N * 16);
        mma_bf16(tmem, smem_desc(aaddr, kPlaneBytes, 128), smem_desc(baddr, N * 16, 128), idesc,
                 (i > 0 || t > 0) ? 1u : 0u);
      }
      mma_commit(&empty[st]);
    }
    mma_commit(done);  // tracks every MMA issued above
  }
  // all warps: wait for the accumulator (bounded)
  if (tid == 0 && !mbar_wait(done, 0u, a.timeout_ns)) s_late = 1;
  __syncthreads();
  if (s_late) {
    if (tid == 0) {
      set_error(a.st, RF_ERR_TIMEOUT);
      // drain: the copies of every issued stage and the MMAs (bounded)
      for (int st = 0; st < kStages; ++st) mbar_wait(&full[st], 0u, a.timeout_ns);
      mbar_wait(done, 0u, a.timeout_ns);
    }
    __syncthreads();
  } else {
    fence_after();
    const int m = warp * 32 + lane, gy = ty0 + m / kTW, gx = tx0 + m % kTW;
    const bool in = gy < a.H && gx < a.W;
    const long long obase = (((long long)b * a.H + gy) * a.W + gx) * a.Cout + n0;
#pragma unroll
    for (int cb = 0; cb < N; cb += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, r);
      if (in && n0 + cb < a.Cout) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] = __uint_as_float(r[j]) + (a.bias ? a.bias[n0 + cb + j] : 0.0f);
          if (a.relu) v[j] = fmaxf(v[j], 0.0f);
        }
        uint4 pk[2];
        __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
        for (int j = 0; j < 8; ++j) h2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        uint4 *dst = reinterpret_cast<uint4 *>(a.y + obase + cb);
        dst[0] = pk[0];
        dst[1] = pk[1];
        if (a.y32) {
          float4 *d32 = reinterpret_cast<float4 *>(a.y32 + obase + cb);
#pragma unroll
          for (int j = 0; j < 4; ++j) d32[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
    }
  }
  (void)issued;
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------------------
// Persistent form: one CTA per SM walks the output tiles (8 x 16 pixels x N
// channels; consecutive tiles share their weights), with two accumulators
// in tensor memory so that a tile's epilogue overlaps the next tile's MMAs.
//  * warp 4 (producer): stage after stage, across tiles, as in
//    conv3x3_tma_kernel (16 input channels per stage, a ring of
//    persist_stages(N) stages);
//  * warp 5, lane 0 (MMA issuer): per tile, waits until the epilogue has
//    released the tile's accumulator (tiles alternate between the two),
//    issues 9 MMAs per stage, commits each stage to its "empty" barrier and
//    the tile to the accumulator's "full" barrier;
//  * warps 0-3 (epilogue; warp w reads TMEM lanes 32w .. 32w+31): wait for
//    the accumulator, add bias, ReLU, store, and release the accumulator
//    (one arrival per warp).
// Every wait is bounded by the context timeout; a timeout records
// RF_ERR_TIMEOUT, every role leaves its loop, and the CTA waits (bounded)
// for the MMAs it issued before freeing TMEM.
// P output tiles (8 x 16 pixels each) stacked vertically form one unit of
// the persistent kernel: they share each weight stage and one halo patch of
// 8P + 2 rows.
__host__ __device__ constexpr unsigned plane_bytes_p(int P) { return (unsigned)(kTH * P + 2) * kTW * 16; }
__host__ __device__ constexpr unsigned stage_a_bytes_p(int P) { return 3u * 2u * plane_bytes_p(P); }
__host__ __device__ constexpr int persist_stages(int N, int P) {
  return (int)((210u * 1024u) / (stage_a_bytes_p(P) + stage_b_bytes(N))) > 8
             ? 8
             : (int)((210u * 1024u) / (stage_a_bytes_p(P) + stage_b_bytes(N)));
}
__host__ __device__ constexpr size_t persist_smem_bytes(int N, int P) {
  return (size_t)persist_stages(N, P) * (stage_a_bytes_p(P) + stage_b_bytes(N)) + (2 * persist_stages(N, P) + 5) * 8 +
         16;
}
constexpr int kPersistThreads = 192;

__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(m)) : "memory");
}

struct TileIdx {
  int tx0, ty0, nt, b;
};
__device__ __forceinline__ TileIdx tile_of(int tile, int tiles_x, int tiles_pix, int ntn, int rows) {
  TileIdx r;
  const int pt = tile % tiles_pix, q = tile / tiles_pix;
  r.nt = q % ntn;
  r.b = q / ntn;
  r.tx0 = (pt % tiles_x) * kTW;
  r.ty0 = (pt / tiles_x) * rows;
  return r;
}

// Persistent form: one CTA per SM walks the units (P stacked 8 x 16 pixel
// tiles x N channels; consecutive units share their weights), with two sets
// of P accumulators in tensor memory so that a unit's epilogue overlaps the
// next unit's MMAs.
//  * warp 4 (producer): stage after stage, across units, the activation
//    planes as in conv3x3_tma_kernel (16 input channels per stage; the box
//    is 8P + 2 rows high), the weight planes by one bulk copy from the
//    packed weights (pack_w_kernel, launched before on the same stream) or,
//    without them, by tensor copies of 16-byte rows;
//  * warp 5, lane 0 (MMA issuer): per unit, waits until the epilogue has
//    released the unit's accumulator set, issues 9 P MMAs per stage (each
//    weight stage serves the P tiles), commits each stage to its "empty"
//    barrier and the unit to the set's "full" barrier;
//  * warps 0-3 (epilogue; warp w reads TMEM lanes 32w .. 32w+31): wait for
//    the set, add bias, ReLU, store, and release it (one arrival per warp).
// Every wait is bounded by the context timeout; a timeout records
// RF_ERR_TIMEOUT, every role leaves its loop, and the CTA waits (bounded)
// for the MMAs it issued before freeing TMEM.
// The weights [Cout][9][Cin] rearranged into the persistent kernel's stage
// order: block (nt, i) -- output channels nt N .. nt N + N - 1, input
// channels 16 i .. 16 i + 15 -- is [tap][8-channel half][n][8 channels],
// byte for byte the B planes a stage holds, so that one bulk copy of
// stage_b_bytes(N) fills them (the tensor-mapped loads of the same planes
// move 16-byte rows, 2 * 9 * N of them per stage).  One thread per 16 bytes.
template <int N>
__global__ void pack_w_kernel(const bf16 *__restrict__ w, bf16 *__restrict__ wp, int Cin, int Cout) {
  const int c8n = Cin / 8, nchunks = Cin / 16;
  const long long total = (long long)Cout * 9 * c8n;
  const uint4 *src = reinterpret_cast<const uint4 *>(w);
  uint4 *dst = reinterpret_cast<uint4 *>(wp);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total;
       j += (long long)gridDim.x * blockDim.x) {
    const int c8g = (int)(j % c8n);
    const long long r = j / c8n;  // co * 9 + tap
    const int t = (int)(r % 9), co = (int)(r / 9);
    const int nt = co / N, n = co % N, i = c8g >> 1, c8 = c8g & 1;
    dst[((((long long)nt * nchunks + i) * 9 + t) * 2 + c8) * N + n] = src[j];
  }
}

template <int N, int P>
__global__ void __launch_bounds__(kPersistThreads, 1)
    conv3x3_persist_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap,
                           TmaArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  constexpr int S = persist_stages(N, P);
  constexpr unsigned kCols = (2 * P * N) < 32 ? 32 : 2 * P * N;
  constexpr unsigned PB = plane_bytes_p(P);
  constexpr unsigned SA = stage_a_bytes_p(P), SB = stage_b_bytes(N), SS = SA + SB;
  static_assert(2 * P * N <= 512, "two accumulator sets fit in tensor memory");
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + S * SS);
  uint64_t *empty = full + S;
  uint64_t *tfull = empty + S;  // [2]
  uint64_t *tempty = tfull + 2;  // [2]
  uint64_t *done = tempty + 2;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  __shared__ int s_late;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int UR = kTH * P;  // pixel rows per unit
  const int tiles_x = (a.W + kTW - 1) / kTW, tiles_pix = tiles_x * ((a.H + UR - 1) / UR);
  const int ntn = a.Cout / N, ntiles = tiles_pix * ntn * a.B;
  const int nchunks = a.Cin / 16;

  if (warp == 0) tmem_alloc(tslot, kCols);
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&tfull[k], 1);
      mbar_init(&tempty[k], 4);
    }
    mbar_init(done, 1);
    fence_mbar_init();
    s_late = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 4) {
    int it = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const TileIdx ti = tile_of(tile, tiles_x, tiles_pix, ntn, UR);
      for (int i = 0; i < nchunks; ++i, ++it) {
        const int st = it % S;
        const unsigned u = (unsigned)(it / S);
        int good = 1;
        if (lane == 0 && it >= S) good = mbar_wait(&empty[st], (u - 1u) & 1u, a.timeout_ns);
        good = __shfl_sync(0xffffffffu, good, 0);
        if (!good || *(volatile int *)&s_late) {
          if (lane == 0) s_late = 1;
          ok = false;
          break;
        }
        unsigned char *sa = sm + st * SS, *sb = sa + SA;
        if (lane == 0) mbar_arrive_tx(&full[st], SS);
        __syncwarp();
        const int c8_0 = i * 2;
        if (lane < 6) {
          const int kx = lane >> 1, c8 = lane & 1;
          tma_load_4d(sa + (kx * 2 + c8) * PB, &xmap, (c8_0 + c8) * 8, ti.tx0 + kx - 1, ti.ty0 - 1, ti.b, &full[st]);
        } else if (a.wpack) {
          if (lane == 6) bulk_load(sb, a.wpack + ((size_t)ti.nt * nchunks + i) * (SB / 2), SB, &full[st]);
        } else if (lane < 24) {
          const int j = lane - 6, t = j >> 1, c8 = j & 1;
          tma_load_3d(sb + (t * 2 + c8) * N * 16, &wmap, (c8_0 + c8) * 8, t, ti.nt * N, &full[st]);
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(N, 128);
      int it = 0, tl = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tl) {
        const int buf = tl & 1;
        const unsigned ub = (unsigned)(tl >> 1);
        if (tl >= 2 && !mbar_wait(&tempty[buf], (ub - 1u) & 1u, a.timeout_ns)) {
          s_late = 1;
          break;
        }
        fence_after();
        for (int i = 0; i < nchunks; ++i, ++it) {
          const int st = it % S;
          const unsigned u = (unsigned)(it / S);
          if (!mbar_wait(&full[st], u & 1u, a.timeout_ns)) {
            s_late = 1;
            ok = false;
            break;
          }
          fence_after();
          const unsigned abase = saddr(sm + st * SS), bbase = abase + SA;
          for (int t = 0; t < 9; ++t) {
            const int ky = t / 3, kx = t % 3;
            const uint64_t bd = smem_desc(bbase + (unsigned)(t * 2 * N * 16), N * 16, 128);
#pragma unroll
            for (int h = 0; h < P; ++h) {
              // tile h: rows 8h + ky .. of copy kx (planes (kx, c8 0 / 1), PB apart)
              const unsigned aaddr = abase + (kx * 2) * PB + (kTH * h + ky) * (kTW * 16);
              mma_bf16(tmem + (uint32_t)((buf * P + h) * N), smem_desc(aaddr, PB, 128), bd, idesc,
                       (i > 0 || t > 0) ? 1u : 0u);
            }
          }
          mma_commit(&empty[st]);
        }
        if (ok) mma_commit(&tfull[buf]);
      }
      mma_commit(done);  // tracks every MMA issued above
    }
  } else {
    // epilogue warps 0-3
    int tl = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tl) {
      const int buf = tl & 1;
      const unsigned ub = (unsigned)(tl >> 1);
      if (!mbar_wait(&tfull[buf], ub & 1u, a.timeout_ns) || *(volatile int *)&s_late) {
        s_late = 1;
        break;
      }
      fence_after();
      const TileIdx ti = tile_of(tile, tiles_x, tiles_pix, ntn, UR);
      const int n0 = ti.nt * N;
      const int m = warp * 32 + lane;
#pragma unroll 1
      for (int h = 0; h < P; ++h) {
        const int gy = ti.ty0 + kTH * h + m / kTW, gx = ti.tx0 + m % kTW;
        const bool in = gy < a.H && gx < a.W;
        const long long obase = (((long long)ti.b * a.H + gy) * a.W + gx) * a.Cout + n0;
#pragma unroll
        for (int cb = 0; cb < N; cb += 16) {
          uint32_t r[16];
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((buf * P + h) * N + cb), r);
          if (in) {
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              v[j] = __uint_as_float(r[j]) + (a.bias ? a.bias[n0 + cb + j] : 0.0f);
              if (a.relu) v[j] = fmaxf(v[j], 0.0f);
            }
            uint4 pk[2];
            __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
            for (int j = 0; j < 8; ++j) h2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            uint4 *dst = reinterpret_cast<uint4 *>(a.y + obase + cb);
            dst[0] = pk[0];
            dst[1] = pk[1];
            if (a.y32) {
              float4 *d32 = reinterpret_cast<float4 *>(a.y32 + obase + cb);
#pragma unroll
              for (int j = 0; j < 4; ++j) d32[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
          }
        }
      }
      // this warp's reads of the accumulator set are done: release it
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }
  __syncthreads();
  if (s_late) {
    if (tid == 0) {
      set_error(a.st, RF_ERR_TIMEOUT);
      mbar_wait(done, 0u, a.timeout_ns);  // the issued MMAs, before TMEM is freed
    }
  } else if (tid == 0) {
    mbar_wait(done, 0u, a.timeout_ns);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// Tensor maps.  x: dims (Cin, W, H, B) of the NHWC input, box (8, 16, 10, 1)
// = one A plane [row][col][8 ch]; w: dims (Cin, 9, Cout) of the weights
// [Cout][9][Cin], box (8, 1, N) = one B plane [n][8 ch].
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <int N>
rf_status encode_maps(const TcArgs &t, CUtensorMap &xmap, CUtensorMap &wmap, int box_rows = kPH) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return RF_ERR_UNSUPPORTED;
  const cuuint64_t xdim[4] = {(cuuint64_t)t.Cin, (cuuint64_t)t.W, (cuuint64_t)t.H, (cuuint64_t)t.B};
  const cuuint64_t xstr[3] = {(cuuint64_t)t.Cin * 2, (cuuint64_t)t.W * t.Cin * 2, (cuuint64_t)t.H * t.W * t.Cin * 2};
  const cuuint32_t xbox[4] = {8, kTW, (cuuint32_t)box_rows, 1};
  const cuuint32_t one4[4] = {1, 1, 1, 1};
  if (enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)t.x, xdim, xstr, xbox, one4,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return RF_ERR_UNSUPPORTED;
  const cuuint64_t wdim[3] = {(cuuint64_t)t.Cin, 9, (cuuint64_t)t.Cout};
  const cuuint64_t wstr[2] = {(cuuint64_t)t.Cin * 2, (cuuint64_t)9 * t.Cin * 2};
  const cuuint32_t wbox[3] = {8, 1, (cuuint32_t)N};
  const cuuint32_t one3[3] = {1, 1, 1};
  if (enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)t.w, wdim, wstr, wbox, one3,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return RF_ERR_UNSUPPORTED;
  return RF_OK;
}

inline TmaArgs tma_args(const TcArgs &t) {
  TmaArgs a;
  a.wpack = t.wpack;
  a.bias = t.bias;
  a.y = t.y;
  a.y32 = t.y32;
  a.B = t.B;
  a.H = t.H;
  a.W = t.W;
  a.Cin = t.Cin;
  a.Cout = t.Cout;
  a.relu = t.relu;
  a.st = t.st;
  a.timeout_ns = t.timeout_ns;
  return a;
}

template <int N>
rf_status launch_tma(const TcArgs &t, cudaStream_t s) {
  alignas(64) CUtensorMap xmap, wmap;
  rf_status rs = encode_maps<N>(t, xmap, wmap);
  if (rs != RF_OK) return rs;
  const TmaArgs a = tma_args(t);
  const size_t smem = tma_smem_bytes(N);
  if (cudaFuncSetAttribute(conv3x3_tma_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  const int tiles = ((t.W + kTW - 1) / kTW) * ((t.H + kTH - 1) / kTH);
  dim3 grid(tiles, (t.Cout + N - 1) / N, t.B);
  conv3x3_tma_kernel<N><<<grid, kThreads, smem, s>>>(xmap, wmap, a);
  return cuda_status(cudaGetLastError());
}

// The persistent kernel: one CTA per SM (at most one per unit of P tiles).
template <int N, int P>
rf_status launch_persist(const TcArgs &t, int num_sms, cudaStream_t s) {
  alignas(64) CUtensorMap xmap, wmap;
  rf_status rs = encode_maps<N>(t, xmap, wmap, kTH * P + 2);
  if (rs != RF_OK) return rs;
  const TmaArgs a = tma_args(t);
  const size_t smem = persist_smem_bytes(N, P);
  if (cudaFuncSetAttribute(conv3x3_persist_kernel<N, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  const long long ntiles =
      (long long)((t.W + kTW - 1) / kTW) * ((t.H + kTH * P - 1) / (kTH * P)) * (t.Cout / N) * t.B;
  if (ntiles > (1LL << 30)) return RF_ERR_INVALID_ARG;
  const int grid = (int)std::min<long long>(ntiles, num_sms);
  if (t.wpack) {
    const long long chunks = (long long)t.Cout * 9 * (t.Cin / 8);
    pack_w_kernel<N><<<(int)std::min<long long>((chunks + 255) / 256, 4LL * num_sms), 256, 0, s>>>(t.w, t.wpack, t.Cin,
                                                                                               t.Cout);
  }
  conv3x3_persist_kernel<N, P><<<grid, kPersistThreads, smem, s>>>(xmap, wmap, a);
  return cuda_status(cudaGetLastError());
}

template <int N>
rf_status launch(const TcArgs &a, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(a.CC, N);
  if (cudaFuncSetAttribute(conv3x3_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return RF_ERR_CUDA;
  const int tiles = ((a.W + kTW - 1) / kTW) * ((a.H + kTH - 1) / kTH);
  dim3 grid(tiles, (a.Cout + N - 1) / N, a.B);
  conv3x3_tc_kernel<N><<<grid, kThreads, smem, s>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace tc
}  // namespace rf

using namespace rf;

extern "C" rf_status rf_unet_conv3x3_tc(rf_ctx *ctx, const uint16_t *x, int B, int H, int W, int Cin,
                                        const uint16_t *w, const float *bias, int Cout, int relu, uint16_t *y,
                                        float *y32, void *stream) {
  if (!ctx || !x || !w || !y || B < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 || Cout < 16 || Cout % 16)
    return RF_ERR_INVALID_ARG;
  if (B > 65535) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  tc::TcArgs a;
  a.x = reinterpret_cast<const tc::bf16 *>(x);
  a.w = reinterpret_cast<const tc::bf16 *>(w);
  a.bias = bias;
  a.y = reinterpret_cast<tc::bf16 *>(y);
  a.y32 = y32;
  a.B = B;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  a.relu = relu;
  // 32-channel chunks keep a CTA's buffers small enough for two CTAs per
  // SM, so that one CTA's loads overlap the other's MMAs
  a.CC = (Cin % 32 == 0) ? 32 : 16;
  a.st = ctx->state;
  a.timeout_ns = ctx->timeout_ns;
  // the persistent kernel takes its weight stages from a packed copy when
  // the layer has 64 or more input and output channels (8 x 128^2 x
  // 128 -> 128: 447 -> 651 TFLOP/s); narrower layers have too few stages
  // per unit to repay the packing launch (32 -> 32: 200 -> 115 TFLOP/s)
  a.wpack = nullptr;
  if (Cin >= 64 && Cout % 64 == 0) {
    if (rf_status rw = ensure(&ctx->wpack, &ctx->wpack_cap, (size_t)Cout * 9 * Cin); rw != RF_OK) return rw;
    a.wpack = reinterpret_cast<tc::bf16 *>(ctx->wpack);
  }
  // the pipelined tensor-copy kernel; the plain one if a tensor map cannot
  // be encoded here
  rf_status rs = RF_ERR_UNSUPPORTED;
  // 8 x 16 tiles per weight stage: as many as two accumulator sets leave
  // room for in tensor memory (2 P N <= 512 columns)
  if (Cout % 128 == 0) rs = tc::launch_persist<128, 2>(a, ctx->num_sms, s);
  else if (Cout % 64 == 0) rs = tc::launch_persist<64, 4>(a, ctx->num_sms, s);
  else if (Cout % 32 == 0) rs = tc::launch_persist<32, 4>(a, ctx->num_sms, s);
  else rs = tc::launch_persist<16, 4>(a, ctx->num_sms, s);
  if (rs != RF_ERR_UNSUPPORTED) return rs;
  if (Cout % 128 == 0) rs = tc::launch_tma<128>(a, s);
  else if (Cout % 64 == 0) rs = tc::launch_tma<64>(a, s);
  else if (Cout % 32 == 0) rs = tc::launch_tma<32>(a, s);
  else rs = tc::launch_tma<16>(a, s);
  if (rs != RF_ERR_UNSUPPORTED) return rs;
  if (Cout % 128 == 0) return tc::launch<128>(a, s);
  if (Cout % 64 == 0) return tc::launch<64>(a, s);
  if (Cout % 32 == 0) return tc::launch<32>(a, s);
  return tc::launch<16>(a, s);
}
