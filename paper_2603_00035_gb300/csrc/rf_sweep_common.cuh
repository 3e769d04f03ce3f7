// rf_sweep_common.cuh -- pieces shared by the band-pipelined line-sweep
// kernels (forward solve and transposed-sweep adjoint): bounded waits, the
// bounded grid barrier, tile geometry and direction mappings.
#pragma once

#include "rf_device.cuh"

namespace rf {

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Per-launch control words (device): abort flag raised by any timed-out
// wait so that every CTA leaves its loops.
struct LaunchCtl {
  DevState *st;
  int *abort;
  long long timeout_ns;
};

__device__ __forceinline__ void raise_timeout(const LaunchCtl &c) {
  set_error(c.st, RF_ERR_TIMEOUT);
  atomicExch(c.abort, 1);
}

// Spin until *p >= target; false (and a raised timeout) on expiry.
__device__ __forceinline__ bool wait_geq(const unsigned *p, unsigned target,
                                         const LaunchCtl &c) {
  if (ld_acquire_u32(p) >= target) return true;
  const unsigned long long t0 = gtimer();
  while (ld_acquire_u32(p) < target) {
    if ((long long)(gtimer() - t0) > c.timeout_ns || ld_acquire_s32(c.abort)) {
      raise_timeout(c);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// Bounded grid-wide barrier for a cooperative launch.  Every CTA calls it.
// One monotone 64-bit arrival counter, zeroed before the launch: the
// arrival returning old value o belongs to barrier floor(o / G) (G CTAs),
// which is complete once the counter reaches (floor(o / G) + 1) G.  No
// reset inside the launch and one atomic per CTA; it measured 1.4 us per
// barrier for 152 CTAs where a count-and-generation barrier took 2.2 us.
__device__ __forceinline__ bool grid_sync(const LaunchCtl &c) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned long long *bar = &c.st->bar;
    unsigned long long o;
    // release: the CTA's stores before the __syncthreads are visible to
    // whoever acquires the counter past this arrival
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(o) : "l"(bar), "l"(1ull) : "memory");
    const unsigned long long target = (o / gridDim.x + 1) * gridDim.x;
    if (ld_acquire_u64(bar) < target) {
      const unsigned long long t0 = gtimer();
      unsigned spins = 0;
      while (ld_acquire_u64(bar) < target) {
        if ((++spins & 15) == 0 && (long long)(gtimer() - t0) > c.timeout_ns) {
          raise_timeout(c);
          ok = 0;
          break;
        }
      }
    }
    ok_s = ok && !ld_acquire_s32(c.abort);
  }
  __syncthreads();
  return ok_s != 0;
}

// Global index of (line step s, line l) for sweep direction dir:
// 0 columns +x, 1 rows +y, 2 columns -x, 3 rows -y.
__device__ __forceinline__ long long gidx(int dir, int s, int l, int ny, int nx) {
  int i, j;
  if ((dir & 1) == 0) {
    j = (dir == 0) ? s : nx - 1 - s;
    i = l;
  } else {
    i = (dir == 1) ? s : ny - 1 - s;
    j = l;
  }
  return (long long)i * nx + j;
}

// Tile offset (ds, dl) of neighbour n for direction dir.
__device__ __forceinline__ void nb_tile_offset(int dir, int n, int &ds, int &dl) {
  const int dx = nb_dx(n), dy = nb_dy(n);
  switch (dir) {
    case 0: ds = dx; dl = dy; break;
    case 1: ds = dy; dl = dx; break;
    case 2: ds = -dx; dl = dy; break;
    default: ds = -dy; dl = dx; break;
  }
}

// Tile offset (step, line) of neighbour n for a compile-time direction.
template <int DIR>
__device__ constexpr int tile_ds(int n) {
  return DIR == 0 ? nb_dx(n) : DIR == 1 ? nb_dy(n) : DIR == 2 ? -nb_dx(n) : -nb_dy(n);
}
template <int DIR>
__device__ constexpr int tile_dl(int n) {
  return (DIR & 1) == 0 ? nb_dy(n) : nb_dx(n);
}

// Change test of the forward sweeps: |tnew - told| > tol + rtol * tnew,
// +inf on exactly one side counts as changed; tol = rtol = 0 is bitwise.
__device__ __forceinline__ bool node_changed(float tnew, float told, float tol, float rtol) {
  if (tol == 0.0f && rtol == 0.0f) return __float_as_uint(tnew) != __float_as_uint(told);
  const bool fn = tnew < kInf, fo = told < kInf;
  if (fn != fo) return true;
  if (!fn) return false;
  return fabsf(tnew - told) > fmaf(rtol, fabsf(tnew), tol);
}

// Copy `total` elements, element f read by ld(f) and written by st(f, v),
// with B independent loads in flight per thread before the first store, so
// a block-wide tile fill costs a few memory latencies instead of one per
// element.
template <int B, class V, class Ld, class St>
__device__ __forceinline__ void batched_copy(int total, Ld ld, St st) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int base = tid; base < total; base += B * nth) {
    V v[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int f = base + u * nth;
      v[u] = (f < total) ? ld(f) : V(0);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int f = base + u * nth;
      if (f < total) st(f, v[u]);
    }
  }
}

}  // namespace rf
