// rf_device.cuh -- device-side pieces shared by the librf kernels: stencil
// geometry, per-node metric constants and the FP32 local update
// (Sec. 3.2, Eqs. 2-3; App. A "Two-Point Update", "One-Point Fallback").
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "../../include/rf.h"

namespace rf {

constexpr float kInf = __builtin_huge_valf();

// Neighbour ring of Fig. 4(a): n = 0..7 counter-clockwise from the
// upper-left; offsets (dx, dy) with +y = +i.
__host__ __device__ constexpr int nb_dx(int n) {
  return (n <= 2) ? -1 : (n == 3 || n == 7) ? 0 : 1;
}
__host__ __device__ constexpr int nb_dy(int n) {
  return (n == 0 || n == 6 || n == 7) ? 1 : (n == 1 || n == 5) ? 0 : -1;
}

// Per-node constants of the local update.  With M = L L^T + eps I and
// displacements m_n = h (dx_n, dy_n):
//   len[c]  = |m|_M for the four displacement classes
//             c = 0: (+-1, 0)   c = 1: (0, +-1)
//             c = 2: +-(1, 1)   c = 3: +-(1, -1)
//   wm[n]   = w . m_n  (drift term, S_n = T_n - wm[n])
//   ax, ay  = |m_1 - m_2|^2_M of stencils whose donors differ along x / y
//   det     = det E = h^4 det M for every stencil (|det [m1|m2]| = h^2)
struct NodeConst {
  float len[4];
  float wm[4];  // for n = 0..3; wm[n+4] = -wm[n]
  float ax, ay, det;
};

__device__ __forceinline__ int len_class(int n) {
  // n: 0 (-1,1) anti, 1 (-1,0) x, 2 (-1,-1) diag, 3 (0,-1) y,
  //    4 (1,-1) anti, 5 (1,0) x, 6 (1,1) diag, 7 (0,1) y
  return (n & 1) ? ((n & 2) ? 1 : 0) : ((n & 2) ? 2 : 3);
}

__device__ __forceinline__ NodeConst node_const(float l11, float l21,
                                                float l22, float wx, float wy,
                                                float h, float eps) {
  NodeConst c;
  const float m11 = fmaf(l11, l11, eps);
  const float m12 = l11 * l21;
  const float m22 = fmaf(l21, l21, fmaf(l22, l22, eps));
  const float h2 = h * h;
  c.ax = h2 * m11;
  c.ay = h2 * m22;
  c.len[0] = sqrtf(c.ax);
  c.len[1] = sqrtf(c.ay);
  c.len[2] = sqrtf(h2 * (m11 + 2.0f * m12 + m22));
  c.len[3] = sqrtf(h2 * (m11 - 2.0f * m12 + m22));
  // det M = (L11 L22)^2 + eps (L11^2 + L21^2 + L22^2 + eps): no cancellation
  const float p = l11 * l22;
  const float detm =
      fmaf(p, p, eps * (l11 * l11 + l21 * l21 + l22 * l22 + eps));
  c.det = (h2 * h2) * detm;
#pragma unroll
  for (int n = 0; n < 4; ++n)
    c.wm[n] = h * (wx * (float)nb_dx(n) + wy * (float)nb_dy(n));
  return c;
}

__device__ __forceinline__ float node_wm(const NodeConst &c, int n) {
  return (n < 4) ? c.wm[n] : -c.wm[n - 4];
}

// Two-point candidate of stencil k (donors k, k+1) in the shifted form
// tau = T0 - min(S):  (s - tau 1)^T adj(E) (s - tau 1) = det E, whose
// discriminant reduces to det E (|m1 - m2|^2_M - Delta^2).  Returns +inf
// when invalid.  On return l1, l2 hold det(E) * lambda = adj(E)(T0 1 - S).
__device__ __forceinline__ float two_point(const NodeConst &c, int k, float T1,
                                           float T2, float &l1, float &l2) {
  const int a = k, b = (k + 1) & 7;
  l1 = l2 = -1.0f;
  if (!(T1 < kInf && T2 < kInf)) return kInf;
  const float S1 = T1 - node_wm(c, a);
  const float S2 = T2 - node_wm(c, b);
  const float e11 = c.len[len_class(a)] * c.len[len_class(a)];
  const float e22 = c.len[len_class(b)] * c.len[len_class(b)];
  // donors of stencils 0,1,4,5 differ along y; of 2,3,6,7 along x
  const float aa = ((k & 2) == 0) ? c.ay : c.ax;
  const float e12 = 0.5f * (e11 + e22 - aa);
  const float d = S2 - S1;
  const float disc = c.det * (aa - d * d);
  if (!(disc >= 0.0f)) return kInf;
  const float sq = sqrtf(disc);
  float tau, u1, u2, T0;
  if (d >= 0.0f) {  // S1 is the smaller
    tau = fmaf(d, e11 - e12, sq) / aa;
    u1 = tau;
    u2 = tau - d;
    T0 = S1 + tau;
  } else {
    tau = fmaf(-d, e22 - e12, sq) / aa;
    u1 = tau + d;
    u2 = tau;
    T0 = S2 + tau;
  }
  l1 = fmaf(e22, u1, -e12 * u2);
  l2 = fmaf(e11, u2, -e12 * u1);
  const bool ok = (l1 >= 0.0f) && (l2 >= 0.0f) && (T1 < T0) && (T2 < T0);
  return ok ? T0 : kInf;
}

__device__ __forceinline__ float one_point(const NodeConst &c, int n, float Tn) {
  return (Tn < kInf) ? (Tn - node_wm(c, n)) + c.len[len_class(n)] : kInf;
}

// Minimum valid candidate (value only).
__device__ __forceinline__ float best_candidate(const NodeConst &c,
                                                const float Tn[8]) {
  float best = kInf;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float l1, l2;
    best = fminf(best, two_point(c, k, Tn[k], Tn[(k + 1) & 7], l1, l2));
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) best = fminf(best, one_point(c, n, Tn[n]));
  return best;
}

// Minimum valid candidate with its identity: tie-break strict '<' in the
// order two-point k = 0..7, then one-point n = 0..7.
struct Winner {
  float value;
  uint8_t id;  // 0 none, 0x10|n one-point, 0x20|k two-point
  float l1, l2;
};

__device__ __forceinline__ Winner winner(const NodeConst &c, const float Tn[8]) {
  Winner w;
  w.value = kInf;
  w.id = 0;
  w.l1 = w.l2 = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float l1, l2;
    const float v = two_point(c, k, Tn[k], Tn[(k + 1) & 7], l1, l2);
    if (v < w.value) {
      w.value = v;
      w.id = (uint8_t)(0x20 | k);
      w.l1 = l1;
      w.l2 = l2;
    }
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float v = one_point(c, n, Tn[n]);
    if (v < w.value) {
      w.value = v;
      w.id = (uint8_t)(0x10 | n);
    }
  }
  return w;
}

// ---- bounded waits -------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_s32(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Device status word layout shared by the kernels (one per context).
struct DevState {
  int status;          // rf_status
  int sweeps;
  int converged;
  int adj_sweeps;
  unsigned bar_count;  // grid barrier arrivals
  unsigned bar_gen;    // grid barrier generation
  unsigned max_res_bits;  // float bits of max |residual| (non-negative)
  unsigned pad;
  unsigned long long cell_updates;
};

__device__ __forceinline__ void set_error(DevState *st, int code) {
  atomicCAS(&st->status, 0, code);
}

}  // namespace rf
