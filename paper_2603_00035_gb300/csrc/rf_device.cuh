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

// Per-node constants of the local update ("node table", 11 floats).  With
// M = L L^T + eps I and displacements m_n = h (dx_n, dy_n):
//   len[c]  = |m|_M for the four displacement classes
//             c = 0: (+-1, 0)   c = 1: (0, +-1)
//             c = 2: +-(1, 1)   c = 3: +-(1, -1)
//   wm[n]   = w . m_n for n = 0..3 (wm[n+4] = -wm[n]); S_n = T_n - w . m_n
//   det     = det E = h^4 det M, the same for every stencil
//             (|det [m1|m2]| = h^2)
//   inv_ax, inv_ay = 1 / |m1 - m2|^2_M for stencils whose donors differ
//             along x / y (|m1 - m2|^2_M = len[0]^2 or len[1]^2)
// They depend on the fields only, so the sweep computes them once per node
// and block, off the line-step critical path.
constexpr int kTabSize = 11;
enum { TAB_LEN = 0, TAB_WM = 4, TAB_DET = 8, TAB_IAX = 9, TAB_IAY = 10 };

__host__ __device__ __forceinline__ int len_class(int n) {
  // n: 0 (-1,1) anti, 1 (-1,0) x, 2 (-1,-1) diag, 3 (0,-1) y,
  //    4 (1,-1) anti, 5 (1,0) x, 6 (1,1) diag, 7 (0,1) y
  return (n & 1) ? ((n & 2) ? 1 : 0) : ((n & 2) ? 2 : 3);
}

__device__ __forceinline__ void node_tab(float l11, float l21, float l22, float wx, float wy, float h,
                                         float eps, float tab[kTabSize]) {
  const float m11 = fmaf(l11, l11, eps);
  const float m12 = l11 * l21;
  const float m22 = fmaf(l21, l21, fmaf(l22, l22, eps));
  const float h2 = h * h;
  tab[TAB_LEN + 0] = sqrtf(h2 * m11);
  tab[TAB_LEN + 1] = sqrtf(h2 * m22);
  tab[TAB_LEN + 2] = sqrtf(h2 * (m11 + 2.0f * m12 + m22));
  tab[TAB_LEN + 3] = sqrtf(h2 * (m11 - 2.0f * m12 + m22));
#pragma unroll
  for (int n = 0; n < 4; ++n) tab[TAB_WM + n] = h * (wx * (float)nb_dx(n) + wy * (float)nb_dy(n));
  // det M = (L11 L22)^2 + eps (L11^2 + L21^2 + L22^2 + eps): no cancellation
  const float p = l11 * l22;
  const float detm = fmaf(p, p, eps * (l11 * l11 + l21 * l21 + l22 * l22 + eps));
  tab[TAB_DET] = (h2 * h2) * detm;
  tab[TAB_IAX] = 1.0f / (tab[TAB_LEN + 0] * tab[TAB_LEN + 0]);
  tab[TAB_IAY] = 1.0f / (tab[TAB_LEN + 1] * tab[TAB_LEN + 1]);
}

// Two-point candidate (Eq. 2) of a stencil with donor times T1, T2,
// donor lengths la = |m1|_M, lb = |m2|_M, drift terms wa = w.m1, wb = w.m2,
// |m1 - m2|^2_M = aa (with its reciprocal inv) and det E.  Shifted form
// tau = T0 - min(S):  (s - tau 1)^T adj(E) (s - tau 1) = det E, whose
// discriminant reduces to det E (aa - Delta^2).  Returns +inf when invalid
// (no real root, lambda < 0, or a donor not earlier than T0).  On return
// l1, l2 = det(E) * lambda = adj(E) (T0 1 - S).
__device__ __forceinline__ float two_point_core(float la, float lb, float wa, float wb, float aa, float inv,
                                                float det, float T1, float T2, float &l1, float &l2) {
  // branch-free: a missing donor (+inf) makes d, disc NaN and every test
  // below false, so the candidate is rejected without divergence
  const float S1 = T1 - wa;
  const float S2 = T2 - wb;
  const float e11 = la * la;
  const float e22 = lb * lb;
  const float e12 = 0.5f * (e11 + e22 - aa);
  const float d = S2 - S1;
  const float disc = det * fmaf(-d, d, aa);
  // sqrt(disc) as disc * rsqrt(disc) (MUFU); 0 at disc = 0
  const float sq = disc > 0.0f ? disc * rsqrtf(disc) : 0.0f;
  const bool s1min = d >= 0.0f;  // S1 is the smaller
  const float tau = fmaf(fabsf(d), s1min ? (e11 - e12) : (e22 - e12), sq) * inv;
  const float u1 = s1min ? tau : tau + d;
  const float u2 = s1min ? tau - d : tau;
  const float T0 = (s1min ? S1 : S2) + tau;
  l1 = fmaf(e22, u1, -e12 * u2);
  l2 = fmaf(e11, u2, -e12 * u1);
  const bool ok = (disc >= 0.0f) && (l1 >= 0.0f) && (l2 >= 0.0f) && (T1 < T0) && (T2 < T0);
  return ok ? T0 : kInf;
}

__device__ __forceinline__ float tab_wm(const float tab[kTabSize], int n) {
  return (n < 4) ? tab[TAB_WM + n] : -tab[TAB_WM + n - 4];
}

__device__ __forceinline__ float two_point(const float tab[kTabSize], int k, float T1, float T2, float &l1,
                                           float &l2) {
  const int a = k, b = (k + 1) & 7;
  // donors of stencils 0,1,4,5 differ along y; of 2,3,6,7 along x
  const bool xs = (k & 2) != 0;
  const float lx = xs ? tab[TAB_LEN + 0] : tab[TAB_LEN + 1];
  return two_point_core(tab[TAB_LEN + len_class(a)], tab[TAB_LEN + len_class(b)], tab_wm(tab, a), tab_wm(tab, b),
                        lx * lx, xs ? tab[TAB_IAX] : tab[TAB_IAY], tab[TAB_DET], T1, T2, l1, l2);
}

// One-point candidate (Eq. 3): T_n - w.m_n + |m_n|_M.
__device__ __forceinline__ float one_point_core(float len, float wm, float Tn) {
  return (Tn < kInf) ? (Tn - wm) + len : kInf;
}

__device__ __forceinline__ float one_point(const float tab[kTabSize], int n, float Tn) {
  return one_point_core(tab[TAB_LEN + len_class(n)], tab_wm(tab, n), Tn);
}

// Minimum valid candidate with its identity: tie-break strict '<' in the
// order two-point k = 0..7, then one-point n = 0..7.
struct Winner {
  float value;
  uint8_t id;  // 0 none, 0x10|n one-point, 0x20|k two-point
  float l1, l2;
};

// With tself finite, only candidates whose donors are all strictly earlier
// than tself are eligible: the record then always forms a DAG that is
// ordered by T (the ordered adjoint relies on it).  tself = +inf gives the
// plain minimum.
__device__ __forceinline__ Winner winner(const float tab[kTabSize], const float Tn[8], float tself = kInf) {
  Winner w;
  w.value = kInf;
  w.id = 0;
  w.l1 = w.l2 = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float l1, l2;
    const float v = two_point(tab, k, Tn[k], Tn[(k + 1) & 7], l1, l2);
    const bool elig = (Tn[k] < tself) && (Tn[(k + 1) & 7] < tself);
    if (v < w.value && elig) {
      w.value = v;
      w.id = (uint8_t)(0x20 | k);
      w.l1 = l1;
      w.l2 = l2;
    }
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float v = one_point(tab, n, Tn[n]);
    if (v < w.value && Tn[n] < tself) {
      w.value = v;
      w.id = (uint8_t)(0x10 | n);
    }
  }
  return w;
}

// Weight with which child q (record id, w1) passes lambda to the neighbour in
// direction `back` (the direction from q to that neighbour); 0 if none.
__device__ __forceinline__ float child_weight(uint8_t id, float w1, int back) {
  const int k = id & 7;
  if (id & 0x10) return (k == back) ? 1.0f : 0.0f;
  if (id & 0x20) return (k == back) ? w1 : ((((k + 1) & 7) == back) ? 1.0f - w1 : 0.0f);
  return 0.0f;
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
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Polling load: the child's multiplier and the epoch tag sit in one 64-bit
// word written by one store, so a relaxed (single-copy atomic) load that
// sees the tag sees the value; unlike an acquire load it does not hold back
// the loads of the other children.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// Publishing store: a parent reads nothing of its child but this one 64-bit
// word (multiplier and epoch tag together), so single-copy atomicity is all
// the hand-over needs -- no release fence, which would first wait for the
// thread's earlier gradient stores to reach L2.
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Device status word layout shared by the kernels (one per context).
struct DevState {
  int status;          // rf_status
  int sweeps;
  int converged;
  int adj_sweeps;
  unsigned long long bar;  // grid barrier arrivals of the running launch (zeroed before it)
  unsigned max_res_bits;  // float bits of max |residual| (non-negative)
  unsigned rounds;        // rounds of the last tile-queue solve
  unsigned long long cell_updates;
  unsigned adj_epoch;  // tag of the adjoint's per-node state words, bumped on the device per launch
  unsigned pad;
};

__device__ __forceinline__ void set_error(DevState *st, int code) {
  atomicCAS(&st->status, 0, code);
}

}  // namespace rf
