// rf_cone.cuh -- the local update of Sec. 3.2 (Eqs. 2-3; App. A "Two-Point
// Update", "One-Point Fallback") in the cone form, shared by the forward
// kernels that evaluate it from per-node constants (the streamed line sweep
// and the tile-queue solve) and by the record of their converged T.
//
// With S_n = T_n - w.m_n and d = S_b - S_a for the stencil with donors a, b,
// the paper's shifted two-point update has the closed form
//     T0 = S_a + C d + sqrt(P - Q d^2),   C = (e_aa - e_ab) / aa,
//     P = det E / aa,  Q = det E / aa^2,
// for either sign of d (C + C' = 1 absorbs the min(S) branch), and the
// barycentric weights are both >= 0 exactly when the minimiser of the
// Hopf-Lax function over the segment is interior:
//     lo < d < hi,   lo = (e_ab - e_bb) / |m_b|,  hi = (e_aa - e_ab) / |m_a|
// (the derivative of the convex segment cost at the two ends).  Causality
// (both donors earlier than T0) is tested as in the paper.  Stencils k and
// k+4 share C, lo, hi (m -> -m leaves every quadratic form unchanged); P, Q
// depend only on whether the donors differ along x or y.
#pragma once

#include "rf_device.cuh"

namespace rf {

// Node record (24 floats, six float4):
//   q0  |m|_M by displacement class (x, y, +-(1,1), +-(1,-1)); the sign of
//       the first is the source flag (negative: source node)
//   q1  w.m_n for n = 0..3 (w.m_{n+4} = -w.m_n)
//   q2  P_x, Q_x, P_y, Q_y   (aa = |m_a - m_b|^2_M = e_x or e_y)
//   q3  C of stencil pairs p = 0..3 (stencil k uses pair k & 3)
//   q4  (lo + hi) / 2 of the pairs
//   q5  (hi - lo) / 2 of the pairs
constexpr int kPlanes = 6;

__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void node_record(float l11, float l21, float l22, float wx, float wy, float h, float eps,
                                            bool src, float4 q[kPlanes]) {
  const float m11 = fmaf(l11, l11, eps);
  const float m12 = l11 * l21;
  const float m22 = fmaf(l21, l21, fmaf(l22, l22, eps));
  const float h2 = h * h;
  float e[4];
  e[0] = h2 * m11;
  e[1] = h2 * m22;
  e[2] = h2 * (m11 + 2.0f * m12 + m22);
  e[3] = h2 * (m11 - 2.0f * m12 + m22);
  float len[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) len[c] = sqrtf(e[c]);
  float wm[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) wm[n] = h * (wx * (float)nb_dx(n) + wy * (float)nb_dy(n));
  // det E = h^4 det M, det M = (L11 L22)^2 + eps (L11^2 + L21^2 + L22^2 + eps)
  const float pp = l11 * l22;
  const float dete = (h2 * h2) * fmaf(pp, pp, eps * (l11 * l11 + l21 * l21 + l22 * l22 + eps));
  const float Px = dete / e[0], Py = dete / e[1];
  const float Qx = Px / e[0], Qy = Py / e[1];
  float C[4], mid[4], half[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int ca = len_class(p), cb = len_class(p + 1);
    const float aa = (p & 2) ? e[0] : e[1];  // donors differ along x for p = 2, 3
    const float dab = e[ca] - e[cb];
    const float hi = 0.5f * (dab + aa) / len[ca];
    const float lo = 0.5f * (dab - aa) / len[cb];
    C[p] = 0.5f * (dab + aa) / aa;
    mid[p] = 0.5f * (hi + lo);
    half[p] = 0.5f * (hi - lo);
  }
  q[0] = make_float4(src ? -len[0] : len[0], len[1], len[2], len[3]);
  q[1] = make_float4(wm[0], wm[1], wm[2], wm[3]);
  q[2] = make_float4(Px, Qx, Py, Qy);
  q[3] = make_float4(C[0], C[1], C[2], C[3]);
  q[4] = make_float4(mid[0], mid[1], mid[2], mid[3]);
  q[5] = make_float4(half[0], half[1], half[2], half[3]);
}

// Minimum over the valid one-point and two-point candidates of a node with
// record q and neighbour times Tn (+inf where missing); +inf if none.
__device__ __forceinline__ float cone_min(const float4 &q0, const float4 &q1, const float4 &q2, const float4 &q3,
                                          const float4 &q4, const float4 &q5, const float Tn[8]) {
  const float len[4] = {fabsf(q0.x), q0.y, q0.z, q0.w};
  const float wm[4] = {q1.x, q1.y, q1.z, q1.w};
  const float C[4] = {q3.x, q3.y, q3.z, q3.w};
  const float mid[4] = {q4.x, q4.y, q4.z, q4.w};
  const float hw[4] = {q5.x, q5.y, q5.z, q5.w};
  float S[8];
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) S[nb] = (nb < 4) ? Tn[nb] - wm[nb] : Tn[nb] + wm[nb - 4];
  // one-point candidates (Eq. 3): S_n + |m_n|_M (+inf donors stay +inf)
  float cand = kInf;
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) cand = fminf(cand, S[nb] + len[len_class(nb)]);
  // two-point candidates (Eq. 2) in the cone form
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int a = k, b = (k + 1) & 7, p = k & 3;
    const bool xs = (k & 2) != 0;
    const float Pk = xs ? q2.x : q2.z, Qk = xs ? q2.y : q2.w;
    const float d = S[b] - S[a];
    const float q = fmaf(-Qk, d * d, Pk);
    const float T0 = fmaf(C[p], d, S[a]) + q * rsqrt_ftz(q);
    const bool ok = (fabsf(d - mid[p]) < hw[p]) && (fmaxf(Tn[a], Tn[b]) < T0);
    if (ok) cand = fminf(cand, T0);
  }
  return cand;
}

// Soft-min relaxation (Sec. 3.3; the reading of rf_softmin.cu) in the cone
// form: every stencil k has the value of its segment minimum -- the valid
// two-point candidate, else the smaller one-point candidate of its
// endpoints -- and the node takes -tau log sum_k exp(-v_k / tau) (the hard
// minimum when tau = 0; +inf when no stencil has a finite value).
__device__ __forceinline__ float cone_softmin(const float4 &q0, const float4 &q1, const float4 &q2,
                                              const float4 &q3, const float4 &q4, const float4 &q5,
                                              const float Tn[8], float tau) {
  const float len[4] = {fabsf(q0.x), q0.y, q0.z, q0.w};
  const float wm[4] = {q1.x, q1.y, q1.z, q1.w};
  const float C[4] = {q3.x, q3.y, q3.z, q3.w};
  const float mid[4] = {q4.x, q4.y, q4.z, q4.w};
  const float hw[4] = {q5.x, q5.y, q5.z, q5.w};
  float S[8], one[8], v[8];
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) {
    S[nb] = (nb < 4) ? Tn[nb] - wm[nb] : Tn[nb] + wm[nb - 4];
    one[nb] = S[nb] + len[len_class(nb)];
  }
  float vmin = kInf;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int a = k, b = (k + 1) & 7, p = k & 3;
    const bool xs = (k & 2) != 0;
    const float Pk = xs ? q2.x : q2.z, Qk = xs ? q2.y : q2.w;
    const float d = S[b] - S[a];
    const float q = fmaf(-Qk, d * d, Pk);
    const float T0 = fmaf(C[p], d, S[a]) + q * rsqrt_ftz(q);
    const bool ok = (fabsf(d - mid[p]) < hw[p]) && (fmaxf(Tn[a], Tn[b]) < T0);
    v[k] = ok ? T0 : fminf(one[a], one[b]);
    vmin = fminf(vmin, v[k]);
  }
  if (!(vmin < kInf) || !(tau > 0.0f)) return vmin;
  float sum = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += (v[k] < kInf) ? expf((vmin - v[k]) / tau) : 0.0f;
  return vmin - tau * logf(sum);
}

// Stencil record of node (i, j) at the converged T in the cone form (Alg. 2
// first loop; App. A closed-form partials): one pass over the 16 candidates
// gives both the plain minimum (for the residual r = T - min valid
// candidate(T)) and the winner among the candidates whose donors are all
// strictly earlier than T (for the record: the recorded stencils form a DAG
// ordered by T).  Tie-break: strict '<' in the order two-point k = 0..7,
// then one-point n = 0..7.  For a two-point winner with donors a, b the
// barycentric weights are (l1, l2) / (l1 + l2), l = adj(E) (T0 1 - S)
// (App. A), evaluated at the winning value only.  f: 5 planes (stride
// `plane`) of the projected fields.
__device__ __forceinline__ void record_node_cone(const float *f, long long plane, long long p, int i, int j, int ny,
                                                 int nx, float h, float eps, bool is_src, const float *T,
                                                 bool want_rec, uint8_t &id, float &w1, float d[5], float &r) {
  id = 0;
  w1 = 0.0f;
  r = 0.0f;
#pragma unroll
  for (int c = 0; c < 5; ++c) d[c] = 0.0f;
  const float T0 = T[p];
  if (is_src || !(T0 < kInf)) return;
  float Tn[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int ii = i + nb_dy(q), jj = j + nb_dx(q);
    Tn[q] = (ii >= 0 && ii < ny && jj >= 0 && jj < nx) ? T[(long long)ii * nx + jj] : kInf;
  }
  const float l11 = f[p], l21 = f[plane + p], l22 = f[2 * plane + p], wx = f[3 * plane + p], wy = f[4 * plane + p];
  float4 qr[kPlanes];
  node_record(l11, l21, l22, wx, wy, h, eps, false, qr);
  const float len[4] = {qr[0].x, qr[0].y, qr[0].z, qr[0].w};
  const float wm[4] = {qr[1].x, qr[1].y, qr[1].z, qr[1].w};
  const float C[4] = {qr[3].x, qr[3].y, qr[3].z, qr[3].w};
  const float mid[4] = {qr[4].x, qr[4].y, qr[4].z, qr[4].w};
  const float hw[4] = {qr[5].x, qr[5].y, qr[5].z, qr[5].w};
  float S[8];
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) S[nb] = (nb < 4) ? Tn[nb] - wm[nb] : Tn[nb] + wm[nb - 4];
  float all = kInf, best = kInf;
  int bid = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int a = k, b = (k + 1) & 7, pr = k & 3;
    const bool xs = (k & 2) != 0;
    const float Pk = xs ? qr[2].x : qr[2].z, Qk = xs ? qr[2].y : qr[2].w;
    const float dd = S[b] - S[a];
    const float qd = fmaf(-Qk, dd * dd, Pk);
    const float Tc = fmaf(C[pr], dd, S[a]) + qd * rsqrt_ftz(qd);
    if ((fabsf(dd - mid[pr]) < hw[pr]) && (fmaxf(Tn[a], Tn[b]) < Tc)) {
      all = fminf(all, Tc);
      if (Tc < best && Tn[a] < T0 && Tn[b] < T0) {
        best = Tc;
        bid = 0x20 | k;
      }
    }
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    if (Tn[n] < kInf) {
      const float v = S[n] + len[len_class(n)];
      all = fminf(all, v);
      if (v < best && Tn[n] < T0) {
        best = v;
        bid = 0x10 | n;
      }
    }
  }
  if (all < kInf) r = T0 - all;
  if (!want_rec || !bid) return;
  id = (uint8_t)bid;
  const int k = bid & 7;
  float vx, vy;
  if (bid & 0x20) {
    const int k2 = (k + 1) & 7;
    const float la = len[len_class(k)], lb = len[len_class(k2)];
    const float lx = (k & 2) ? len[0] : len[1];
    const float e11 = la * la, e22 = lb * lb, e12 = 0.5f * (e11 + e22 - lx * lx);
    const float u1 = best - S[k], u2 = best - S[k2];
    const float l1 = fmaf(e22, u1, -e12 * u2), l2 = fmaf(e11, u2, -e12 * u1);
    const float sum = l1 + l2;
    w1 = sum > 0.0f ? fminf(fmaxf(l1 / sum, 0.0f), 1.0f) : 0.5f;
    vx = h * (w1 * (float)nb_dx(k) + (1.0f - w1) * (float)nb_dx(k2));
    vy = h * (w1 * (float)nb_dy(k) + (1.0f - w1) * (float)nb_dy(k2));
  } else {
    w1 = 1.0f;
    vx = h * (float)nb_dx(k);
    vy = h * (float)nb_dy(k);
  }
  // dT0/dw = -v, dT0/dM = v v^T / (2 |v|_M), dT0/dL = 2 (dT0/dM) L
  const float m11 = fmaf(l11, l11, eps), m12 = l11 * l21, m22 = fmaf(l21, l21, fmaf(l22, l22, eps));
  const float vm = sqrtf(vx * (m11 * vx + m12 * vy) + vy * (m12 * vx + m22 * vy));
  const float s = 0.5f / vm;
  const float D11 = s * vx * vx, D12 = s * vx * vy, D22 = s * vy * vy;
  d[0] = 2.0f * (D11 * l11 + D12 * l21);
  d[1] = 2.0f * (D12 * l11 + D22 * l21);
  d[2] = 2.0f * D22 * l22;
  d[3] = -vx;
  d[4] = -vy;
}

}  // namespace rf
