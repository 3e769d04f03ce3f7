// rf_metric.cu -- the paper's own parameterisation of the metric and drift
// (App. B, "Feasibility Projections" and "Total Variation Regularization";
// Eq. 8): the eigenvalue-clamp projection of G, the drift clip and
// G^-1-norm rescale, the factor form the solver reads, their backward, and
// the drift / Frobenius / Log-Euclidean total-variation regularisers with
// their gradients.
//
// All three kernels are elementwise or 5-point stencils over SoA planes and
// bound by HBM: projection 20 B read + 40 B written per node; backward
// 20 + 20 + 20 B read + 20 B written; TV 20 B read + 40 B read-modify-write
// of the gradient.  The TV kernel stages a 34 x 10 halo tile of the
// (transformed) fields in shared memory so every node is read once per tile.
#include <cmath>

#include "rf_ctx.h"

namespace rf {

// ---------------------------------------------------------------------------
// per-node eigen-structure of a symmetric 2x2 matrix, without trigonometry:
// with r = sqrt((g11-g22)^2 + 4 g12^2), cos 2theta = (g11-g22)/r and
// sin 2theta = 2 g12/r are the double-angle values of the principal angle
// theta = atan2(2 g12, g11 - g22)/2 (theta = 0 when r = 0).
// ---------------------------------------------------------------------------
struct Eig2 {
  float lp, lm, r, c2, s2;
};

__device__ __forceinline__ Eig2 eig2(float g11, float g12, float g22) {
  Eig2 e;
  const float d = g11 - g22, t = 2.0f * g12;
  e.r = sqrtf(fmaf(d, d, t * t));
  const float tr = g11 + g22;
  e.lp = 0.5f * (tr + e.r);
  e.lm = 0.5f * (tr - e.r);
  const bool iso = !(e.r > 0.0f);
  const float ir = iso ? 0.0f : __frcp_rn(e.r);
  e.c2 = iso ? 1.0f : d * ir;
  e.s2 = t * ir;
  return e;
}

// U diag(mp, mm) U^T in double-angle form
__device__ __forceinline__ void from_eig(const Eig2 &e, float mp, float mm, float &o11, float &o12,
                                         float &o22) {
  const float hs = 0.5f * (mp + mm), hd = 0.5f * (mp - mm);
  o11 = fmaf(hd, e.c2, hs);
  o22 = fmaf(-hd, e.c2, hs);
  o12 = hd * e.s2;
}

// Daleckii-Krein adjoint on component gradients (d11, d12, d22), the
// symmetric-matrix gradient being [[d11, d12/2], [d12/2, d22]]; F the
// divided-difference matrix of the scalar function.  Returns components.
__device__ __forceinline__ void dk_adjoint(const Eig2 &e, float F11, float F12, float F22, float &d11,
                                           float &d12, float &d22) {
  const float cc = 0.5f * (1.0f + e.c2), ss = 0.5f * (1.0f - e.c2), cs = 0.5f * e.s2;
  const float S11 = d11, S12 = 0.5f * d12, S22 = d22;
  const float A11 = cc * S11 + e.s2 * S12 + ss * S22;
  const float A22 = ss * S11 - e.s2 * S12 + cc * S22;
  const float A12 = cs * (S22 - S11) + e.c2 * S12;
  const float B11 = F11 * A11, B12 = F12 * A12, B22 = F22 * A22;
  d11 = cc * B11 - e.s2 * B12 + ss * B22;
  d22 = ss * B11 + e.s2 * B12 + cc * B22;
  d12 = 2.0f * (cs * (B11 - B22) + e.c2 * B12);
}

// Forward intermediates of one node, shared by the projection and its
// backward so both take the same branch decisions in the same precision.
struct ProjNode {
  Eig2 e;
  float mp, mm;          // clamped eigenvalues
  float o11, o12, o22;   // projected G
  float bn;              // |b|_2
  bool clip_e;           // Euclidean clip taken
  float e1, e2;          // drift after the Euclidean clip
  float p1, p2, n;       // G^-1 e and |e|_{G^-1}
  bool clip_n;           // G^-1-norm rescale taken
  float q1, q2;          // projected drift
  float l11, l21, l22;   // chol(G - eps I)
};

__device__ __forceinline__ ProjNode proj_node(float g11, float g12, float g22, float b1, float b2,
                                              const rf_metric_params &m) {
  ProjNode P;
  P.e = eig2(g11, g12, g22);
  P.mp = fminf(fmaxf(P.e.lp, m.lam_min), m.lam_max);
  P.mm = fminf(fmaxf(P.e.lm, m.lam_min), m.lam_max);
  from_eig(P.e, P.mp, P.mm, P.o11, P.o12, P.o22);
  P.bn = hypotf(b1, b2);
  P.clip_e = P.bn > m.b_max;
  const float se = P.clip_e ? m.b_max / P.bn : 1.0f;
  P.e1 = b1 * se;
  P.e2 = b2 * se;
  const float det = P.mp * P.mm;  // det of the projected G
  P.p1 = (P.o22 * P.e1 - P.o12 * P.e2) / det;
  P.p2 = (P.o11 * P.e2 - P.o12 * P.e1) / det;
  P.n = sqrtf(fmaxf(fmaf(P.e1, P.p1, P.e2 * P.p2), 0.0f));
  const float c = 1.0f - m.delta;
  P.clip_n = P.n > c;
  const float sn = P.clip_n ? c / P.n : 1.0f;
  P.q1 = P.e1 * sn;
  P.q2 = P.e2 * sn;
  const float a11 = P.o11 - m.eps;
  P.l11 = sqrtf(a11);
  P.l21 = P.o12 / P.l11;
  // l22^2 = det(G - eps I) / (G - eps I)_11, det(G - eps I) = (mp-eps)(mm-eps)
  P.l22 = sqrtf((P.mp - m.eps) * (P.mm - m.eps) / a11);
  return P;
}

// V consecutive nodes of one plane (V = 4: one 16-byte load or store).
// Plain (coherent) loads: the projection may run in place.
template <int V>
struct Vec {
  float v[V];
};

template <int V>
__device__ __forceinline__ Vec<V> ldv(const float *p) {
  Vec<V> r;
  if constexpr (V == 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    r.v[0] = t.x;
    r.v[1] = t.y;
    r.v[2] = t.z;
    r.v[3] = t.w;
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) r.v[k] = p[k];
  }
  return r;
}

template <int V>
__device__ __forceinline__ void stv(float *p, const Vec<V> &r) {
  if constexpr (V == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) p[k] = r.v[k];
  }
}

struct MetricArgs {
  long long n;
  const float *gb;   // 5 planes
  float *gbp;        // 5 planes or null
  float *proj;       // 5 planes or null
  rf_metric_params m;
  DevState *st;
};

// V nodes per thread and iteration (V = 4 when n and every plane base are
// 16-byte aligned): 5 x 16 B in flight per thread keeps enough bytes in
// flight for HBM at 2-3 CTAs per SM; the grid is exactly the
// resident CTAs, striding over the nodes.
template <int V>
__global__ void __launch_bounds__(256, 3) metric_project_kernel(MetricArgs a) {
  const long long n = a.n, units = n / V;
  bool bad = false;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
       u += (long long)gridDim.x * blockDim.x) {
    const long long p = u * V;
    Vec<V> in[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) in[c] = ldv<V>(a.gb + c * n + p);
    Vec<V> o[5], l[5];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float g11 = in[0].v[k], g12 = in[1].v[k], g22 = in[2].v[k], b1 = in[3].v[k], b2 = in[4].v[k];
      bad |= !(isfinite(g11) && isfinite(g12) && isfinite(g22) && isfinite(b1) && isfinite(b2));
      const ProjNode P = proj_node(g11, g12, g22, b1, b2, a.m);
      o[0].v[k] = P.o11;
      o[1].v[k] = P.o12;
      o[2].v[k] = P.o22;
      o[3].v[k] = P.q1;
      o[4].v[k] = P.q2;
      l[0].v[k] = P.l11;
      l[1].v[k] = P.l21;
      l[2].v[k] = P.l22;
      l[3].v[k] = -P.q1;
      l[4].v[k] = -P.q2;
    }
    if (a.gbp) {
#pragma unroll
      for (int c = 0; c < 5; ++c) stv<V>(a.gbp + c * n + p, o[c]);
    }
    if (a.proj) {
#pragma unroll
      for (int c = 0; c < 5; ++c) stv<V>(a.proj + c * n + p, l[c]);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_error(a.st, RF_ERR_NONFINITE_INPUT);
}

struct MetricBwdArgs {
  long long n;
  const float *gb;
  const float *dproj;  // 5 planes or null
  const float *dgbp;   // 5 planes or null
  float *dgb;
  rf_metric_params m;
};

// backward of one node from its raw inputs and the two incoming gradients
__device__ __forceinline__ void project_backward_node(const float in[5], float dl[5], const float dq[5],
                                                      bool has_dl, bool has_dq, const rf_metric_params &m,
                                                      float out[5]) {
  const ProjNode P = proj_node(in[0], in[1], in[2], in[3], in[4], m);
  const float c = 1.0f - m.delta;
  float d11 = 0.f, d12 = 0.f, d22 = 0.f, db1 = 0.f, db2 = 0.f;
  if (has_dl) {
    // L = chol(G - eps I), w = -b, in reverse
    d22 = dl[2] / (2.0f * P.l22);
    const float dl21b = dl[1] - dl[2] * P.l21 / P.l22;
    d12 = dl21b / P.l11;
    d11 = (dl[0] - dl21b * P.l21 / P.l11) / (2.0f * P.l11);
    db1 = -dl[3];
    db2 = -dl[4];
  }
  if (has_dq) {
    d11 += dq[0];
    d12 += dq[1];
    d22 += dq[2];
    db1 += dq[3];
    db2 += dq[4];
  }
  // drift rescale q = c e / n(e, G): into e and into the projected G
  float de1 = db1, de2 = db2;
  if (P.clip_n) {
    const float bg = db1 * P.e1 + db2 * P.e2;
    const float inv = 1.0f / P.n, in2 = inv * inv;
    de1 = c * inv * (db1 - P.p1 * bg * in2);
    de2 = c * inv * (db2 - P.p2 * bg * in2);
    const float k = 0.5f * c * bg * in2 * inv;
    d11 += k * P.p1 * P.p1;
    d12 += 2.0f * k * P.p1 * P.p2;
    d22 += k * P.p2 * P.p2;
  }
  // Euclidean clip e = b b_max/|b|
  if (P.clip_e) {
    const float ib = 1.0f / P.bn;
    const float be = (in[3] * de1 + in[4] * de2) * ib * ib;
    de1 = m.b_max * ib * (de1 - in[3] * be);
    de2 = m.b_max * ib * (de2 - in[4] * be);
  }
  // eigenvalue clamp (Daleckii-Krein): f' = 1 inside [lam_min, lam_max]
  const float Fp = (P.e.lp >= m.lam_min && P.e.lp <= m.lam_max) ? 1.0f : 0.0f;
  const float Fm = (P.e.lm >= m.lam_min && P.e.lm <= m.lam_max) ? 1.0f : 0.0f;
  const float F12 = P.e.r > 0.0f ? (P.mp - P.mm) / P.e.r : Fp;
  dk_adjoint(P.e, Fp, F12, Fm, d11, d12, d22);
  out[0] = d11;
  out[1] = d12;
  out[2] = d22;
  out[3] = de1;
  out[4] = de2;
}

template <int V>
__global__ void __launch_bounds__(256, 2) metric_project_backward_kernel(MetricBwdArgs a) {
  const long long n = a.n, units = n / V;
  const bool has_dl = a.dproj != nullptr, has_dq = a.dgbp != nullptr;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
       u += (long long)gridDim.x * blockDim.x) {
    const long long p = u * V;
    Vec<V> in[5], dl[5], dq[5], out[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      in[c] = ldv<V>(a.gb + c * n + p);
      if (has_dl) dl[c] = ldv<V>(a.dproj + c * n + p);
      if (has_dq) dq[c] = ldv<V>(a.dgbp + c * n + p);
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      float i5[5], l5[5], q5[5], o5[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        i5[c] = in[c].v[k];
        l5[c] = has_dl ? dl[c].v[k] : 0.0f;
        q5[c] = has_dq ? dq[c].v[k] : 0.0f;
      }
      project_backward_node(i5, l5, q5, has_dl, has_dq, a.m, o5);
#pragma unroll
      for (int c = 0; c < 5; ++c) out[c].v[k] = o5[c];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) stv<V>(a.dgb + c * n + p, out[c]);
  }
}

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// grid-stride grid of exactly the resident CTAs (no partial last wave)
template <class K>
inline int resident_grid(K kernel, const rf_ctx *ctx, long long units) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return blocks_for(units, 256, ctx->num_sms * per_sm);
}

// ---------------------------------------------------------------------------
// total variation
// ---------------------------------------------------------------------------
constexpr int kTvX = 32, kTvY = 8;          // nodes per tile (one thread each)
constexpr int kTvFX = kTvX + 2, kTvFY = kTvY + 2;  // staged field: one halo each side
constexpr int kTvUX = kTvX + 1, kTvUY = kTvY + 1;  // unit differences: left/top halo

struct TvArgs {
  int ny, nx;
  const float *gb;
  int mode;
  float wg, wb;
  float *partial;  // [blocks][2]
  float *grad;     // 5 planes or null
  DevState *st;
};

// log G on the eigenvectors (G SPD): components of U diag(log lp, log lm) U^T;
// e and hd = (log lp - log lm)/2 are returned for the backward's factors
__device__ __forceinline__ bool logm2(float g11, float g12, float g22, float &l11, float &l12,
                                      float &l22, Eig2 &e, float &hd) {
  e = eig2(g11, g12, g22);
  if (!(e.lm > 0.0f) || !isfinite(e.lp)) return false;
  const float ll = logf(e.lm);
  hd = 0.5f * log1pf(e.r / e.lm);  // (log lp - log lm)/2 without cancellation
  const float hs = ll + hd;
  l11 = fmaf(hd, e.c2, hs);
  l22 = fmaf(-hd, e.c2, hs);
  l12 = hd * e.s2;
  return true;
}

template <int MODE>
__global__ void __launch_bounds__(kTvX * kTvY, 8) tv_kernel(TvArgs a) {
  constexpr int NC = MODE == RF_TV_NONE ? 2 : 5;  // staged components
  constexpr int C0 = MODE == RF_TV_NONE ? 3 : 0;  // first plane staged
  __shared__ float f[NC][kTvFY][kTvFX];
  __shared__ float ux[NC][kTvUY][kTvUX], uy[NC][kTvUY][kTvUX];
  __shared__ float red[2][kTvX * kTvY / 32];
  // Log-Euclidean: the Daleckii-Krein factors of the tile's own nodes
  // (cos 2theta, sin 2theta, 1/lp, (log lp - log lm)/(lp - lm), 1/lm)
  __shared__ float dk[MODE == RF_TV_LOG_EUCLIDEAN ? 5 : 1][kTvY][kTvX];
  const int x0 = blockIdx.x * kTvX, y0 = blockIdx.y * kTvY;
  const int nx = a.nx, ny = a.ny;
  const long long n = (long long)nx * ny;
  const int tid = threadIdx.x;
  bool bad = false;
  // 1. stage rows y0-1 .. y0+kTvY, columns x0-1 .. x0+kTvX (log G for LE)
  for (int i = tid; i < kTvFY * kTvFX; i += blockDim.x) {
    const int fy = i / kTvFX, fx = i - fy * kTvFX;
    const int y = y0 - 1 + fy, x = x0 - 1 + fx;
    float v[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = 0.0f;
    if (y >= 0 && y < ny && x >= 0 && x < nx) {
      const long long p = (long long)y * nx + x;
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = __ldg(a.gb + (C0 + c) * n + p);
      if constexpr (MODE == RF_TV_LOG_EUCLIDEAN) {
        float l11, l12, l22, hd;
        Eig2 e;
        const bool ok = logm2(v[0], v[1], v[2], l11, l12, l22, e, hd);
        if (!ok) {
          bad = true;
          l11 = l12 = l22 = 0.0f;
        }
        v[0] = l11;
        v[1] = l12;
        v[2] = l22;
        if (fy >= 1 && fy <= kTvY && fx >= 1 && fx <= kTvX) {
          const int oy = fy - 1, ox = fx - 1;
          dk[0][oy][ox] = e.c2;
          dk[1][oy][ox] = e.s2;
          dk[2][oy][ox] = ok ? 1.0f / e.lp : 0.0f;
          dk[3][oy][ox] = ok ? (e.r > 0.0f ? 2.0f * hd / e.r : 1.0f / e.lp) : 0.0f;
          dk[4][oy][ox] = ok ? 1.0f / e.lm : 0.0f;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) f[c][fy][fx] = v[c];
  }
  __syncthreads();
  // 2. normalised differences u = w D f / N at nodes rows y0-1 .. y0+kTvY-1,
  //    columns x0-1 .. x0+kTvX-1 (zero outside the grid and at N = 0);
  //    the norms of the tile's own nodes go to the value sums
  float sg = 0.0f, sb = 0.0f;
  for (int i = tid; i < kTvUY * kTvUX; i += blockDim.x) {
    const int uyi = i / kTvUX, uxi = i - uyi * kTvUX;
    const int y = y0 - 1 + uyi, x = x0 - 1 + uxi;
    const bool in = y >= 0 && y < ny && x >= 0 && x < nx;
    const bool hx = in && x + 1 < nx, hy = in && y + 1 < ny;
    float dx[NC], dy[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      // node (y, x) is staged at f[.][uyi][uxi]
      dx[c] = hx ? f[c][uyi][uxi + 1] - f[c][uyi][uxi] : 0.0f;
      dy[c] = hy ? f[c][uyi + 1][uxi] - f[c][uyi][uxi] : 0.0f;
    }
    const bool own = uyi >= 1 && uxi >= 1 && in;
    if constexpr (MODE != RF_TV_NONE) {
      const float s = dx[0] * dx[0] + dy[0] * dy[0] + 2.0f * (dx[1] * dx[1] + dy[1] * dy[1]) +
                      dx[2] * dx[2] + dy[2] * dy[2];
      const float N = sqrtf(s);
      const float inv = N > 0.0f ? 1.0f / N : 0.0f;
      const float w[3] = {1.0f, 2.0f, 1.0f};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        ux[c][uyi][uxi] = w[c] * dx[c] * inv;
        uy[c][uyi][uxi] = w[c] * dy[c] * inv;
      }
      if (own) sg += N;
    }
    {
      constexpr int B0 = NC - 2;
      const float N = sqrtf(dx[B0] * dx[B0] + dy[B0] * dy[B0] + dx[B0 + 1] * dx[B0 + 1] +
                            dy[B0 + 1] * dy[B0 + 1]);
      const float inv = N > 0.0f ? 1.0f / N : 0.0f;
#pragma unroll
      for (int c = B0; c < NC; ++c) {
        ux[c][uyi][uxi] = dx[c] * inv;
        uy[c][uyi][uxi] = dy[c] * inv;
      }
      if (own) sb += N;
    }
  }
  // block sums of the norms (fixed order: warp shuffles, then warp 0)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sg += __shfl_xor_sync(0xffffffffu, sg, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = sg;
    red[1][tid >> 5] = sb;
  }
  __syncthreads();
  if (tid == 0) {
    float tg = 0.0f, tb = 0.0f;
    for (int w = 0; w < kTvX * kTvY / 32; ++w) {
      tg += red[0][w];
      tb += red[1][w];
    }
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    a.partial[2 * blk] = tg;
    a.partial[2 * blk + 1] = tb;
  }
  if (__syncthreads_or(bad) && tid == 0) set_error(a.st, RF_ERR_NONFINITE_INPUT);
  // 3. gradient at the tile's own node: adjoint of the forward differences
  if (!a.grad) return;
  const int ty = tid / kTvX, tx = tid - ty * kTvX;
  const int y = y0 + ty, x = x0 + tx;
  if (y >= ny || x >= nx) return;
  const long long p = (long long)y * nx + x;
  const int ui = ty + 1, uj = tx + 1;
  float g[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    g[c] = -ux[c][ui][uj] - uy[c][ui][uj];
    if (x > 0) g[c] += ux[c][ui][uj - 1];
    if (y > 0) g[c] += uy[c][ui - 1][uj];
  }
  if constexpr (MODE == RF_TV_LOG_EUCLIDEAN) {
    // back through log G: F_ii = 1/lambda_i, F_12 = (log lp - log lm)/(lp - lm)
    // (a non-SPD node has all factors 0 and contributes nothing)
    Eig2 e;
    e.c2 = dk[0][ty][tx];
    e.s2 = dk[1][ty][tx];
    dk_adjoint(e, dk[2][ty][tx], dk[3][ty][tx], dk[4][ty][tx], g[0], g[1], g[2]);
  }
  if constexpr (MODE != RF_TV_NONE) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.grad[c * n + p] += a.wg * g[c];
  }
  a.grad[3 * n + p] += a.wb * g[NC - 2];
  a.grad[4 * n + p] += a.wb * g[NC - 1];
}

// deterministic final sum of the per-block partials (double accumulation)
__global__ void __launch_bounds__(1024) tv_reduce_kernel(const float *partial, int blocks, int mode,
                                                         float *value2) {
  __shared__ double s[2][32];
  double a0 = 0.0, a1 = 0.0;
  for (int i = threadIdx.x; i < blocks; i += blockDim.x) {
    a0 += partial[2 * i];
    a1 += partial[2 * i + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s[0][threadIdx.x >> 5] = a0;
    s[1][threadIdx.x >> 5] = a1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t0 += s[0][w];
      t1 += s[1][w];
    }
    value2[0] = mode == RF_TV_NONE ? 0.0f : (float)t0;
    value2[1] = (float)t1;
  }
}

inline bool params_ok(const rf_metric_params *m) {
  return m && m->eps >= 0.0f && m->lam_min > m->eps && m->lam_max >= m->lam_min &&
         std::isfinite(m->lam_max) && m->b_max > 0.0f && m->delta > 0.0f && m->delta < 1.0f;
}

}  // namespace rf

using namespace rf;

extern "C" rf_status rf_metric_project(rf_ctx *ctx, const rf_grid *grid, const float *gb5,
                                       const rf_metric_params *prm, float *gbp5, float *proj5,
                                       void *stream) {
  if (!ctx || !grid_ok(grid) || !gb5 || !params_ok(prm)) return RF_ERR_INVALID_ARG;
  if (!gbp5 && !proj5) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  MetricArgs a;
  a.n = (long long)grid->ny * grid->nx;
  a.gb = gb5;
  a.gbp = gbp5;
  a.proj = proj5;
  a.m = *prm;
  a.st = ctx->state;
  const bool vec = a.n % 4 == 0 && aligned16(gb5) && (!gbp5 || aligned16(gbp5)) && (!proj5 || aligned16(proj5));
  if (vec)
    metric_project_kernel<4><<<resident_grid(metric_project_kernel<4>, ctx, a.n / 4), 256, 0, s>>>(a);
  else
    metric_project_kernel<1><<<resident_grid(metric_project_kernel<1>, ctx, a.n), 256, 0, s>>>(a);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_metric_project_backward(rf_ctx *ctx, const rf_grid *grid, const float *gb5,
                                                const rf_metric_params *prm, const float *dproj5,
                                                const float *dgbp5, float *dgb5, void *stream) {
  if (!ctx || !grid_ok(grid) || !gb5 || !params_ok(prm) || !dgb5) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  MetricBwdArgs a;
  a.n = (long long)grid->ny * grid->nx;
  a.gb = gb5;
  a.dproj = dproj5;
  a.dgbp = dgbp5;
  a.dgb = dgb5;
  a.m = *prm;
  const bool vec = a.n % 4 == 0 && aligned16(gb5) && aligned16(dgb5) && (!dproj5 || aligned16(dproj5)) &&
                   (!dgbp5 || aligned16(dgbp5));
  if (vec)
    metric_project_backward_kernel<4><<<resident_grid(metric_project_backward_kernel<4>, ctx, a.n / 4), 256, 0,
                                         s>>>(a);
  else
    metric_project_backward_kernel<1><<<resident_grid(metric_project_backward_kernel<1>, ctx, a.n), 256, 0,
                                         s>>>(a);
  return cuda_status(cudaGetLastError());
}

extern "C" rf_status rf_tv(rf_ctx *ctx, const rf_grid *grid, const float *gb5, int metric_mode,
                           float w_metric, float w_drift, float *value2, float *grad5,
                           void *stream) {
  if (!ctx || !grid_ok(grid) || !gb5) return RF_ERR_INVALID_ARG;
  if (metric_mode != RF_TV_NONE && metric_mode != RF_TV_FROBENIUS &&
      metric_mode != RF_TV_LOG_EUCLIDEAN)
    return RF_ERR_INVALID_ARG;
  if (!value2 && !grad5) return RF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  dim3 grid2((grid->nx + kTvX - 1) / kTvX, (grid->ny + kTvY - 1) / kTvY);
  const long long blocks = (long long)grid2.x * grid2.y;
  rf_status r = ensure(&ctx->tvbuf, &ctx->tvbuf_cap, (size_t)(2 * blocks));
  if (r != RF_OK) return r;
  TvArgs a;
  a.ny = grid->ny;
  a.nx = grid->nx;
  a.gb = gb5;
  a.mode = metric_mode;
  a.wg = w_metric;
  a.wb = w_drift;
  a.partial = ctx->tvbuf;
  a.grad = grad5;
  a.st = ctx->state;
  if (metric_mode == RF_TV_FROBENIUS)
    tv_kernel<RF_TV_FROBENIUS><<<grid2, kTvX * kTvY, 0, s>>>(a);
  else if (metric_mode == RF_TV_LOG_EUCLIDEAN)
    tv_kernel<RF_TV_LOG_EUCLIDEAN><<<grid2, kTvX * kTvY, 0, s>>>(a);
  else
    tv_kernel<RF_TV_NONE><<<grid2, kTvX * kTvY, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return RF_ERR_CUDA;
  if (value2) tv_reduce_kernel<<<1, 1024, 0, s>>>(ctx->tvbuf, (int)blocks, metric_mode, value2);
  return cuda_status(cudaGetLastError());
}
