/*
 * rf_oracle.c -- plain, slow FP64 CPU oracle for the differentiable
 * Randers eikonal solver (arXiv 2603.00035).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path in
 * paper_2603_00035_gb300/csrc; the two meet only through the seeded inputs
 * that the tests hand to both.
 *
 * Notation follows the paper: metric G (here M = L L^T + eps I), drift b.
 * The build uses F(x,v) = sqrt(v^T M v) + w^T v, which is the paper's
 * two-point / one-point update (Eqs. 2-3) with G = M and b = -w:
 *     S_i = T_i + m_i . b = T_i - m_i . w.
 *
 * Grid: node (i,j) sits at (x,y) = (j h, i h), row-major [ny][nx].
 * Neighbour ring (Fig. 4a): eight neighbours numbered counter-clockwise from
 * the upper-left one; stencil k uses neighbours k and (k+1) mod 8.
 *
 * Readings of the paper used here:
 *  - every finite neighbour contributes its one-point candidate (Eq. 3) and
 *    every stencil with two finite donors contributes its two-point candidate
 *    (Eq. 2) when valid; the node takes the minimum (Sec. 3.2, App. A);
 *  - validity of a two-point candidate = real root, T_1 < T_0, T_2 < T_0 and
 *    lambda = Q (T_0 1 - S) >= 0 componentwise (App. A);
 *  - out-of-grid neighbours are +inf; sources are fixed at 0;
 *  - ties between candidates: strict '<' in the order two-point k = 0..7,
 *    then one-point n = 0..7; the first minimum names the active stencil.
 *
 * Every function states the passage it follows.  Parity unpinned: none
 * (each function is pinned by a -m "not gpu" test, see tests/test_oracle_*).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_NOT_CONVERGED 3
#define ORC_ERR_NO_SOURCE 6

/* Fig. 4(a): offsets (dx, dy) of neighbours 0..7, counter-clockwise from the
 * upper-left.  "Up" is +y, i.e. +i (row index grows with y). */
static const int ORC_DX[8] = {-1, -1, -1, 0, 1, 1, 1, 0};
static const int ORC_DY[8] = {1, 0, -1, -1, -1, 0, 1, 1};

/* Metric from the lower-triangular factor: M = L L^T + eps I. */
static void metric_from_L(double l11, double l21, double l22, double eps,
                          double *g11, double *g12, double *g22) {
  *g11 = l11 * l11 + eps;
  *g12 = l11 * l21;
  *g22 = l21 * l21 + l22 * l22 + eps;
}

static double quad(double g11, double g12, double g22, double ax, double ay,
                   double bx, double by) {
  /* a^T G b */
  return ax * (g11 * bx + g12 * by) + ay * (g12 * bx + g22 * by);
}

/* Candidate set of one node, given the eight neighbour times. */
typedef struct {
  double two[8];     /* two-point candidate of stencil k (Eq. 2)         */
  int two_ok[8];     /* 1 if valid                                         */
  double lam[8][2];  /* lambda = Q (T0 1 - S) of stencil k                 */
  int two_geo_only[8]; /* real root and lambda >= 0 but causality failed  */
  double one[8];     /* one-point candidate through neighbour n (Eq. 3)    */
  int one_ok[8];
} orc_cands;

/*
 * Local update at one node (Sec. 3.2, Eqs. 2-3; App. A "Two-Point Update",
 * "One-Point Fallback").  Tn[n] = arrival time of neighbour n (+inf when
 * missing).  m_n = h (dx_n, dy_n) is the displacement from the node to
 * neighbour n.
 */
static void cell_candidates(const double Tn[8], double h, double g11,
                            double g12, double g22, double wx, double wy,
                            orc_cands *c) {
  double mx[8], my[8], S[8];
  for (int n = 0; n < 8; ++n) {
    mx[n] = h * ORC_DX[n];
    my[n] = h * ORC_DY[n];
    /* drift-adjusted time S_n = T_n + m_n . b with b = -w */
    S[n] = Tn[n] - (mx[n] * wx + my[n] * wy);
    /* Eq. 3: T0 = T_n + m_n . b + sqrt(m_n^T G m_n) */
    c->one_ok[n] = isfinite(Tn[n]);
    c->one[n] = c->one_ok[n]
                    ? S[n] + sqrt(quad(g11, g12, g22, mx[n], my[n], mx[n], my[n]))
                    : INFINITY;
  }
  for (int k = 0; k < 8; ++k) {
    int a = k, b = (k + 1) & 7;
    c->two[k] = INFINITY;
    c->two_ok[k] = 0;
    c->two_geo_only[k] = 0;
    c->lam[k][0] = c->lam[k][1] = 0.0;
    if (!isfinite(Tn[a]) || !isfinite(Tn[b]))
      continue;
    /* stencil matrix Mm = [m1 | m2]; stencil metric E = Mm^T G Mm */
    double e11 = quad(g11, g12, g22, mx[a], my[a], mx[a], my[a]);
    double e12 = quad(g11, g12, g22, mx[a], my[a], mx[b], my[b]);
    double e22 = quad(g11, g12, g22, mx[b], my[b], mx[b], my[b]);
    double det = e11 * e22 - e12 * e12;
    if (!(det > 0.0))
      continue;
    /* Q = E^{-1} */
    double q11 = e22 / det, q12 = -e12 / det, q22 = e11 / det;
    /* Quadratic (S - T0 1)^T Q (S - T0 1) = 1, written for tau = T0 - min S
     * (a translation of the same quadratic): (s - tau 1)^T Q (s - tau 1) = 1
     * with s = S - min(S) 1. */
    double smin = S[a] < S[b] ? S[a] : S[b];
    double s1 = S[a] - smin, s2 = S[b] - smin;
    double qa = q11 + 2.0 * q12 + q22;                   /* 1^T Q 1     */
    double qb = (q11 + q12) * s1 + (q12 + q22) * s2;     /* 1^T Q s     */
    double qc = q11 * s1 * s1 + 2.0 * q12 * s1 * s2 + q22 * s2 * s2 - 1.0;
    double disc = qb * qb - qa * qc;
    if (disc < 0.0)
      continue;
    double tau = (qb + sqrt(disc)) / qa; /* larger root */
    double T0 = smin + tau;
    /* lambda = Q (T0 1 - S) */
    double u1 = T0 - S[a], u2 = T0 - S[b];
    double l1 = q11 * u1 + q12 * u2;
    double l2 = q12 * u1 + q22 * u2;
    c->lam[k][0] = l1;
    c->lam[k][1] = l2;
    int geo = (l1 >= 0.0) && (l2 >= 0.0);
    int causal = (Tn[a] < T0) && (Tn[b] < T0);
    c->two[k] = T0;
    c->two_ok[k] = geo && causal;
    c->two_geo_only[k] = geo && !causal;
  }
}

/* Minimum valid candidate and its identity (tie-break: two-point k=0..7,
 * then one-point n=0..7, strict '<').  *kind: 0 none, 1 one-point, 2 two. */
static double cell_best(const orc_cands *c, int *kind, int *idx,
                        double *second) {
  double best = INFINITY, sec = INFINITY;
  int bk = 0, bi = 0;
  for (int k = 0; k < 8; ++k)
    if (c->two_ok[k]) {
      if (c->two[k] < best) {
        sec = best;
        best = c->two[k];
        bk = 2;
        bi = k;
      } else if (c->two[k] < sec) {
        sec = c->two[k];
      }
    }
  for (int n = 0; n < 8; ++n)
    if (c->one_ok[n]) {
      if (c->one[n] < best) {
        sec = best;
        best = c->one[n];
        bk = 1;
        bi = n;
      } else if (c->one[n] < sec) {
        sec = c->one[n];
      }
    }
  if (kind) *kind = bk;
  if (idx) *idx = bi;
  if (second) *second = sec;
  return best;
}

static void gather_neighbours(int ny, int nx, const double *T, int i, int j,
                              const uint8_t *accepted, double Tn[8]) {
  for (int n = 0; n < 8; ++n) {
    int ii = i + ORC_DY[n], jj = j + ORC_DX[n];
    if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) {
      Tn[n] = INFINITY;
      continue;
    }
    size_t q = (size_t)ii * nx + jj;
    Tn[n] = (accepted && !accepted[q]) ? INFINITY : T[q];
  }
}

/* Evaluate the candidate set of node (i,j) with the current field T. */
static void node_candidates(int ny, int nx, double h, double eps,
                            const double *L11, const double *L21,
                            const double *L22, const double *wx,
                            const double *wy, const double *T,
                            const uint8_t *accepted, int i, int j,
                            orc_cands *c) {
  size_t p = (size_t)i * nx + j;
  double g11, g12, g22, Tn[8];
  metric_from_L(L11[p], L21[p], L22[p], eps, &g11, &g12, &g22);
  gather_neighbours(ny, nx, T, i, j, accepted, Tn);
  cell_candidates(Tn, h, g11, g12, g22, wx[p], wy[p], c);
}

/* ------------------------------------------------------------------ */
/* Exported: one node's candidates from explicit inputs (for pin tests). */
void orc_cell_eval(const double *Tn, double h, double g11, double g12,
                   double g22, double wx, double wy, double *two,
                   int *two_ok, double *lam, double *one, int *one_ok) {
  orc_cands c;
  cell_candidates(Tn, h, g11, g12, g22, wx, wy, &c);
  for (int k = 0; k < 8; ++k) {
    two[k] = c.two[k];
    two_ok[k] = c.two_ok[k];
    lam[2 * k] = c.lam[k][0];
    lam[2 * k + 1] = c.lam[k][1];
    one[k] = c.one[k];
    one_ok[k] = c.one_ok[k];
  }
}

/* ------------------------------------------------------------------ */
/*
 * Feasibility projection (metric in factor form; w-norm formula of App. B):
 *   M = L L^T + eps I,   n = |w|_{M^-1} = sqrt((wx^2 M22 - 2 wx wy M12 +
 *   wy^2 M11) / det M),  w_out = w * min(1, c / n),  c = 1 - delta.
 * The boundary n == c counts as unclipped.  L passes through unchanged.
 */
int orc_project(int64_t n, const double *L11, const double *L21,
                const double *L22, const double *wx, const double *wy,
                double eps, double delta, double *wpx, double *wpy,
                uint8_t *clip) {
  if (n < 0 || !(delta > 0.0 && delta < 1.0) || eps < 0.0)
    return ORC_ERR_INVALID_ARG;
  double c = 1.0 - delta;
  for (int64_t p = 0; p < n; ++p) {
    double g11, g12, g22;
    metric_from_L(L11[p], L21[p], L22[p], eps, &g11, &g12, &g22);
    double det = g11 * g22 - g12 * g12;
    double nn = sqrt((wx[p] * wx[p] * g22 - 2.0 * wx[p] * wy[p] * g12 +
                      wy[p] * wy[p] * g11) / det);
    if (nn > c) {
      wpx[p] = wx[p] * (c / nn);
      wpy[p] = wy[p] * (c / nn);
      clip[p] = 1;
    } else {
      wpx[p] = wx[p];
      wpy[p] = wy[p];
      clip[p] = 0;
    }
  }
  return ORC_OK;
}

/*
 * Backward of orc_project.  Inputs: gradients with respect to the
 * solver-side parameters (L11, L21, L22, w_proj x, w_proj y), five planes of
 * n values each (gin).  Output: gradients with respect to the raw inputs
 * (gout, same layout).  For a clipped cell, with P = M^{-1}, g = dL/dw_out:
 *   dL/dw_raw = (c/n) (g - P w (w^T g) / n^2)
 *   dL/dM    += (c (w^T g) / (2 n^3)) (P w)(P w)^T      (symmetric form)
 * and dL/dL = 2 (dL/dM) L restricted to the lower triangle.
 */
int orc_project_backward(int64_t n, const double *L11, const double *L21,
                         const double *L22, const double *wx,
                         const double *wy, const uint8_t *clip, double eps,
                         double delta, const double *gin, double *gout) {
  if (n < 0)
    return ORC_ERR_INVALID_ARG;
  double c = 1.0 - delta;
  for (int64_t p = 0; p < n; ++p) {
    double gl11 = gin[p], gl21 = gin[n + p], gl22 = gin[2 * n + p];
    double gx = gin[3 * n + p], gy = gin[4 * n + p];
    if (clip[p]) {
      double g11, g12, g22;
      metric_from_L(L11[p], L21[p], L22[p], eps, &g11, &g12, &g22);
      double det = g11 * g22 - g12 * g12;
      /* P = M^{-1} */
      double p11 = g22 / det, p12 = -g12 / det, p22 = g11 / det;
      double pwx = p11 * wx[p] + p12 * wy[p];
      double pwy = p12 * wx[p] + p22 * wy[p];
      double n2 = wx[p] * pwx + wy[p] * pwy;
      double nn = sqrt(n2);
      double wg = wx[p] * gx + wy[p] * gy;
      double ox = (c / nn) * (gx - pwx * wg / n2);
      double oy = (c / nn) * (gy - pwy * wg / n2);
      double s = c * wg / (2.0 * nn * n2);
      double D11 = s * pwx * pwx, D12 = s * pwx * pwy, D22 = s * pwy * pwy;
      gl11 += 2.0 * (D11 * L11[p] + D12 * L21[p]);
      gl21 += 2.0 * (D12 * L11[p] + D22 * L21[p]);
      gl22 += 2.0 * D22 * L22[p];
      gx = ox;
      gy = oy;
    }
    gout[p] = gl11;
    gout[n + p] = gl21;
    gout[2 * n + p] = gl22;
    gout[3 * n + p] = gx;
    gout[4 * n + p] = gy;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
static int count_sources(int64_t n, const uint8_t *src) {
  int64_t k = 0;
  for (int64_t p = 0; p < n; ++p)
    k += src[p] != 0;
  return k > 0;
}

/*
 * Gauss-Seidel fast sweeping (Alg. 1; Sec. 3.2; App. A "Forward Solve").
 * T = 0 on sources, +inf elsewhere.  One iteration = four sweeps in the
 * paper's order: columns left->right, rows along +i, columns right->left,
 * rows along -i; nodes are updated in place, raster order inside a sweep,
 * T <- min(T, min valid candidate) (replace = 0, the literal Alg. 1) or
 * T <- min valid candidate (replace = 1; values may then also rise).  Stops
 * after the first iteration that changes no value bitwise in FP64 (the
 * paper's 1e-6 tolerance is replaced by exact no-change).
 */
int orc_solve_gs(int ny, int nx, double h, double eps, const double *L11,
                 const double *L21, const double *L22, const double *wx,
                 const double *wy, const uint8_t *src, double *T,
                 int max_iter, int replace, int *iters_out,
                 int64_t *updates_out) {
  if (ny < 1 || nx < 1 || !(h > 0.0))
    return ORC_ERR_INVALID_ARG;
  int64_t n = (int64_t)ny * nx;
  for (int64_t p = 0; p < n; ++p)
    T[p] = src[p] ? 0.0 : INFINITY;
  if (!count_sources(n, src)) {
    if (iters_out) *iters_out = 0;
    return ORC_ERR_NO_SOURCE;
  }
  int64_t updates = 0;
  int it;
  for (it = 1; it <= max_iter; ++it) {
    int changed = 0;
    for (int d = 0; d < 4; ++d) {
      int lines = (d % 2 == 0) ? nx : ny;
      int len = (d % 2 == 0) ? ny : nx;
      for (int s = 0; s < lines; ++s) {
        int line = (d < 2) ? s : lines - 1 - s;
        for (int q = 0; q < len; ++q) {
          int i = (d % 2 == 0) ? q : line;
          int j = (d % 2 == 0) ? line : q;
          size_t p = (size_t)i * nx + j;
          ++updates;
          if (src[p])
            continue;
          orc_cands c;
          node_candidates(ny, nx, h, eps, L11, L21, L22, wx, wy, T, NULL, i,
                          j, &c);
          double best = cell_best(&c, NULL, NULL, NULL);
          if (replace ? (best != T[p]) : (best < T[p])) {
            T[p] = best;
            changed = 1;
          }
        }
      }
    }
    if (!changed)
      break;
  }
  if (iters_out) *iters_out = it > max_iter ? max_iter : it;
  if (updates_out) *updates_out = updates;
  return it > max_iter ? ORC_ERR_NOT_CONVERGED : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Ordered (label-setting) solve of the same discrete system: a binary heap
 * of tentative values; the smallest is accepted; each unaccepted, non-source
 * neighbour re-evaluates its candidates using accepted neighbours only.
 * Correct because every valid candidate exceeds its donors (the causality
 * test of App. A, and |m|_M - w.m > 0 when |w|_{M^-1} < 1). */
typedef struct {
  double v;
  int64_t p;
} heap_item;

static void heap_push(heap_item *h, int64_t *sz, double v, int64_t p) {
  int64_t k = (*sz)++;
  while (k > 0) {
    int64_t par = (k - 1) / 2;
    if (h[par].v <= v)
      break;
    h[k] = h[par];
    k = par;
  }
  h[k].v = v;
  h[k].p = p;
}

static heap_item heap_pop(heap_item *h, int64_t *sz) {
  heap_item top = h[0];
  heap_item last = h[--(*sz)];
  int64_t k = 0;
  for (;;) {
    int64_t l = 2 * k + 1, r = l + 1, m = k;
    double mv = last.v;
    if (l < *sz && h[l].v < mv) {
      m = l;
      mv = h[l].v;
    }
    if (r < *sz && h[r].v < mv)
      m = r;
    if (m == k)
      break;
    h[k] = h[m];
    k = m;
  }
  if (*sz > 0)
    h[k] = last;
  return top;
}

int orc_solve_ordered(int ny, int nx, double h, double eps, const double *L11,
                      const double *L21, const double *L22, const double *wx,
                      const double *wy, const uint8_t *src, double *T) {
  if (ny < 1 || nx < 1 || !(h > 0.0))
    return ORC_ERR_INVALID_ARG;
  int64_t n = (int64_t)ny * nx;
  for (int64_t p = 0; p < n; ++p)
    T[p] = src[p] ? 0.0 : INFINITY;
  if (!count_sources(n, src))
    return ORC_ERR_NO_SOURCE;
  uint8_t *acc = (uint8_t *)calloc((size_t)n, 1);
  /* each node is pushed at most 9 times (once as a source, once per
   * accepted neighbour) */
  heap_item *hp = (heap_item *)malloc(sizeof(heap_item) * (size_t)(9 * n + 1));
  if (!acc || !hp) {
    free(acc);
    free(hp);
    return ORC_ERR_INVALID_ARG;
  }
  int64_t sz = 0;
  for (int64_t p = 0; p < n; ++p)
    if (src[p])
      heap_push(hp, &sz, 0.0, p);
  while (sz > 0) {
    heap_item it = heap_pop(hp, &sz);
    if (acc[it.p] || it.v > T[it.p])
      continue;
    acc[it.p] = 1;
    int i = (int)(it.p / nx), j = (int)(it.p % nx);
    for (int k = 0; k < 8; ++k) {
      int ii = i + ORC_DY[k], jj = j + ORC_DX[k];
      if (ii < 0 || ii >= ny || jj < 0 || jj >= nx)
        continue;
      int64_t q = (int64_t)ii * nx + jj;
      if (acc[q] || src[q])
        continue;
      orc_cands c;
      node_candidates(ny, nx, h, eps, L11, L21, L22, wx, wy, T, acc, ii, jj,
                      &c);
      double best = cell_best(&c, NULL, NULL, NULL);
      if (best < T[q]) {
        T[q] = best;
        heap_push(hp, &sz, best, q);
      }
    }
  }
  free(acc);
  free(hp);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Residual of the discrete system: r_p = T_p - min valid candidate(T) at
 * every non-source node (0 at sources; 0 where both are +inf). */
int orc_residual(int ny, int nx, double h, double eps, const double *L11,
                 const double *L21, const double *L22, const double *wx,
                 const double *wy, const uint8_t *src, const double *T,
                 double *res) {
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      size_t p = (size_t)i * nx + j;
      if (src[p]) {
        res[p] = T[p];
        continue;
      }
      orc_cands c;
      node_candidates(ny, nx, h, eps, L11, L21, L22, wx, wy, T, NULL, i, j,
                      &c);
      double best = cell_best(&c, NULL, NULL, NULL);
      res[p] = (isinf(best) && isinf(T[p])) ? 0.0 : T[p] - best;
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/*
 * Stencil identification and closed-form partials (Alg. 2, first loop;
 * App. A "Explicit residuals and closed-form partial derivatives").
 *
 * For the active update of node p:
 *   two-point: R = u^T Q u - 1, u = S - T0 1;
 *     dR/dT0 = -2 1^T Q u, dR/dT_k = 2 e_k^T Q u   (Eq. 7)
 *     dR/db = 2 Mm Q u,    dR/dG = -Mm Q u u^T Q Mm^T
 *   one-point: R = r^2 - e, r = T_i + m.b - T0, e = m^T G m;
 *     dR/dT0 = -2 r, dR/dT_i = 2 r, dR/db = 2 r m, dR/dG = -m m^T.
 * With b = -w: dR/dw = -dR/db.  dR/dL = 2 (dR/dG) L on the lower triangle.
 *
 * Outputs per node:
 *   id     0 = source/unreached, 0x10|n = one-point via neighbour n,
 *          0x20|k = two-point stencil k;
 *   jac    [3] = dR/dT0, dR/dT_first donor, dR/dT_second donor
 *          (second = 0 for one-point);
 *   drt    [5] = dR/d(L11, L21, L22, wx, wy);
 *   margin = second-best valid candidate - best (+inf if none);
 * and *geo_only_count = number of two-point candidates at the converged T
 * with a real root and lambda >= 0 that causality rejected.
 * Arrays jac and drt are planar: jac[c*n + p], drt[c*n + p].
 */
int orc_record(int ny, int nx, double h, double eps, const double *L11,
               const double *L21, const double *L22, const double *wx,
               const double *wy, const uint8_t *src, const double *T,
               uint8_t *id, double *jac, double *drt, double *margin,
               int64_t *geo_only_count) {
  int64_t n = (int64_t)ny * nx, geo = 0;
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      int64_t p = (int64_t)i * nx + j;
      id[p] = 0;
      for (int c = 0; c < 3; ++c)
        jac[c * n + p] = 0.0;
      for (int c = 0; c < 5; ++c)
        drt[c * n + p] = 0.0;
      margin[p] = INFINITY;
      if (src[p] || !isfinite(T[p]))
        continue;
      orc_cands cs;
      node_candidates(ny, nx, h, eps, L11, L21, L22, wx, wy, T, NULL, i, j,
                      &cs);
      for (int k = 0; k < 8; ++k)
        geo += cs.two_geo_only[k];
      int kind, idx;
      double second;
      double best = cell_best(&cs, &kind, &idx, &second);
      if (kind == 0)
        continue;
      margin[p] = second - best;
      double dRdG11, dRdG12, dRdG22, dRdbx, dRdby;
      if (kind == 2) {
        int a = idx, b = (idx + 1) & 7;
        double m1x = h * ORC_DX[a], m1y = h * ORC_DY[a];
        double m2x = h * ORC_DX[b], m2y = h * ORC_DY[b];
        /* Q u = -lambda, with lambda = Q (T0 1 - S) from the update */
        double qu1 = -cs.lam[idx][0], qu2 = -cs.lam[idx][1];
        id[p] = (uint8_t)(0x20 | idx);
        jac[p] = -2.0 * (qu1 + qu2);
        jac[n + p] = 2.0 * qu1;
        jac[2 * n + p] = 2.0 * qu2;
        /* Mm Q u */
        double vx = m1x * qu1 + m2x * qu2, vy = m1y * qu1 + m2y * qu2;
        dRdbx = 2.0 * vx;
        dRdby = 2.0 * vy;
        dRdG11 = -vx * vx;
        dRdG12 = -vx * vy;
        dRdG22 = -vy * vy;
      } else {
        double mx = h * ORC_DX[idx], my = h * ORC_DY[idx];
        double Ti = T[(int64_t)(i + ORC_DY[idx]) * nx + (j + ORC_DX[idx])];
        double r = Ti - (mx * wx[p] + my * wy[p]) - best;
        id[p] = (uint8_t)(0x10 | idx);
        jac[p] = -2.0 * r;
        jac[n + p] = 2.0 * r;
        jac[2 * n + p] = 0.0;
        dRdbx = 2.0 * r * mx;
        dRdby = 2.0 * r * my;
        dRdG11 = -mx * mx;
        dRdG12 = -mx * my;
        dRdG22 = -my * my;
      }
      /* G = L L^T + eps I  =>  dR/dL = 2 (dR/dG) L  (lower triangle) */
      drt[p] = 2.0 * (dRdG11 * L11[p] + dRdG12 * L21[p]);
      drt[n + p] = 2.0 * (dRdG12 * L11[p] + dRdG22 * L21[p]);
      drt[2 * n + p] = 2.0 * dRdG22 * L22[p];
      drt[3 * n + p] = -dRdbx; /* b = -w */
      drt[4 * n + p] = -dRdby;
    }
  if (geo_only_count) *geo_only_count = geo;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
typedef struct {
  double t;
  int64_t p;
} order_item;

static int by_decreasing_t(const void *a, const void *b) {
  const order_item *x = (const order_item *)a, *y = (const order_item *)b;
  if (x->t > y->t) return -1;
  if (x->t < y->t) return 1;
  return (x->p < y->p) ? -1 : (x->p > y->p);
}

/*
 * Implicit-differentiation backward pass (Alg. 2; Eqs. 4-6).
 * Nodes sorted by decreasing T; back-substitution
 *   lambda_i = (g_i - sum_{j : i in donors(j)} J_ji lambda_j) / J_ii,
 * then dL/dtheta_i = -lambda_i dR_i/dtheta_i.
 * Sources carry the residual R = T - 0 (J_ii = 1, no parameters); unreached
 * nodes (T = +inf) have no residual: their lambda is 0 and g is ignored.
 *
 * Outputs: lam_norm[p] = J_pp * lambda_p, the multiplier of the residual
 * scaled to unit diagonal (R_p / J_pp = T_p - f_p(donors)), which is the
 * quantity the GPU path reports; grad = 5 planes dL/d(L11,L21,L22,wx,wy).
 */
int orc_adjoint(int ny, int nx, const uint8_t *src, const double *T,
                const uint8_t *id, const double *jac, const double *drt,
                const double *g, double *lam_norm, double *grad) {
  int64_t n = (int64_t)ny * nx;
  order_item *ord = (order_item *)malloc(sizeof(order_item) * (size_t)n);
  double *lam = (double *)calloc((size_t)n, sizeof(double));
  if (!ord || !lam) {
    free(ord);
    free(lam);
    return ORC_ERR_INVALID_ARG;
  }
  for (int64_t p = 0; p < n; ++p) {
    ord[p].t = T[p];
    ord[p].p = p;
  }
  qsort(ord, (size_t)n, sizeof(order_item), by_decreasing_t);
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = ord[k].p;
    if (!isfinite(T[p])) {
      lam[p] = 0.0;
      continue;
    }
    int i = (int)(p / nx), j = (int)(p % nx);
    double acc = g[p];
    /* children: neighbours q whose active update uses p as a donor */
    for (int nb = 0; nb < 8; ++nb) {
      int ii = i + ORC_DY[nb], jj = j + ORC_DX[nb];
      if (ii < 0 || ii >= ny || jj < 0 || jj >= nx)
        continue;
      int64_t q = (int64_t)ii * nx + jj;
      int back = (nb + 4) & 7; /* direction from q to p */
      uint8_t a = id[q];
      double Jqp = 0.0;
      if ((a & 0xF0) == 0x10 && (a & 7) == back)
        Jqp = jac[n + q];
      else if ((a & 0xF0) == 0x20 && (a & 7) == back)
        Jqp = jac[n + q];
      else if ((a & 0xF0) == 0x20 && (((a & 7) + 1) & 7) == back)
        Jqp = jac[2 * n + q];
      acc -= Jqp * lam[q];
    }
    if (src[p]) {
      lam[p] = acc; /* R = T - 0 at a source: unit diagonal */
    } else if (id[p] != 0 && jac[p] != 0.0) {
      lam[p] = acc / jac[p];
    } else {
      lam[p] = 0.0; /* no active update recorded: no residual */
    }
  }
  for (int64_t p = 0; p < n; ++p) {
    int reached = isfinite(T[p]) && !src[p] && id[p] != 0;
    double Jpp = src[p] ? 1.0 : (reached ? jac[p] : 0.0);
    lam_norm[p] = isfinite(T[p]) ? Jpp * lam[p] : 0.0;
    for (int c = 0; c < 5; ++c)
      grad[c * n + p] = reached ? -lam[p] * drt[c * n + p] : 0.0;
  }
  free(ord);
  free(lam);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/*
 * Soft-min relaxation of the stencil selection (Sec. 3.3, "Stencil
 * Boundaries and Non-Smoothness", names soft-min relaxations as an
 * alternative to the hard minimum without giving a formula).  Reading used
 * here: each of the node's 8 stencils k (donors k, k+1) has the value of
 * the minimum of its segment -- the two-point candidate when it is valid
 * (App. A), else the smaller one-point candidate of its finite endpoints --
 *     c_k = two_k if valid, else min(one_k, one_{k+1}),
 * and the node takes
 *     T0 = -tau log sum_k exp(-c_k / tau)
 * over the stencils with a value, evaluated as c_min - tau log sum_k
 * exp(-(c_k - c_min) / tau), with the softmax weights p_k = exp(-(c_k -
 * T0) / tau) (they sum to 1; computed as e_k / sum e).  A per-candidate sum would count a two-point
 * update that turns valid at lambda = 0 next to the one-point update it
 * equals there, so T0 would jump at every such switch; the segment minimum
 * moves continuously through it.  tau -> 0 gives the hard minimum (the
 * minimum over the stencil values equals the minimum over all valid
 * candidates); tau = 0 is the hard minimum exactly.
 * Per stencil: p[k], and src[k] = the candidate that gives c_k (8 + k: the
 * two-point of stencil k; n: the one-point through neighbour n; -1: none).
 * Returns T0 (+inf: no stencil has a value).
 */
static double stencil_value(const orc_cands *c, int k, int *from) {
  int a = k, b = (k + 1) & 7;
  if (c->two_ok[k]) {
    *from = 8 + k;
    return c->two[k];
  }
  double va = c->one_ok[a] ? c->one[a] : INFINITY;
  double vb = c->one_ok[b] ? c->one[b] : INFINITY;
  if (!isfinite(va) && !isfinite(vb)) {
    *from = -1;
    return INFINITY;
  }
  *from = (va <= vb) ? a : b;
  return va <= vb ? va : vb;
}

static double cell_softmin(const orc_cands *c, double tau, double p[8], int from[8]) {
  double v[8], cmin = INFINITY;
  for (int k = 0; k < 8; ++k) {
    v[k] = stencil_value(c, k, &from[k]);
    p[k] = 0.0;
    if (v[k] < cmin) cmin = v[k];
  }
  if (!isfinite(cmin))
    return INFINITY;
  if (!(tau > 0.0)) {
    for (int k = 0; k < 8; ++k)
      if (v[k] == cmin) {
        p[k] = 1.0;
        break;
      }
    return cmin;
  }
  /* e_k relative to the minimum (no overflow); p_k = e_k / s sums to 1
   * exactly, where exp(-(c_k - T0)/tau) would lose the digits of the
   * difference when tau is tiny */
  double e[8], s = 0.0;
  for (int k = 0; k < 8; ++k) {
    e[k] = isfinite(v[k]) ? exp(-(v[k] - cmin) / tau) : 0.0;
    s += e[k];
  }
  for (int k = 0; k < 8; ++k)
    p[k] = e[k] / s;
  return cmin - tau * log(s);
}

/* Exported: the soft-min of one node (for pin tests); p[8] = stencil
 * weights, from[8] = the candidate behind each stencil value (see
 * cell_softmin). */
double orc_cell_softmin(const double *Tn, double h, double g11, double g12,
                        double g22, double wx, double wy, double tau,
                        double *p, int *from) {
  orc_cands c;
  cell_candidates(Tn, h, g11, g12, g22, wx, wy, &c);
  return cell_softmin(&c, tau, p, from);
}

/*
 * Gauss-Seidel sweeps of the soft-min system (the sweep order of
 * orc_solve_gs): T = 0 on sources, +inf elsewhere, then every non-source
 * node is replaced by the soft-min of its candidates, until an iteration of
 * four sweeps changes no value by more than tol (absolute).  The soft
 * update is smooth, so the values converge geometrically rather than
 * stopping exactly.
 */
int orc_solve_softmin_gs(int ny, int nx, double h, double eps,
                         const double *L11, const double *L21,
                         const double *L22, const double *wx,
                         const double *wy, const uint8_t *src, double tau,
                         double tol, int max_iter, double *T,
                         int *iters_out) {
  if (ny < 1 || nx < 1 || !(h > 0.0) || tau < 0.0)
    return ORC_ERR_INVALID_ARG;
  int64_t n = (int64_t)ny * nx;
  for (int64_t p = 0; p < n; ++p)
    T[p] = src[p] ? 0.0 : INFINITY;
  if (!count_sources(n, src)) {
    if (iters_out) *iters_out = 0;
    return ORC_ERR_NO_SOURCE;
  }
  int it;
  for (it = 1; it <= max_iter; ++it) {
    double change = 0.0;
    for (int d = 0; d < 4; ++d) {
      int lines = (d % 2 == 0) ? nx : ny;
      int len = (d % 2 == 0) ? ny : nx;
      for (int s = 0; s < lines; ++s) {
        int line = (d < 2) ? s : lines - 1 - s;
        for (int q = 0; q < len; ++q) {
          int i = (d % 2 == 0) ? q : line;
          int j = (d % 2 == 0) ? line : q;
          size_t p = (size_t)i * nx + j;
          if (src[p])
            continue;
          orc_cands c;
          double pk[8];
          int from[8];
          node_candidates(ny, nx, h, eps, L11, L21, L22, wx, wy, T, NULL, i,
                          j, &c);
          double v = cell_softmin(&c, tau, pk, from);
          double dv = (isinf(v) && isinf(T[p])) ? 0.0 : fabs(v - T[p]);
          if (isinf(v) != isinf(T[p])) dv = INFINITY;
          if (dv > change) change = dv;
          T[p] = v;
        }
      }
    }
    if (change <= tol)
      break;
  }
  if (iters_out) *iters_out = it > max_iter ? max_iter : it;
  return it > max_iter ? ORC_ERR_NOT_CONVERGED : ORC_OK;
}

/*
 * Partials of one candidate of node (i, j) at T (the closed forms of
 * orc_record, normalised by dR/dT0): wa, wb = dc/dT of its donors (wb = 0
 * for one-point), dth[5] = dc/d(L11, L21, L22, wx, wy).
 */
static void candidate_partials(int kind, int idx, const orc_cands *cs,
                               double h, double L11, double L21, double L22,
                               double wx, double wy, double Ti, double c,
                               double *wa, double *wb, double dth[5]) {
  double jac0, jac1, jac2, dRdG11, dRdG12, dRdG22, dRdbx, dRdby;
  if (kind == 2) {
    int a = idx, b = (idx + 1) & 7;
    double m1x = h * ORC_DX[a], m1y = h * ORC_DY[a];
    double m2x = h * ORC_DX[b], m2y = h * ORC_DY[b];
    double qu1 = -cs->lam[idx][0], qu2 = -cs->lam[idx][1];
    jac0 = -2.0 * (qu1 + qu2);
    jac1 = 2.0 * qu1;
    jac2 = 2.0 * qu2;
    double vx = m1x * qu1 + m2x * qu2, vy = m1y * qu1 + m2y * qu2;
    dRdbx = 2.0 * vx;
    dRdby = 2.0 * vy;
    dRdG11 = -vx * vx;
    dRdG12 = -vx * vy;
    dRdG22 = -vy * vy;
  } else {
    double mx = h * ORC_DX[idx], my = h * ORC_DY[idx];
    double r = Ti - (mx * wx + my * wy) - c;
    jac0 = -2.0 * r;
    jac1 = 2.0 * r;
    jac2 = 0.0;
    dRdbx = 2.0 * r * mx;
    dRdby = 2.0 * r * my;
    dRdG11 = -mx * mx;
    dRdG12 = -mx * my;
    dRdG22 = -my * my;
  }
  double drt[5];
  drt[0] = 2.0 * (dRdG11 * L11 + dRdG12 * L21);
  drt[1] = 2.0 * (dRdG12 * L11 + dRdG22 * L21);
  drt[2] = 2.0 * dRdG22 * L22;
  drt[3] = -dRdbx;
  drt[4] = -dRdby;
  *wa = (jac0 != 0.0) ? -jac1 / jac0 : 0.0;
  *wb = (jac0 != 0.0) ? -jac2 / jac0 : 0.0;
  for (int k = 0; k < 5; ++k)
    dth[k] = (jac0 != 0.0) ? -drt[k] / jac0 : 0.0;
}

/*
 * Record of the soft-min system at T: for every non-source reached node,
 * wnb[nb * n + p] = dT_p / dT(neighbour nb) = sum_k p_k dc_k/dT_nb and
 * dth[c * n + p] = dT_p / dtheta_c = sum_k p_k dc_k/dtheta_c over its
 * candidates (the chain rule through the soft-min); zero elsewhere.
 */
int orc_softmin_record(int ny, int nx, double h, double eps,
                       const double *L11, const double *L21, const double *L22,
                       const double *wx, const double *wy, const uint8_t *src,
                       const double *T, double tau, double *wnb, double *dth) {
  int64_t n = (int64_t)ny * nx;
  for (int64_t p = 0; p < n; ++p) {
    for (int c = 0; c < 8; ++c) wnb[c * n + p] = 0.0;
    for (int c = 0; c < 5; ++c) dth[c * n + p] = 0.0;
  }
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      int64_t p = (int64_t)i * nx + j;
      if (src[p] || !isfinite(T[p]))
        continue;
      orc_cands cs;
      double Tn[8];
      node_candidates(ny, nx, h, eps, L11, L21, L22, wx, wy, T, NULL, i, j,
                      &cs);
      gather_neighbours(ny, nx, T, i, j, NULL, Tn);
      double pk[8];
      int from[8];
      cell_softmin(&cs, tau, pk, from);
      for (int k = 0; k < 8; ++k) {
        if (!(pk[k] > 0.0) || from[k] < 0)
          continue;
        double wa, wb, d5[5];
        if (from[k] >= 8) {
          candidate_partials(2, k, &cs, h, L11[p], L21[p], L22[p], wx[p], wy[p],
                             0.0, cs.two[k], &wa, &wb, d5);
          wnb[k * n + p] += pk[k] * wa;
          wnb[((k + 1) & 7) * n + p] += pk[k] * wb;
        } else {
          const int nb = from[k];
          candidate_partials(1, nb, &cs, h, L11[p], L21[p], L22[p], wx[p], wy[p],
                             Tn[nb], cs.one[nb], &wa, &wb, d5);
          wnb[nb * n + p] += pk[k] * wa;
        }
        for (int c = 0; c < 5; ++c) dth[c * n + p] += pk[k] * d5[c];
      }
    }
  return ORC_OK;
}

/*
 * Adjoint of the soft-min system (Alg. 2's back-substitution for the
 * relaxed residual R_p = T_p - softmin_p(T)): lambda_p = g_p + sum over
 * neighbours q of wnb_q(direction q -> p) lambda_q, dL/dtheta_p = lambda_p
 * dth_p.  A soft value can fall below one of its donors, so the weight graph
 * need not be ordered by T: the solve sweeps the nodes in decreasing T
 * (Gauss-Seidel), which is exact in one pass when it is, and repeats until
 * no multiplier changes by more than tol relative.  Returns the number of
 * passes in *passes_out.  Sources and unreached nodes: zero gradient.
 */
int orc_softmin_adjoint(int ny, int nx, const uint8_t *src, const double *T,
                        const double *wnb, const double *dth, const double *g,
                        double tol, int max_pass, double *lam, double *grad,
                        int *passes_out) {
  int64_t n = (int64_t)ny * nx;
  order_item *ord = (order_item *)malloc(sizeof(order_item) * (size_t)n);
  if (!ord)
    return ORC_ERR_INVALID_ARG;
  for (int64_t p = 0; p < n; ++p) {
    ord[p].t = T[p];
    ord[p].p = p;
    lam[p] = 0.0;
  }
  qsort(ord, (size_t)n, sizeof(order_item), by_decreasing_t);
  int pass;
  for (pass = 1; pass <= max_pass; ++pass) {
    double change = 0.0, scale = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      int64_t p = ord[k].p;
      if (!isfinite(T[p]))
        continue;
      int i = (int)(p / nx), j = (int)(p % nx);
      double acc = g[p];
      for (int nb = 0; nb < 8; ++nb) {
        int ii = i + ORC_DY[nb], jj = j + ORC_DX[nb];
        if (ii < 0 || ii >= ny || jj < 0 || jj >= nx)
          continue;
        int64_t q = (int64_t)ii * nx + jj;
        acc += wnb[((nb + 4) & 7) * n + q] * lam[q];
      }
      double d = fabs(acc - lam[p]);
      if (d > change) change = d;
      if (fabs(acc) > scale) scale = fabs(acc);
      lam[p] = acc;
    }
    if (change <= tol * (scale > 0.0 ? scale : 1.0))
      break;
  }
  if (passes_out) *passes_out = pass > max_pass ? max_pass : pass;
  for (int64_t p = 0; p < n; ++p)
    for (int c = 0; c < 5; ++c)
      grad[c * n + p] = (isfinite(T[p]) && !src[p]) ? lam[p] * dth[c * n + p] : 0.0;
  free(ord);
  return pass > max_pass ? ORC_ERR_NOT_CONVERGED : ORC_OK;
}
