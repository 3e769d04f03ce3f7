/*
 * rf.h -- C ABI of librf, the GB300 (sm_103a) implementation of the hot path
 * of "Differentiable Randers-Finsler Eikonal Solvers" (arXiv 2603.00035):
 * feasibility projection, fast-sweep forward solve with stencil record, and
 * the adjoint of the converged discrete system.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grids are row-major [ny][nx] float32; node (i,j) sits at (x,y) =
 *    (j h, i h).  Neighbour n of a node is at offset (dx,dy) with
 *    n = 0..7 -> (-1,+1) (-1,0) (-1,-1) (0,-1) (+1,-1) (+1,0) (+1,+1) (0,+1)
 *    (counter-clockwise from the upper-left, Fig. 4a); stencil k pairs
 *    neighbours k and (k+1) mod 8.
 *  - A "5-plane" array is 5 consecutive planes of ny*nx float32 values:
 *    L11, L21, L22, wx, wy (the metric factor and the drift).  The metric is
 *    M = L L^T + eps I, L lower-triangular; the Randers cost of a
 *    displacement v is F(v) = sqrt(v^T M v) + w^T v.  In the paper's
 *    notation (Eq. 1-3) this is G = M and b = -w.
 *  - Every pointer argument is DEVICE memory owned by the caller unless the
 *    comment says otherwise; the library never frees it.  All work is
 *    enqueued on `stream` (a cudaStream_t passed as void*; NULL = the legacy
 *    default stream) and is asynchronous unless stated.
 *  - Every call returns rf_status.  Host-detectable problems (null pointers,
 *    bad sizes) return immediately without enqueuing work.  Problems found on
 *    the device are written to the context's device status word and are
 *    returned by rf_ctx_last_stats() after the stream is synchronised.
 *  - One rf_ctx serves one stream at a time (its workspace is shared).
 */
#ifndef RF_H_
#define RF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rf_status {
  RF_OK = 0,
  RF_ERR_INVALID_ARG = 1,     /* null pointer, size < 1, h <= 0, ...        */
  RF_ERR_CUDA = 2,            /* a CUDA runtime call failed                 */
  RF_ERR_NOT_CONVERGED = 3,   /* max_sweeps reached; T/lambda still written */
  RF_ERR_TIMEOUT = 4,         /* a bounded device wait expired              */
  RF_ERR_NONFINITE_INPUT = 5, /* NaN/Inf in an input field                  */
  RF_ERR_NO_SOURCE = 6,       /* the source mask is empty                   */
  RF_ERR_NO_MEMORY = 7,       /* workspace allocation failed                */
  RF_ERR_UNSUPPORTED = 8      /* configuration not supported on this device */
} rf_status;

typedef struct rf_ctx rf_ctx;

typedef struct rf_grid {
  int32_t ny, nx; /* rows (y) and columns (x); each >= 1                   */
  float h;        /* grid spacing, > 0                                      */
} rf_grid;

enum rf_mode {
  RF_MODE_COLD = 0, /* T = 0 on sources, +inf elsewhere, then sweep          */
  RF_MODE_WARM = 1  /* start from the caller's T (sources forced to 0)       */
};

enum rf_adjoint_algo {
  RF_ADJ_SWEEP = 0,   /* transposed line sweeps until lambda stops changing */
  RF_ADJ_ORDERED = 1, /* radix sort on T, then dependency-ordered gather   */
  RF_ADJ_LEVELS = 2,  /* DAG-depth pass, radix sort on the level, then one
                         gather per level with a grid barrier between
                         levels; lambda equals RF_ADJ_ORDERED's bit for bit */
  RF_ADJ_TILES = 3    /* 16 x 16 tiles taken by decreasing latest T, the
                         chain inside a tile followed in shared memory;
                         lambda equals RF_ADJ_ORDERED's bit for bit        */
};

/* Forward-solve kernel variants.  The first three run the paper's schedule
 * (Sec. 3.2: column/row line fronts, sweeps in alternating directions) and
 * differ in how a line step gets its per-node constants; TILES runs another
 * schedule to the same fixed point.
 *  TILED1    node tables built per block in shared memory, one thread per
 *            node evaluates all 16 candidates;
 *  STREAMED  node records (24 floats) computed once per solve into a
 *            device buffer of 192 bytes per node owned by the context, and
 *            copied per line step by the bulk-copy engine; one thread per
 *            node, two-point candidates in the cone form (same values up to
 *            FP32 rounding);
 *  TILED4    as TILED1 with four threads per node and a shuffle minimum;
 *  TILES     tile queue: 16 x 16 (or 32 x 32) tiles iterated (Jacobi, one
 *            thread per node, four 16 x 16 tiles per 1024-thread CTA) to a
 *            local fixed point with their halo ring fixed; a tile whose boundary moved queues its
 *            neighbours for the next round, and each round processes the
 *            queued tiles within a window of the smallest arrival time
 *            (delta-stepping); deterministic (tiles read their neighbours'
 *            state as of the round's start).  Same fixed point as the line
 *            sweeps (every node at T = min valid candidate(T) to the change
 *            tolerance), a dependent chain of iterations along the front
 *            instead of sweeps x grid lines.
 * AUTO = TILES when its workspace can be allocated, else STREAMED when its
 * shape fits the device, else TILED1. */
enum rf_sweep_variant {
  RF_SWEEP_AUTO = 0,
  RF_SWEEP_TILED1 = 1,
  RF_SWEEP_STREAMED = 2,
  RF_SWEEP_TILED4 = 4,
  RF_SWEEP_TILES = 8
};

typedef struct rf_opts {
  float tol;          /* absolute part of the change test (see rtol)        */
  int32_t max_sweeps; /* cap on directional sweeps (4 per iteration)       */
  int32_t mode;       /* enum rf_mode                                       */
  int32_t band;       /* line sweeps: lines per band (0 = auto); TILES:
                         tile side, 16 or 32 (0 = 16)                     */
  int32_t block;      /* line steps per block, <= band (0 = auto)           */
  float rtol;         /* a node counts as changed in a sweep when
                         |T_new - T_old| > tol + rtol * T_new (either value
                         +inf: changed unless both are); the solve stops at
                         the first sweep with no changed node.  tol = rtol =
                         0 asks for bitwise no-change, which FP32 rounding
                         can turn into an ulp-level 2-cycle; the default
                         (opts NULL) is tol 0, rtol 1e-6 (about 8 ulp)     */
  int32_t variant;    /* enum rf_sweep_variant (0 = auto)                   */
  float window;       /* TILES: a round processes the queued tiles whose
                         key (smallest new boundary time that queued them)
                         is within window x (tile side) x (mean edge
                         cost) of the previous round's smallest key; the
                         rest wait for a later round (0 = auto: 4 with
                         16 x 16 tiles, 2 with 32 x 32)                    */
} rf_opts;

/* Per-node record of the converged forward solve (Alg. 2, first loop). */
typedef struct rf_record {
  uint8_t *id; /* [ny*nx] 0 = source/unreached; 0x10|n = one-point through
                  neighbour n; 0x20|k = two-point on stencil k            */
  float *w1;   /* [ny*nx] dT0/dT(first donor) (1 for one-point); the second
                  donor's weight is 1 - w1                                */
  float *dT;   /* [5*ny*nx] dT0/d(L11, L21, L22, wx, wy), 5 planes        */
} rf_record;

typedef struct rf_stats {
  int32_t status;       /* rf_status found on the device                  */
  int32_t sweeps;       /* directional sweeps run (forward; TILES: node
                           updates / nodes, rounded up)                   */
  int32_t converged;    /* 1 if the last sweep changed nothing            */
  int32_t adj_sweeps;   /* sweeps of the last adjoint (RF_ADJ_SWEEP), DAG
                           levels of the last RF_ADJ_LEVELS adjoint, tiles
                           that yielded in the last RF_ADJ_TILES adjoint */
  int64_t cell_updates; /* node updates of the last forward (line sweeps:
                           sweeps * ny * nx; TILES: nodes evaluated)      */
  float max_residual;   /* max |T - min valid candidate(T)| (record pass) */
  int32_t rounds;       /* rounds of the last TILES solve (0 otherwise)     */
} rf_stats;

/* ---- context ------------------------------------------------------------
 * rf_ctx_create: binds a context to CUDA device `device`, allocates a small
 * fixed workspace.  Larger buffers (the second sweep buffer, adjoint
 * buffers) are allocated on first use and grown on demand; a call that must
 * grow them allocates with cudaMalloc, so call once at full size before
 * capturing a CUDA graph.  rf_ctx_destroy frees everything the context owns
 * (not caller buffers). */
rf_status rf_ctx_create(rf_ctx **ctx, int device);
rf_status rf_ctx_destroy(rf_ctx *ctx);

/* Bound (nanoseconds, >= 0) on every device-side wait of the kernels this
 * context launches (neighbour progress flags, grid barriers).  When a wait
 * expires the kernel records RF_ERR_TIMEOUT, every CTA leaves its loops and
 * the launch ends; the context stays usable.  Default 2e9 (2 s). */
rf_status rf_ctx_set_timeout(rf_ctx *ctx, int64_t timeout_ns);

/* RF_ADJ_TILES: how long (ns, >= 0) a tile whose nodes wait for children
 * held by other tiles may see no progress before it yields its CTA and is
 * retried later (default 2000000).  A scheduling choice only: the results do
 * not depend on it; 0 yields at every stall. */
rf_status rf_ctx_set_adjoint_park(rf_ctx *ctx, int64_t park_ns);

/* Synchronise the stream of the context's last call and copy the device
 * statistics (including the device status word) into *out (host memory).
 * Returns out->status. */
rf_status rf_ctx_last_stats(rf_ctx *ctx, rf_stats *out);

/* Human-readable name of a status code (static string, never NULL). */
const char *rf_status_string(rf_status s);

/* ---- a1: feasibility projection -----------------------------------------
 * Paper: App. B "Feasibility Projections" (the G^-1-norm of b) and the
 * metric in factor form M = L L^T + eps I.  For each node:
 *   n = |w|_{M^-1} = sqrt((wx^2 M22 - 2 wx wy M12 + wy^2 M11) / det M),
 *   w_out = w * min(1, (1 - delta) / n);
 * L passes through.  raw5, proj5: 5-plane arrays (may alias only if equal);
 * clip: [ny*nx] uint8, 1 where the drift was rescaled (n > 1 - delta).
 * eps >= 0, 0 < delta < 1.  A NaN/Inf input sets RF_ERR_NONFINITE_INPUT in
 * the device status word. */
rf_status rf_project(rf_ctx *ctx, const rf_grid *grid, const float *raw5,
                     float eps, float delta, float *proj5, uint8_t *clip,
                     void *stream);

/* a9: backward of rf_project.  dproj5 = dL/d(L11, L21, L22, w_out x, w_out
 * y) (5 planes); draw5 = dL/d(raw inputs) (5 planes, may alias dproj5).  For
 * a clipped node, with P = M^-1, g = dL/dw_out, c = 1 - delta:
 *   dL/dw = (c/n)(g - P w (w^T g)/n^2),
 *   dL/dM += c (w^T g)/(2 n^3) (P w)(P w)^T,  dL/dL = 2 (dL/dM) L. */
rf_status rf_project_backward(rf_ctx *ctx, const rf_grid *grid,
                              const float *raw5, const uint8_t *clip,
                              float eps, float delta, const float *dproj5,
                              float *draw5, void *stream);

/* ---- the paper's own parameterisation (G, b) -----------------------------
 * Paper: App. B "Feasibility Projections" and "Total Variation
 * Regularization"; Eq. 8 (the regularised inverse problem).
 * gb5: 5 planes (g11, g12, g22, b1, b2) -- the symmetric metric G and the
 * drift b of the paper, [ny*nx] each, row-major.  The solver reads the
 * factor form proj5 = (L11, L21, L22, wx, wy) with M = L L^T + eps I = G and
 * w = -b (the drift-sign reading: the solver's cost is sqrt(v^T M v) + w.v).
 */
typedef struct rf_metric_params {
  float lam_min; /* eigenvalue floor, eps < lam_min <= lam_max */
  float lam_max; /* eigenvalue ceiling */
  float b_max;   /* Euclidean clip of the drift, > 0 (INFINITY: none) */
  float delta;   /* feasibility margin: |b|_{G^-1} <= 1 - delta, 0<delta<1 */
  float eps;     /* the solver's eps (M = L L^T + eps I), >= 0 */
} rf_metric_params;

/* Projection layer, per node in App. B's order:
 *   1. eigenvalues lambda_pm = ((g11+g22) +- sqrt((g11-g22)^2 + 4 g12^2))/2
 *      clamped to [lam_min, lam_max], G rebuilt on the principal axes
 *      (angle atan2(2 g12, g11 - g22)/2);
 *   2. |b|_2 clipped to b_max, then b scaled by (1-delta)/n when
 *      n = |b|_{G^-1} = sqrt((b1^2 g22 - 2 b1 b2 g12 + b2^2 g11)/det G)
 *      (projected G) exceeds 1 - delta;
 *   3. L = chol(G - eps I), w = -b.
 * gbp5 (nullable): projected (g11, g12, g22, b1, b2), may alias gb5 (the
 * in-place projection of projected gradient descent).  proj5 (nullable):
 * the solver's factor form.  Non-finite input sets RF_ERR_NONFINITE_INPUT in
 * the device status word. */
rf_status rf_metric_project(rf_ctx *ctx, const rf_grid *grid, const float *gb5,
                            const rf_metric_params *prm, float *gbp5,
                            float *proj5, void *stream);

/* Backward of rf_metric_project (recomputed from gb5, nothing stored):
 * dgb5 = dL/d(gb5) of a loss that reads proj5 (gradient dproj5, nullable)
 * and/or gbp5 (gradient dgbp5, nullable; e.g. a regulariser).  The clamp is
 * differentiated by the Daleckii-Krein formula (derivative 1 inside the
 * closed interval, 0 outside; divided difference across the two
 * eigenvalues); g12's gradient is with respect to the one parameter that
 * enters G twice.  dgb5 may alias dgbp5. */
rf_status rf_metric_project_backward(rf_ctx *ctx, const rf_grid *grid,
                                     const float *gb5,
                                     const rf_metric_params *prm,
                                     const float *dproj5, const float *dgbp5,
                                     float *dgb5, void *stream);

/* Total-variation regularisers of App. B with forward differences (zero in
 * the last column/row, no grid spacing):
 *   R(b) = sum_ij sqrt(sum_d (D_d b1)^2 + (D_d b2)^2),
 *   R(G) = sum_ij sqrt(sum_d (D_d a11)^2 + 2 (D_d a12)^2 + (D_d a22)^2)
 * with a = G (RF_TV_FROBENIUS) or a = log G (RF_TV_LOG_EUCLIDEAN, closed
 * form on the eigenvectors; G must be SPD, else RF_ERR_NONFINITE_INPUT in
 * the device status word).  value2 (device, nullable): [R(G), R(b)]
 * (unweighted; R(G) = 0 for RF_TV_NONE), deterministic order.  grad5
 * (device, nullable): += w_metric dR(G)/d(g11,g12,g22), w_drift
 * dR(b)/d(b1,b2); the subgradient is 0 where a node's norm is 0. */
enum rf_tv_metric { RF_TV_NONE = 0, RF_TV_FROBENIUS = 1, RF_TV_LOG_EUCLIDEAN = 2 };
rf_status rf_tv(rf_ctx *ctx, const rf_grid *grid, const float *gb5,
                int metric_mode, float w_metric, float w_drift, float *value2,
                float *grad5, void *stream);

/* ---- covariate encoder head (Sec. 5 "Encoder Architecture") -------------
 * The global pathway gives each grid a baseline (G0, b0), the
 * fully-convolutional pathway per-node residuals; they combine as
 * G = G0 + alpha G_local, b = b0 + alpha b_local.
 * local: FP32 NHWC [B][H][W][C] (channels 0..4 = residuals of g11, g12,
 * g22, b1, b2; C >= 5); base: FP32 [B][Cb] (channels 0..4 = G0, b0;
 * Cb >= 5); gb: FP32 out, per grid five planes of H*W nodes, grids back to
 * back (gb[(b*5 + c)*H*W + p]) -- each grid's gb5 for rf_metric_project. */
rf_status rf_encoder_combine(rf_ctx *ctx, const float *local, int B, int H,
                             int W, int C, const float *base, int Cb,
                             float alpha, float *gb, void *stream);
/* Adjoint: dlocal (BF16 NHWC [B][H][W][C]) = alpha dgb on channels 0..4,
 * 0 on the rest; dbase (BF16 [B][Cb]) = dgb summed over each grid's nodes
 * (fixed-order reduction) on channels 0..4, 0 on the rest. */
rf_status rf_encoder_combine_backward(rf_ctx *ctx, const float *dgb, int B,
                                      int H, int W, int C, int Cb, float alpha,
                                      uint16_t *dlocal, uint16_t *dbase,
                                      void *stream);

/* ---- a2-a5: forward solve -------------------------------------------------
 * Paper: Sec. 3.2 (Eqs. 2-3), App. A "Forward Solve Pseudocode" (Alg. 1).
 * proj5: projected 5-plane fields; src: [ny*nx] uint8 source mask (non-zero
 * = source, T = 0).  T: [ny*nx] output (and input guess when opts->mode ==
 * RF_MODE_WARM).  Each node takes the minimum over its valid one-point and
 * two-point candidates; sweeps run in the order columns +x, rows +y,
 * columns -x, rows -y, every line of a sweep updated as a parallel front,
 * until a sweep changes nothing (or opts->max_sweeps).  Convergence is
 * decided on the device.  Unreached nodes stay +inf.
 * rec (nullable): when given, the stencil id, donor weight and the partials
 * dT0/dtheta of every node's winning update at the converged T are written
 * (Alg. 2 "Identify active stencil"; App. A closed-form partials), plus the
 * max residual into the stats.  opts may be NULL (defaults: tol 0, rtol 1e-6,
 * max_sweeps 64, cold start, automatic variant and shape).  TILES caps its
 * rounds at max_sweeps x (tiles along the longer side). */
rf_status rf_sweep_forward(rf_ctx *ctx, const rf_grid *grid,
                           const float *proj5, float eps, const uint8_t *src,
                           const rf_opts *opts, float *T, rf_record *rec,
                           void *stream);

/* a5 alone: stencil identification and closed-form partials of a given
 * (converged) T -- the record rf_sweep_forward writes when rec != NULL.
 * Paper: Alg. 2 "Identify active stencil"; App. A closed-form partials.
 * Also stores max |T - min valid candidate(T)| in the context statistics. */
rf_status rf_record_stencils(rf_ctx *ctx, const rf_grid *grid,
                             const float *proj5, float eps, const uint8_t *src,
                             const float *T, rf_record *rec, void *stream);

/* Forward solve that allocates nothing (the paper has no counterpart: this
 * is a deployment variant of rf_sweep_forward without stencil record).
 * For callers that cannot allocate device memory at solve time -- a host
 * framework that has reserved the device's memory for its own allocator or
 * enforces a memory budget, or a latency-critical loop that must not pay
 * cudaMalloc's device-wide synchronisation.  It needs no rf_ctx: it runs on
 * the calling thread's current device, with its scratch (second sweep
 * buffer, progress and change flags, status word) in one fixed file-scope
 * device array of about 4 MiB that every GPU loading the library keeps
 * until the process exits.  It calls no cudaMalloc/cudaFree.
 * Limits: ny * nx <= 1048576 nodes and opts->max_sweeps <= 1024; larger
 * requests return RF_ERR_INVALID_ARG before any work is enqueued.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array, which keeps
 * the previous call's contents (the call clears what must start at zero):
 * calls whose work overlaps on the GPU race with each other, so serialise
 * them (one stream, or events).
 * Arguments as rf_sweep_forward (T: caller's device output, and warm-start
 * input when opts->mode == RF_MODE_WARM).  stats: HOST pointer, nullable;
 * when given the call synchronises `stream`, fills *stats and returns the
 * device status; when NULL the call is asynchronous and returns after
 * enqueuing (launch errors only).  Device-detected errors (not converged,
 * an expired wait, an empty source mask) live in the shared array's status
 * word, which the next call clears: they can only be seen by passing stats,
 * so a caller that must know whether T converged passes it.
 * The cached device address of the array is valid for the lifetime of the
 * CUDA context that looked it up: do not use this entry point again after
 * cudaDeviceReset on that device. */
rf_status rf_sweep_forward_static(const rf_grid *grid, const float *proj5,
                                  float eps, const uint8_t *src,
                                  const rf_opts *opts, float *T,
                                  rf_stats *stats, void *stream);

/* B7: residual r = T - min valid candidate(T) at every non-source node.
 * res (nullable): [ny*nx] per-node residual; max_abs (device float*,
 * nullable): max |r| over nodes with finite T. */
rf_status rf_residual(rf_ctx *ctx, const rf_grid *grid, const float *proj5,
                      float eps, const uint8_t *src, const float *T,
                      float *res, float *max_abs, void *stream);

/* ---- a6-a8: adjoint ---------------------------------------------------------
 * Paper: Sec. 3.3 (Eqs. 4-6), App. A Alg. 2 and the closed-form partials.
 * Solves lambda_p = g_p + sum over children q (neighbours whose recorded
 * update uses p as a donor) of dT_q/dT_p lambda_q -- the unit-diagonal form
 * of J^T lambda = g -- then writes dL/dtheta_p = lambda_p dT0_p/dtheta_p
 * into dLdproj5 (5 planes, zero at sources and unreached nodes).
 * T, rec: from rf_sweep_forward; dLdT: [ny*nx] (ignored where T = +inf);
 * lambda (nullable): [ny*nx] output.  algo: enum rf_adjoint_algo.
 * RF_ADJ_ORDERED, RF_ADJ_LEVELS and RF_ADJ_TILES wait (bounded by the
 * context's timeout) for donors or children named by the record; a record whose donors do not
 * have strictly smaller T ends in RF_ERR_TIMEOUT in the stats, with the
 * outputs incomplete.  Scratch: the context's buffers, grown as needed. */
rf_status rf_adjoint(rf_ctx *ctx, const rf_grid *grid, const uint8_t *src,
                     const float *T, const rf_record *rec, const float *dLdT,
                     float *dLdproj5, float *lambda, int algo, void *stream);

/* ---- whole steps on host buffers --------------------------------------------
 * Sec. 3 end to end for the inverse problem (a1 projection, a2-a4 forward
 * solve, a5 record, a6-a8 adjoint, a9 projection backward), input and
 * output in host memory.  For each step i < n_steps: raw5_h[i] (5 planes
 * [ny*nx] FP32: L11, L21, L22, wx, wy before projection), src_h[i]
 * ([ny*nx] uint8) and dLdT_h[i] ([ny*nx] FP32) are copied to the device;
 * the step projects (eps, delta), solves (opts, NULL for defaults),
 * records, solves the adjoint (algo: enum rf_adjoint_algo) and projects
 * back; T_h[i] ([ny*nx]) and dLdraw_h[i] ([5*ny*nx], dL/draw5) receive the
 * results.  Steps are pipelined: step i + 1's input copy and step i - 1's
 * output copy run on the context's two copy streams while step i computes
 * on `stream` (two device buffer sets, allocated on first use and kept by
 * the context).  Host buffers should be page-locked for the copies to
 * overlap.  Returns when every result has arrived; device errors of the
 * solves are in the context statistics (rf_ctx_last_stats). */
rf_status rf_step_host(rf_ctx *ctx, const rf_grid *grid, int n_steps,
                       const float *const *raw5_h,
                       const uint8_t *const *src_h,
                       const float *const *dLdT_h, float eps, float delta,
                       const rf_opts *opts, int algo, float *const *T_h,
                       float *const *dLdraw_h, void *stream);

/* ---- soft-min relaxation of the stencil selection --------------------------
 * Paper: Sec. 3.3 "Stencil Boundaries and Non-Smoothness" names soft-min
 * relaxations as an alternative to the hard minimum, without a formula.
 * Reading implemented: each of a node's 8 stencils k (donors k, k+1) has
 * the value c_k of its segment minimum -- the two-point candidate when valid
 * (App. A), else the smaller one-point candidate of its finite endpoints --
 * and the node takes T = -tau log sum_k exp(-c_k / tau) (tau > 0; tau = 0 is
 * the hard minimum).  T is continuous where a two-point update turns valid,
 * smooth elsewhere except where validity (causality) switches.  A soft value
 * lies up to tau log 8 below its candidate minimum: tau must stay well below
 * the cheapest edge cost (|m|_M - w.m over the grid's steps), else the
 * values run to -inf -- reported as RF_ERR_NOT_CONVERGED as soon as a
 * non-source node goes negative.
 *
 * rf_softmin_forward: the relaxed system solved from T = 0 on sources,
 * +inf elsewhere (warm mode: the caller's T) until no node would change by
 * more than tol + rtol |T| (opts as rf_sweep_forward).  opts->variant AUTO
 * or TILES: the tile queue of RF_SWEEP_TILES with the soft-min update (the
 * sweeps statistic is node updates / nodes); a line-sweep variant: Jacobi
 * iterations over all nodes in one persistent launch (at most max_sweeps x
 * max(ny, nx) iterations, reported as the sweeps statistic).  Arguments as
 * rf_sweep_forward without the record. */
rf_status rf_softmin_forward(rf_ctx *ctx, const rf_grid *grid, const float *proj5, float eps,
                             const uint8_t *src, float tau, const rf_opts *opts, float *T, void *stream);
/* Record of the relaxed system at T: wnb (8 planes, [8][ny*nx]) =
 * dT_p / dT(neighbour n of p), dT (5 planes) = dT_p / d(L11, L21, L22, wx,
 * wy); both zero at sources and unreached nodes.  The weights of a node sum
 * to 1. */
rf_status rf_softmin_record(rf_ctx *ctx, const rf_grid *grid, const float *proj5, float eps,
                            const uint8_t *src, const float *T, float tau, float *wnb, float *dT, void *stream);
/* Adjoint of the relaxed system: lambda_p = g_p + sum over neighbours q of
 * wnb_q(q -> p) lambda_q, iterated (block Jacobi: 16 x 16 tiles, 16 Jacobi
 * steps per tile between grid-wide exchanges) until no multiplier changes by
 * more than 1e-7 relative between two exchanges (their count is the
 * adj_sweeps statistic), dLdproj5 = lambda dT (5 planes, zero at sources
 * and unreached nodes); lambda (nullable). */
rf_status rf_softmin_adjoint(rf_ctx *ctx, const rf_grid *grid, const uint8_t *src, const float *T,
                             const float *wnb, const float *dT, const float *dLdT, float *dLdproj5,
                             float *lambda, void *stream);

/* ---- a10: batched solve ---------------------------------------------------
 * Many grids of uneven size and source count, forward + record (+ adjoint
 * and parameter gradients when dLdT != NULL) in one call.
 * Paper: batched solves across problem instances (Sec. 3.4 "Computational
 * Efficiency"); each grid is the discrete system of rf_sweep_forward and
 * rf_adjoint.
 * Packed layout: every per-node array holds all grids back to back; grid g
 * occupies nodes [descs[g].offset, descs[g].offset + ny*nx) of each plane
 * (row-major inside the grid), and 5-plane arrays have plane stride
 * total_nodes; the offsets increase in descriptor order and the grids do
 * not overlap (checked on the device: RF_ERR_INVALID_ARG in the status
 * word).  descs: DEVICE array of n_grids descriptors; put the largest grid
 * first.  max_line >= every grid's max(ny, nx).  T, rec: outputs (rec
 * required; the adjoint reads it).  dLdT (nullable) and dLdproj5: packed
 * like T and proj5; rec and dLdproj5 are not written between grids.
 * grid_status (DEVICE, nullable): 3 int32 per grid = status, forward sweeps
 * (TILES: node updates / nodes, rounded up), adjoint sweeps (0 for the
 * tiled adjoint).
 * opts->variant AUTO or TILES: every grid's tiles share one tile queue (see
 * RF_SWEEP_TILES; band = tile side), then one record pass and the tiled
 * adjoint over the packed grids (RF_ADJ_TILES, tiles handed out eight
 * grids at a time) -- a few launches on `stream`.  Line-sweep
 * variants: one persistent launch, CTAs taking whole grids in array order,
 * the transposed-sweep adjoint; max_line <= 1024 (shared-memory lines).
 * Both allocate only on first use (workspace grown to the call's size);
 * after one call of the same sizes the call is safe to capture in a CUDA
 * graph.  Device errors also go to the context's status word. */
typedef struct rf_batch_desc {
  int32_t ny, nx; /* grid shape */
  float h;        /* spacing */
  int32_t pad;
  int64_t offset; /* first node of the grid in the packed arrays */
} rf_batch_desc;

rf_status rf_batch_solve(rf_ctx *ctx, const rf_batch_desc *descs, int n_grids,
                         int64_t total_nodes, int32_t max_line,
                         const float *proj5, float eps, const uint8_t *src,
                         const rf_opts *opts, float *T, rf_record *rec,
                         const float *dLdT, float *dLdproj5,
                         int32_t *grid_status, void *stream);

/* ---- a11, a12: kernels of the learned warm start ---------------------------
 * The paper has no network; these serve the build's learned initial guess
 * (a small U-Net, BF16 weights/activations, FP32 accumulation) that enters
 * rf_sweep_forward through RF_MODE_WARM.  Tensors are NHWC, BF16 values
 * passed as uint16_t (IEEE bfloat16 bit patterns); every channel count given
 * to a convolution is a multiple of 16.  All pointers are device memory
 * owned by the caller; calls only enqueue work on `stream`.
 *
 * rf_unet_conv3x3: y = act(conv3x3_same(x, w) + bias), w [Cout][3][3][Cin],
 *   bias [Cout] FP32 (nullable), relu 0/1, y [B][H][W][Cout] BF16, y32
 *   (nullable) the same values in FP32.  Implicit GEMM on the tensor cores.
 *   With w replaced by rf_unet_flip_weights(w) it computes the data
 *   gradient dx from dy. */
rf_status rf_unet_conv3x3(rf_ctx *ctx, const uint16_t *x, int B, int H, int W,
                          int Cin, const uint16_t *w, const float *bias,
                          int Cout, int relu, uint16_t *y, float *y32,
                          void *stream);
/* The same convolution on the fifth-generation tensor cores (tcgen05.mma,
 * BF16 operands in shared memory, FP32 accumulator in tensor memory): same
 * arguments, same result up to FP32 summation order.  With 64 or more input
 * channels and Cout a multiple of 64 it first copies w, in the order the
 * kernel's pipeline stages hold it, into the context's workspace (grown on
 * first use to Cout * 9 * Cin BF16 values; RF_ERR_NO_MEMORY if that fails),
 * so two such calls on one context must not run on different streams at
 * once.  A tensor-core wait that exceeds the context timeout sets
 * RF_ERR_TIMEOUT in the context statistics. */
rf_status rf_unet_conv3x3_tc(rf_ctx *ctx, const uint16_t *x, int B, int H,
                             int W, int Cin, const uint16_t *w,
                             const float *bias, int Cout, int relu,
                             uint16_t *y, float *y32, void *stream);
/* dw [Cout][3][3][Cin] (FP32) += sum over pixels of dy (x) im2col(x): the
 * weight gradient; the caller zeroes dw. */
rf_status rf_unet_conv3x3_wgrad(rf_ctx *ctx, const uint16_t *x,
                                const uint16_t *dy, int B, int H, int W,
                                int Cin, int Cout, float *dw, void *stream);
/* The same weight gradient on the fifth-generation tensor cores: per tap a
 * GEMM (M = output channels, N = input channels, K = pixels) with both BF16
 * operands staged in shared memory as they lie in memory (MN-major) and
 * the 9 FP32 accumulators in tensor memory; partial sums over pixel-row
 * ranges are added to dw (the caller zeroes it).  Cin, Cout multiples of
 * 16; x, dy 16-byte aligned (else RF_ERR_INVALID_ARG).  A tensor-core wait
 * beyond the context timeout sets RF_ERR_TIMEOUT in the statistics. */
rf_status rf_unet_conv3x3_wgrad_tc(rf_ctx *ctx, const uint16_t *x,
                                   const uint16_t *dy, int B, int H, int W,
                                   int Cin, int Cout, float *dw,
                                   void *stream);
/* db [C] (FP32) += sum over npix pixels of dy [npix][C]. */
rf_status rf_unet_bias_grad(rf_ctx *ctx, const uint16_t *dy, int64_t npix,
                            int C, float *db, void *stream);
/* wt [Cin][3][3][Cout] = w [Cout][3][3][Cin] flipped in both spatial axes:
 * the weights of the data-gradient convolution. */
rf_status rf_unet_flip_weights(rf_ctx *ctx, const uint16_t *w, int Cin,
                               int Cout, uint16_t *wt, void *stream);
/* 2x2 max pooling (H, W even): y [B][H/2][W/2][C], arg = argmax 0..3 per
 * output; the backward scatters dy to the argmax positions (dx fully
 * written). */
rf_status rf_unet_maxpool2(rf_ctx *ctx, const uint16_t *x, int B, int H,
                           int W, int C, uint16_t *y, uint8_t *arg,
                           void *stream);
rf_status rf_unet_maxpool2_backward(rf_ctx *ctx, const uint16_t *dy,
                                    const uint8_t *arg, int B, int H, int W,
                                    int C, uint16_t *dx, void *stream);
/* Nearest 2x upsampling of x [B][H][W][C] to y [B][2H][2W][C]; the
 * backward sums the four children into dx [B][H][W][C]. */
rf_status rf_unet_upsample2(rf_ctx *ctx, const uint16_t *x, int B, int H,
                            int W, int C, uint16_t *y, void *stream);
rf_status rf_unet_upsample2_backward(rf_ctx *ctx, const uint16_t *dy, int B,
                                     int H, int W, int C, uint16_t *dx,
                                     void *stream);
/* split == 0: y [npix][Ca+Cb] = concat(a [npix][Ca], b [npix][Cb]) along
 * channels; split == 1: the reverse copy (the backward). */
rf_status rf_unet_concat(rf_ctx *ctx, uint16_t *a, int Ca, uint16_t *b,
                         int Cb, int64_t npix, uint16_t *y, int split,
                         void *stream);
/* dy[i] = 0 where y[i] <= 0 (backward of a ReLU whose output is y). */
rf_status rf_unet_relu_backward(rf_ctx *ctx, uint16_t *dy, const uint16_t *y,
                                int64_t n, void *stream);
/* Masked mean-squared error on channel 0 of pred32 [npix][C]:
 * loss += sum m (p - t)^2 / count; dpred [npix][C] = 2 m (p - t) / count on
 * channel 0 and 0 elsewhere.  mask nullable (all ones). */
rf_status rf_unet_mse(rf_ctx *ctx, const float *pred32, int C,
                      const float *target, const float *mask, int64_t npix,
                      float count, uint16_t *dpred, float *loss,
                      void *stream);
/* y = bf16(x), round to nearest even. */
rf_status rf_unet_cast_bf16(rf_ctx *ctx, const float *x, uint16_t *y,
                            int64_t n, void *stream);
/* planes [B][Cp][H][W] FP32 -> y [B][H][W][C] BF16, channels >= Cp zero. */
rf_status rf_unet_pack_input(rf_ctx *ctx, const float *planes, int Cp, int B,
                             int H, int W, int C, uint16_t *y, void *stream);

/* y += x, n BF16 values (FP32 arithmetic): joins skip gradients. */
rf_status rf_unet_add(rf_ctx *ctx, uint16_t *y, const uint16_t *x, int64_t n,
                      void *stream);
/* Network input features: for every pixel of image b, the distance to the
 * nearest source and the displacement (x, y) to it, in domain units (h per
 * pixel); out [B][3][H][W] FP32.  src_ij [nsrc][2] (row, column) device
 * int32, grouped by image: image b owns entries src_off[b] ..
 * src_off[b+1] - 1 (src_off [B+1]). */
rf_status rf_unet_source_features(rf_ctx *ctx, int B, int H, int W, float h,
                                  const int32_t *src_ij,
                                  const int32_t *src_off, float *out,
                                  void *stream);
/* Box average of FP32 planes x [P][H][W] by an integer factor f (H, W
 * divisible by f) into y [P][H/f][W/f]. */
rf_status rf_unet_box_down(rf_ctx *ctx, const float *x, int P, int H, int W,
                           int f, float *y, void *stream);
/* Node-aligned bilinear resampling of FP32 planes x [P][Hi][Wi] into
 * y [P][Ho][Wo] (corners map to corners), multiplied by scale. */
rf_status rf_unet_bilinear(rf_ctx *ctx, const float *x, int P, int Hi,
                           int Wi, int Ho, int Wo, float scale, float *y,
                           void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RF_H_ */
