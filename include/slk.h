/*
 * slk.h -- C-ABI of the GB300 (sm_103a) hot path of Scalable Laplacian
 * K-modes, SLK-BO variant (Ziko, Granger, Ben Ayed, "Scalable Laplacian
 * K-modes", NeurIPS 2018, arXiv:1810.13044).
 *
 * Problem statement (Eq. 1): N points x_p in R^D, L clusters, affinities
 * k(x_p, x_q), modes m_l that are data points, one-hot assignments z_p.
 * Algorithm 1 alternates (i) z-updates -- the soft-max of Eq. (soft-max),
 * z_p <- exp(a_p + lambda b_p) / 1^t exp(a_p + lambda b_p), with the unary
 * term a_{p,l} = k(x_p, m_l) (Eq. general-second) and the pairwise term
 * b_{p,l} = sum_q k(x_p, x_q) z_{q,l} (Eq. general-third) -- and (ii) mode
 * updates m_l = x_p, p = argmax_q z_{q,l} (Eq. mode_byproduct).
 *
 * Conventions shared by every entry point
 *   - Array arguments are DEVICE pointers (cudaMalloc / torch CUDA tensors)
 *     owned by the caller, unless marked [host].  Dense matrices are
 *     row-major and C-contiguous: X is N x D float32, A and Z are N x L
 *     float32.  The graph is CSR: row_ptr[N+1] int64, col_idx[nnz] int32,
 *     w[nnz] float32 or NULL for binary (all-one) weights.
 *   - All work is enqueued on the context's stream.  Entry points with
 *     [host] outputs synchronise that stream before returning; the others
 *     return as soon as the work is enqueued.
 *   - The library owns only the context and its scratch workspace, which it
 *     grows with cudaMalloc on demand and frees in slk_destroy.
 *   - Errors: arguments are checked before anything is launched; a bad one
 *     returns SLK_ERR_INVALID_ARG and writes nothing.  CUDA failures return
 *     SLK_ERR_CUDA, failed allocations SLK_ERR_OOM; slk_last_error() then
 *     holds a one-line message.  There is no CPU fallback: without a usable
 *     GPU every compute call fails.
 *   - Sizes: 2 <= N < 2^31, 1 <= D, 1 <= L <= 256, L <= N, 1 <= k <= 24,
 *     k <= N - 1.  Inputs must be finite.
 */
#ifndef SLK_H
#define SLK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slk_ctx slk_ctx;

typedef enum {
    SLK_OK = 0,
    SLK_NOT_CONVERGED = 1,      /* warning: max_outer reached, results valid */
    SLK_ERR_INVALID_ARG = -1,
    SLK_ERR_CUDA = -2,
    SLK_ERR_OOM = -3,
    SLK_ERR_TIMEOUT = -4,       /* a device-side wait gave up; results invalid */
    SLK_ERR_NO_DEVICE = -5,
    SLK_ERR_SCRATCH_LIMIT = -6  /* problem larger than a fixed scratch area (see below) */
} slk_status;

enum { SLK_AFFINITY_BINARY = 0, SLK_AFFINITY_HEAT = 1 };
enum { SLK_KNN_FP32 = 0, SLK_KNN_BF16_RERANK = 1 };
enum { SLK_SIGMA_MEDIAN = 0, SLK_SIGMA_MEANSQ = 1 };

/* Limits checked by every entry point. */
#define SLK_MAX_L 256
#define SLK_MAX_K 24

/* Library version string, e.g. "slk-gb300 0.1 sm_103a". */
const char* slk_version(void);

/* Create a context bound to CUDA device `device` and stream `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle.  Fails with SLK_ERR_NO_DEVICE when no such device is usable. */
slk_status slk_create(slk_ctx** ctx, int device, void* stream);
slk_status slk_destroy(slk_ctx* ctx);
slk_status slk_set_stream(slk_ctx* ctx, void* stream);
/* Message of the last failed call on this context ("" if none). */
const char* slk_last_error(const slk_ctx* ctx);

/* kNN affinity graph of Section 4.2: for each point p, the k nearest points
 * q != p by Euclidean distance, ascending by (distance, index).
 *   X        [N x D]   features.
 *   row_ptr  [N+1]     out: row_ptr[p] = k p.
 *   col_idx  [N k]     out: neighbour indices.
 *   dist2    [N k]     out: squared distances, each the float32 sum of
 *                      (x_pj - x_qj)^2.
 *   w        [N k]     out (may be NULL for BINARY): weights; BINARY writes
 *                      1, HEAT writes exp(-dist2 / (2 sigma^2)).
 *   affinity SLK_AFFINITY_*; sigma (> 0) is used by HEAT only.
 *   precision SLK_KNN_FP32: float32 SIMT distance tiles; SLK_KNN_BF16_RERANK:
 *            bfloat16 tensor-core (tcgen05) distance tiles.  Both produce
 *            candidates that are re-ranked with exact float32 distances and
 *            certified by a rounding-error bound.  With BF16_RERANK the rows
 *            that fail it get two-term bfloat16 tensor-core tiles (each
 *            feature as h + l, h = bf16(v), l = bf16(v - h)) under their own
 *            certificate next, then float32 candidate tiles under the float32
 *            certificate (the two-term stage from 100000 points on, for at
 *            most 65536 rows; the rest go straight to the float32 one); rows
 *            still uncertified are recomputed by an exact float32 scan, so
 *            both precisions return the same graph.
 *   fallback_rows [host, nullable]: receives how many rows the first
 *            certificate left open (for BF16_RERANK: the rows sent to the
 *            float32 stage).
 * Brute force, O(N^2 D) -- the paper's exact option for small sets. */
slk_status slk_knn_graph(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t k,
                         int32_t affinity, int32_t precision, float sigma,
                         int64_t* row_ptr, int32_t* col_idx, float* dist2, float* w,
                         int64_t* fallback_rows);

/* Rows per stage of the last kNN graph built on ctx (by slk_knn_graph,
 * slk_solve, slk_solve_host, slk_solve_ms): rows[0] the rows the first
 * certificate left open, rows[1] (BF16_RERANK) the rows sent to the float32
 * stage (left open by the two-term stage, or below 100000 points, where that
 * stage is skipped, by the first certificate), rows[2] the rows rescanned
 * exactly.
 *   rows [3] host out.
 * Synchronises ctx's stream.  SLK_ERR_INVALID_ARG if rows is NULL. */
slk_status slk_knn_stage_rows(slk_ctx* ctx, int64_t* rows);

/* Kernel width of Section 4.2 from the n = N k squared kNN distances dist2.
 *   rule SLK_SIGMA_MEDIAN: sigma = median of sqrt(dist2) (mean of the two
 *        middle values when n is even); SLK_SIGMA_MEANSQ: the paper's
 *        estimator sigma^2 = (1/n) sum dist2.
 *   sigma_out [host] receives sigma. */
slk_status slk_sigma(slk_ctx* ctx, const float* dist2, int64_t n, int32_t rule, float* sigma_out);

/* Unary term, Eq. (general-second), with the Gaussian kernel of Section 4.2:
 * A[p,l] = exp(-||x_p - x_{mode_idx[l]}||^2 / (2 sigma^2)).
 *   mode_idx [L] int32 point indices in [0, N).
 *   Z0 [N x L] (nullable): receives softmax(A) row by row, the
 *   initialisation of the inner loop of Algorithm 1. */
slk_status slk_unary(slk_ctx* ctx, const float* X, int64_t N, int32_t D,
                     const int32_t* mode_idx, int32_t L, float sigma, float* A, float* Z0);

/* Inner loop of Algorithm 1: the soft-max z-update of Eq. (soft-max),
 * z_p <- softmax(a_p + lambda b_p), b_p = sum_{e in row p} w_e z_{col_idx[e]},
 * applied to all rows from the same iterate, repeated until
 * max_{p,l} |z_new - z_old| <= tol or max_iters updates (tol < 0: exactly
 * max_iters).
 *   Z      [N x L] in: starting iterate; out: the last iterate.
 *   Z_prev [N x L] out: the iterate the last update started from (the mode
 *          update needs it); its input contents are ignored.  Must not alias Z.
 *   iters_done [host, nullable], last_delta [host, nullable].
 * Runs as one persistent cooperative kernel with a device-wide barrier
 * between updates; a barrier wait longer than 2 s gives up and the call
 * returns SLK_ERR_TIMEOUT, with Z and Z_prev undefined (they may hold a
 * partly written update). */
slk_status slk_bound_iterate(slk_ctx* ctx, const float* A, const int64_t* row_ptr,
                             const int32_t* col_idx, const float* w, int64_t N, int32_t L,
                             float lambda, float* Z, float* Z_prev, int32_t max_iters, float tol,
                             int32_t* iters_done, float* last_delta);

/* Self-test of the failure path of the z-update kernels (no counterpart in
 * the paper).  One block waits at the same bounded device-wide barrier for a
 * second block that is never launched, so the wait must give up after
 * timeout_ms (1 .. 2000) milliseconds.  Returns SLK_ERR_TIMEOUT -- the status
 * slk_bound_iterate reports when its barrier gives up -- and leaves the
 * context usable; any other status means the failure path is broken.
 * Synchronises the context stream. */
slk_status slk_barrier_selftest(slk_ctx* ctx, int32_t timeout_ms);

/* SLK-BO mode update, Eq. (mode_byproduct): mode_idx[l] <- argmax_q z_{q,l}
 * (ties to the smaller q), where z_q = softmax(s_q) is the last iterate and
 * s_q = a_q + lambda b_q its logits, recomputed from Z_prev (NULL: s = A, the
 * initial iterate).  The comparison uses log z_{q,l} =
 * (s_l - max s) - log1p(sum_{j != argmax} exp(s_j - max s)), which does not
 * saturate when z is close to 1.
 *   mode_idx [L] in: previous modes; out: new modes.
 *   labels   [N] (nullable) out: argmax_l z_{q,l} (ties to the smaller l).
 *   mode_key [L] (nullable) out: log z at the new modes.
 *   changed  [host, nullable]: 1 if any mode index changed, else 0. */
slk_status slk_mode_update(slk_ctx* ctx, const float* A, const float* Z_prev,
                           const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                           int64_t N, int32_t L, float lambda, int32_t* mode_idx,
                           int32_t* labels, float* mode_key, int32_t* changed);

/* Discrete energy, Eq. (1), at the one-hot assignment given by labels and
 * the modes m_l = x_{mode_idx[l]}:
 *   E = -sum_p k(x_p, m_{labels[p]}) + (lambda/2) sum_p sum_{e in row p} w_e ||z_p - z_q||^2,
 * with ||z_p - z_q||^2 = 2 [labels[p] != labels[q]].  Distances, kernel values
 * and sums are computed in float64.  E [host] receives the value. */
slk_status slk_energy(slk_ctx* ctx, const float* X, int32_t D, const int32_t* labels,
                      const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                      int64_t N, int32_t L, const int32_t* mode_idx, float sigma, float lambda,
                      double* E);

typedef struct {
    int32_t max_outer;      /* outer iterations of Algorithm 1 (default 50) */
    int32_t max_inner;      /* z-updates per outer iteration (default 100), >= 1 */
    float tol_inner;        /* stop the inner loop when max |dz| <= tol (default 1e-6) */
    int32_t sigma_rule;     /* SLK_SIGMA_* used when sigma <= 0 (default MEDIAN) */
    int32_t affinity;       /* SLK_AFFINITY_* (default BINARY) */
    int32_t knn_precision;  /* SLK_KNN_* (default FP32) */
    int32_t refine_init;    /* slk_solve, slk_solve_host, slk_solve_ms: 1 = start from
                               slk_initial_modes(init_modes) instead of init_modes (default 0) */
    int32_t reorder;        /* slk_solve, slk_solve_host: iterate on rows sorted by their nearest
                               initial mode, for cache locality of the z-updates (results are
                               identical): -1 = when Z exceeds 64 MB (default), 0 = never, 1 = always */
    /* SLK-MS only (slk_solve_ms): */
    int32_t max_ms;         /* mean-shift iterations per outer iteration (default 100) */
    float tol_ms;           /* stop them when max_l ||m_l move||_2 <= tol_ms * sigma (default 1e-5) */
    float tol_modes;        /* stop the outer loop when the modes moved <= tol_modes * sigma (default 1e-3) */
    /* slk_solve, slk_solve_host, slk_solve_ms: */
    int32_t symmetrize;     /* 1 = iterate on the symmetric affinity (K + K^t) / 2 of the kNN graph
                               (slk_symmetrize) instead of the directed K; rows then keep the given
                               order (reorder is ignored).  Default 0.  slk_solve_batched and the
                               server refuse 1 with SLK_ERR_INVALID_ARG */
} slk_params;

typedef struct {
    int32_t outer_iters;        /* outer iterations run */
    int32_t inner_iters_total;  /* z-updates summed over outer iterations */
    int32_t converged;          /* 1 if the modes stopped changing */
    float sigma;                /* kernel width used */
    double energy;              /* E of Eq. (1) after the last outer iteration */
    int64_t knn_fallback_rows;  /* kNN rows the first certificate left open (bfloat16: the rows
                                   sent to the two-term tensor-core stage) */
    int32_t ms_iters_total;     /* SLK-MS: mean-shift iterations summed over outer iterations */
    int64_t knn_float32_rows;   /* bfloat16: rows sent to the float32 stage (those the
                                   two-term certificate left open; below 100000 points, where
                                   the two-term stage is skipped, those the first certificate
                                   left open); 0 otherwise */
    int64_t knn_exact_rows;     /* rows recomputed by the exact float32 scan */
} slk_stats;

/* Fill *p with the defaults listed in slk_params. */
void slk_default_params(slk_params* p);

/* Whole SLK-BO on the GPU: kNN graph, kernel width (sigma <= 0: estimated by
 * params->sigma_rule), then Algorithm 1 from init_modes until the modes do
 * not change or params->max_outer outer iterations.
 *   init_modes [L] device int32 point indices (e.g. K-means++ seeds).
 *   Z [N x L], labels [N], modes [L]: device outputs.
 *   stats [host, nullable].
 * Returns SLK_NOT_CONVERGED (results valid) when max_outer is reached. */
slk_status slk_solve(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L, int32_t k,
                     float lambda, float sigma, const int32_t* init_modes,
                     const slk_params* params, float* Z, int32_t* labels, int32_t* modes,
                     slk_stats* stats);

/* slk_solve on HOST buffers: X [host, N x D], init_modes [host, L]; outputs
 * labels [host, N], modes [host, L] and Z [host, N x L, nullable].  Copies in
 * and out through the context's device workspace; for pinned host memory the
 * copies run at full link speed. */
slk_status slk_solve_host(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L,
                          int32_t k, float lambda, float sigma, const int32_t* init_modes,
                          const slk_params* params, float* Z, int32_t* labels, int32_t* modes,
                          slk_stats* stats);

/* K-means++ seeds (Section 4.2 takes the initial seeds from K-means++,
 * Arthur & Vassilvitskii 2007), with the random draws made by the caller:
 * seeds[0] = first; seeds[i] (i >= 1) is the first point p whose running sum
 * D(x_0)^2 + ... + D(x_p)^2 exceeds u[i-1] * sum_q D(x_q)^2, where D(x)^2 is
 * the squared Euclidean distance to the closest of seeds[0..i-1] (float64
 * sums); the last point if no running sum does, and point floor(u[i-1] N) if
 * every D(x)^2 is 0.  Two launches per seed: a float64 distance pass over X
 * and a one-block selection.
 *   X [N x D]; first in [0, N); u [host, L - 1] uniforms in [0, 1) (NULL
 *   allowed when L = 1); seeds [L] device int32 out.  1 <= L <= N.
 * Synchronises the context stream. */
slk_status slk_kmeanspp(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L,
                        int32_t first, const double* u, int32_t* seeds);

/* The symmetric affinity K' = (K + K^t) / 2 of a sparse K (Prop. 1 assumes a
 * symmetric psd K; the kNN affinity of Section 4.2 is directed).  Row p of K'
 * is the union of row p and column p of K by increasing column, with
 * K'_pq = (K_pq + K_qp) / 2 (float32) and a missing entry counting 0.
 *   row_ptr [N+1], col_idx [nnz], w [nnz] or NULL (binary): K on the device,
 *   every row with at most SLK_MAX_K entries (a kNN graph), else
 *   SLK_ERR_INVALID_ARG.
 *   out_row_ptr [N+1], out_col [2 nnz], out_w [2 nnz]: device outputs sized
 *   for the largest case (no entry of K mirrored by another); out_nnz [host,
 *   nullable] receives out_row_ptr[N].  Synchronises the context stream. */
slk_status slk_symmetrize(slk_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx,
                          const float* w, int64_t N, int64_t* out_row_ptr, int32_t* out_col,
                          float* out_w, int64_t* out_nnz);

/* Starting modes (Section 4.2: the starting mode of each cluster follows the
 * mode definition of Eq. (1) from the initial assignments): every point is
 * assigned to its nearest seed (squared Euclidean distance, ties to the
 * smaller l), then
 *   modes[l] = argmax_{y in X} sum_{p: assign[p] = l} k(x_p, y),
 * k the Gaussian kernel of width sigma, ties to the smaller index; a cluster
 * with no point keeps its seed.  The dense N x N kernel sums run as float32
 * distance tiles of the centred data (norm expansion) with float64 row sums;
 * their rounding bound selects the points that can still be the maximiser,
 * whose sums are then recomputed from float32 differences (float64 sums).
 *   seeds [L] device int32 (e.g. K-means++ indices); modes [L] device out;
 *   assign [N] device out (nullable); density [L] host out (nullable): the
 *   maximum of each cluster's sum (0 for an empty cluster); candidates [host,
 *   nullable]: the number of (point, cluster) sums recomputed exactly. */
slk_status slk_initial_modes(slk_ctx* ctx, const float* X, int64_t N, int32_t D,
                             const int32_t* seeds, int32_t L, float sigma, int32_t* modes,
                             int32_t* assign, double* density, int64_t* candidates);

/* ---------------------------------------------------------------- SLK-MS
 * The mean-shift variant of Algorithm 1 (Section 3.1, "Modes via
 * mean-shift"; Algorithm 1, SLK-MS branch): the modes are vectors m_l in R^D
 * instead of data points.  M is L x D float32 row-major on the DEVICE. */

#define SLK_MS_MAX_D 4096

/* a_{p,l} = exp(-||x_p - m_l||^2 / (2 sigma^2)) with vector modes M
 * (Eq. general-second); Z0 [nullable] = softmax rows as in slk_unary. */
slk_status slk_unary_vec(slk_ctx* ctx, const float* X, int64_t N, int32_t D, const float* M,
                         int32_t L, float sigma, float* A, float* Z0);

/* SLK-MS mode update, Eq. (mean-shift), iterated with the assignments fixed:
 *   m_l <- sum_p z_{p,l} k(x_p, m_l) x_p / sum_p z_{p,l} k(x_p, m_l)
 * for every l from the same previous modes, until max_l ||m_l^new - m_l^old||_2
 * <= tol * sigma (tol < 0: exactly max_iters iterations) or max_iters.  z is
 * the final iterate of the inner loop; it enters through the logits of its
 * last update (A, Z_prev, graph and lambda as in slk_mode_update; Z_prev NULL:
 * no update ran and s = a) as log z = log softmax(s), so float32 z that round
 * to 0 or 1 keep their weights.  Sums are taken relative to the largest
 * exponent per label, combined across the grid in float64; the iteration state
 * is float64 inside one call.
 *   X [N x D], A [N x L], Z_prev [N x L, nullable]: device inputs;
 *   M [L x D] device, in: starting modes, out: modes after the last iteration;
 *   labels [N, device, nullable] out: argmax_l z_{p,l}, ties to the smaller l;
 *   iters_done, last_shift [host, nullable]: iterations run and the largest
 *   move of the last one.
 * 1 <= D <= SLK_MS_MAX_D.  Returns SLK_ERR_TIMEOUT if a bounded wait gave up. */
slk_status slk_mean_shift(slk_ctx* ctx, const float* X, int32_t D, const float* A,
                          const float* Z_prev, const int64_t* row_ptr, const int32_t* col_idx,
                          const float* w, int64_t N, int32_t L, float lambda, float sigma,
                          float* M, int32_t max_iters, float tol, int32_t* labels,
                          int32_t* iters_done, float* last_shift);

/* Eq. (1) at one-hot labels with vector modes M (otherwise as slk_energy). */
slk_status slk_energy_vec(slk_ctx* ctx, const float* X, int32_t D, const int32_t* labels,
                          const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                          int64_t N, int32_t L, const float* M, float sigma, float lambda,
                          double* E);

/* Whole SLK-MS on the GPU: kNN graph and sigma as in slk_solve, modes
 * m_l^0 = x_{init_modes[l]}, then per outer iteration: unary term from M,
 * z = softmax(a), z-updates (Eq. soft-max), labels, mean-shift modes
 * (slk_mean_shift with params->max_ms, params->tol_ms), energy.  Stops when
 * no mode moved more than params->tol_modes * sigma in an outer iteration, or
 * after params->max_outer.
 *   init_modes [L] device int32; Z [N x L], labels [N], M [L x D]: device outputs.
 * Returns SLK_NOT_CONVERGED (results valid) when max_outer is reached. */
slk_status slk_solve_ms(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L, int32_t k,
                        float lambda, float sigma, const int32_t* init_modes,
                        const slk_params* params, float* Z, int32_t* labels, float* M,
                        slk_stats* stats);

/* One clustering problem of a batch (all pointers DEVICE, caller-owned). */
typedef struct {
    const float* X;             /* N x D features */
    int64_t N;
    int32_t D;
    int32_t L;                  /* 1 <= L <= SLK_BATCH_MAX_L */
    int32_t k;                  /* kNN neighbours */
    float lambda;
    float sigma;                /* <= 0: estimated by params->sigma_rule */
    const int32_t* init_modes;  /* [L] initial mode indices */
    float* Z;                   /* out [N x L] */
    int32_t* labels;            /* out [N] */
    int32_t* modes;             /* out [L] */
} slk_instance;

#define SLK_BATCH_MAX_L 128
#define SLK_BATCH_MAX_COUNT 4096

/* Batched SLK-BO: `count` independent problems of different N, D, L solved
 * together.  Each gets its own kNN graph and sigma (as in slk_solve); the
 * iterative part of Algorithm 1 then runs for all of them at once:
 * segmented unary, mode-update and energy kernels over the concatenated
 * rows, and one persistent segment-indexed launch for the z-updates
 * (Eq. soft-max), with a convergence test, iteration count and outer-loop
 * state per problem, so every result equals the one slk_solve gives for
 * that problem alone.  The per-outer-iteration launch sequence is captured
 * once in a CUDA graph and replayed; the launch shape of the z-update kernel
 * (threads per block, rows per lane group) is chosen by timing the
 * candidates on the first batch of a given shape and cached in the context.
 *   instances [host array of count, 1 <= count <= SLK_BATCH_MAX_COUNT], params as in slk_solve (max_outer,
 *   max_inner, tol_inner, sigma_rule, affinity, knn_precision), stats [host
 *   array of count, nullable].
 * Returns SLK_NOT_CONVERGED when some problem hit max_outer. */
slk_status slk_solve_batched(slk_ctx* ctx, const slk_instance* instances, int32_t count,
                             const slk_params* params, slk_stats* stats);

/* Continuous-batching server.  Requests (slk_instance, device pointers that
 * stay valid until the request is done) are queued by slk_server_submit and
 * admitted, first come first served, when a slot is free and the request's
 * device state fits in the server's memory arena (memory_bytes, allocated
 * once by slk_server_create): kNN graph, unary term, scratch iterate, and the
 * kNN scratch while the graph is being built.  An admitted request's graph
 * and sigma are built on an auxiliary stream, overlapping the work already
 * on the device.  slk_server_step admits what fits, then advances every
 * request that has its graph by one step -- the start of an outer iteration
 * when due, up to `quantum` z-updates (one persistent launch for all
 * requests), and the mode update and energy for requests whose inner loop
 * ended -- and releases the requests that finished.  Every request keeps its
 * own update count, convergence test and outer-loop state on the device, so
 * its result is the same alone and in any mix.
 *   cfg: max_slots (1 .. SLK_BATCH_MAX_COUNT), quantum (>= 1), memory_bytes.
 *   params: as in slk_solve; applied to every request.
 * slk_server_step synchronises the context stream; n_running / n_queued
 * [host, nullable] receive the counts after the step.  slk_server_poll
 * reports a ticket's state (0 queued, 1 building its graph, 2 iterating,
 * 3 done, with stats [host, nullable]); a done ticket is reported once and
 * then forgotten.  A request larger than the whole arena is refused at
 * submission with SLK_ERR_OOM. */
typedef struct slk_server slk_server;
typedef struct {
    int32_t max_slots;
    int32_t quantum;
    int64_t memory_bytes;
} slk_server_config;
slk_status slk_server_create(slk_ctx* ctx, const slk_server_config* cfg, const slk_params* params,
                             slk_server** out);
slk_status slk_server_destroy(slk_server* srv);
slk_status slk_server_submit(slk_server* srv, const slk_instance* req, int64_t* ticket);
slk_status slk_server_step(slk_server* srv, int32_t* n_running, int32_t* n_queued);
slk_status slk_server_poll(slk_server* srv, int64_t ticket, int32_t* state, slk_stats* stats);
/* Arena bytes a request needs while its graph is built (its peak) [host out]. */
slk_status slk_server_request_bytes(slk_server* srv, const slk_instance* req, int64_t* bytes);

/* slk_bound_iterate for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a deployment variant.  It serves code
 * that may not call cudaMalloc -- for example a plug-in running inside a
 * host framework that has already reserved the device memory for its own
 * pool, or a latency-critical serving loop where an allocation (which can
 * synchronise the whole device) is not allowed after start-up.  It needs
 * no context and allocates nothing: the ping-pong iterate and the barrier /
 * convergence words live in one file-scope static device array of
 * SLK_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads this library
 * holds until the process exits.
 *   stream   cudaStream_t to run on; the work runs on the calling thread's
 *            current device.
 *   A, row_ptr, col_idx, w, N, L, lambda, Z, max_iters, tol, iters_done,
 *   last_delta: as in slk_bound_iterate (Z in: starting iterate, out: the
 *            last iterate); the previous iterate is not returned.
 * N * L must not exceed SLK_NOALLOC_MAX_ELEMS, else SLK_ERR_SCRATCH_LIMIT is
 * returned before anything runs.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress), and so does the first call
 * after the device's context was replaced (cudaDeviceReset); make that first
 * call before any stream capture.  Every call reuses the same array and
 * re-initialises the words that must start at zero; calls that overlap on the
 * GPU (other streams, other threads) race on it and must be serialised by the
 * caller.  After SLK_ERR_TIMEOUT, Z is undefined.  The call synchronises
 * `stream` before returning. */
#define SLK_NOALLOC_MAX_ELEMS (4u << 20)   /* 4,194,304 floats = 16 MiB */
#define SLK_NOALLOC_SCRATCH_BYTES (4096u + 4u * SLK_NOALLOC_MAX_ELEMS)
slk_status slk_bound_iterate_noalloc(void* stream, const float* A, const int64_t* row_ptr,
                                     const int32_t* col_idx, const float* w, int64_t N,
                                     int32_t L, float lambda, float* Z, int32_t max_iters,
                                     float tol, int32_t* iters_done, float* last_delta);

/* Phase profiling.  While enabled, every call records a pair of CUDA events
 * on the context's stream around each phase below (no synchronisation is
 * added); slk_profile_read synchronises the stream and returns, per phase,
 * the summed device time in milliseconds and the number of timed calls,
 * plus the number of kernels the library launched since profiling was
 * enabled (counted whether or not events are recorded).  Enabling clears the
 * totals. */
enum {
    SLK_PHASE_KNN_PREP = 0,     /* centring, rounding, norms */
    SLK_PHASE_KNN_CAND,         /* distance tiles + per-row candidate lists */
    SLK_PHASE_KNN_RERANK,       /* exact float32 rerank + certificate */
    SLK_PHASE_KNN_FALLBACK,     /* exact scan of uncertified rows */
    SLK_PHASE_SIGMA,
    SLK_PHASE_UNARY,
    SLK_PHASE_BOUND,            /* z-updates (inner loop) */
    SLK_PHASE_MODE,
    SLK_PHASE_ENERGY,
    SLK_PHASE_MEANSHIFT,        /* SLK-MS mode iterations */
    SLK_PHASE_TRANSFER,         /* host <-> device copies of the host-buffer entry points */
    SLK_PHASE_COUNT
};
slk_status slk_profile(slk_ctx* ctx, int32_t enable);
slk_status slk_profile_read(slk_ctx* ctx, double* ms /* [host, SLK_PHASE_COUNT] */,
                            int64_t* calls /* [host, SLK_PHASE_COUNT] */,
                            int64_t* kernel_launches /* [host] */);

#ifdef __cplusplus
}
#endif
#endif /* SLK_H */
