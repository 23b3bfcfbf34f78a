/*
 * FP64 CPU oracle for Scalable Laplacian K-modes, SLK-BO and SLK-MS variants
 * (Ziko, Granger, Ben Ayed, NeurIPS 2018, arXiv:1810.13044).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
 * reference legs may load it.  It shares no code, header, table or constant
 * with the CUDA library, and it never reads anything the CUDA path produced.
 *
 * Plain, slow, obviously correct: every function is the paper's definition
 * written out with scalar loops in double precision.  Built with OpenMP, the
 * loops whose iterations are independent (one output row each, or a
 * maximum) are shared among threads; every sum keeps its sequential order,
 * so results do not depend on the thread count.
 * Inputs X are the float32 features; every other real value is double.
 *
 * Conventions: X is N x D row-major; A, Z, S are N x L row-major; the affinity
 * graph is CSR (row_ptr[N+1] int64, col_idx[nnz] int32, w[nnz] double or NULL
 * for binary weights).  Indices are 0-based.  Functions return 0 on success
 * and a negative code on bad arguments (nothing is written then).
 */
#ifndef SLK_ORACLE_H
#define SLK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of threads of the row-parallel loops (n > 0 sets it first);
 * 1 when the library was built without OpenMP. */
int oracle_threads(int n);

/* Exact kNN of Section 4.2: for each requested row p, the k points q != p with
 * the smallest squared Euclidean distance, ascending by (distance, index). */
int oracle_knn_rows(const float* X, int64_t N, int D, int k,
                    const int64_t* rows, int64_t nrows,
                    int32_t* idx_out, double* d2_out);
int oracle_knn(const float* X, int64_t N, int D, int k, int32_t* idx_out, double* d2_out);

/* Squared distances ||x_p[i] - x_q[i]||^2 of n point pairs (the sum of the
 * kNN scan, so they equal the d2 it reports for the same pairs). */
int oracle_pair_d2(const float* X, int64_t N, int D, const int64_t* p, const int64_t* q,
                   int64_t n, double* out);

/* Kernel width of Section 4.2.  rule 0: sigma = median of the n Euclidean
 * kNN distances sqrt(d2) (mean of the two middle values for even n);
 * rule 1: sigma^2 = mean of the squared kNN distances (the paper's estimator). */
double oracle_sigma(const double* d2, int64_t n, int rule);

/* Gaussian kernel of Section 4.2: exp(-d2 / (2 sigma^2)). */
double oracle_gauss(double d2, double sigma);

/* Heat-kernel edge weights w_e = exp(-d2_e / (2 sigma^2)). */
void oracle_heat_weights(const double* d2, int64_t nnz, double sigma, double* w);

/* Unary term, Eq. (general-second): a_{p,l} = k(x_p, m_l) with m_l = x_{modes[l]}. */
int oracle_unary(const float* X, int64_t N, int D, const int32_t* modes, int L,
                 double sigma, double* A);

/* Row softmax z_p = exp(s_p) / 1^t exp(s_p) (Algorithm 1 initialisation with s = a). */
void oracle_softmax_rows(const double* S, int64_t N, int L, double* Z);

/* Pairwise term, Eq. (general-third): b_{p,l} = sum_q k(x_p, x_q) z_{q,l} over row p of K. */
void oracle_pairwise(const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                     int64_t N, int L, const double* Z, double* B);

/* Logits of the z-update, s_p = a_p + lambda b_p (argument of the soft-max update). */
void oracle_logits(const double* A, const int64_t* row_ptr, const int32_t* col_idx,
                   const double* w, int64_t N, int L, double lambda,
                   const double* Z, double* S);

/* Inner loop of Algorithm 1: repeat the soft-max z-update (Jacobi: every row
 * from the previous Z) until max |z_new - z_old| <= tol or max_iters updates.
 * Z is in/out.  If Zprev is not NULL it receives the iterate the last update
 * started from (needed for the mode keys).  tol < 0 runs exactly max_iters. */
int oracle_bound_iterate(const double* A, const int64_t* row_ptr, const int32_t* col_idx,
                         const double* w, int64_t N, int L, double lambda,
                         double* Z, int max_iters, double tol,
                         double* Zprev, int* iters_done, double* last_delta);

/* SLK-BO mode update, Eq. (mode_byproduct): m_l = argmax_q z_{q,l}, compared on
 * log z_{q,l} computed from the logits S of the last update (ties -> smaller q).
 * keys_out (nullable, N x L) receives log z_{q,l}. */
void oracle_log_z(const double* S, int64_t N, int L, double* logZ);
void oracle_mode_update(const double* S, int64_t N, int L, int32_t* modes_out, double* best_key);

/* Discrete labels: argmax_l z_{p,l} (ties -> smaller l), compared on the logits. */
void oracle_labels(const double* S, int64_t N, int L, int32_t* labels);

/* Discrete energy, Eq. (1), at one-hot assignments given by labels and modes
 * m_l = x_{modes[l]}:  -sum_p sum_l z_{p,l} k(x_p, m_l)
 *                      + lambda/2 sum_p sum_{q in row p} w_pq ||z_p - z_q||^2. */
double oracle_energy(const float* X, int D, const int32_t* labels,
                     const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                     int64_t N, int L, const int32_t* modes, double sigma, double lambda);

/* Relaxed objective, Eq. (2), with pairwise weight lam_pair:
 * sum_p z_p^t log z_p - sum_{p,l} z_{p,l} a_{p,l} - lam_pair sum_p sum_{q in row p} w_pq z_p^t z_q. */
double oracle_relaxed(const double* A, const double* Z, const int64_t* row_ptr,
                      const int32_t* col_idx, const double* w, int64_t N, int L,
                      double lam_pair);

/* Algorithm 1 (SLK-BO) on a given graph and kernel width.
 * Outer loop: a from the modes, z = softmax(a), inner z-updates, mode update,
 * energy; stop when the modes do not change or after max_outer steps.
 * Outputs: Z (N x L), labels[N], modes[L] (in: initial modes, out: final),
 * energy, and counters.  Returns 1 if max_outer was hit without convergence. */
int oracle_solve_graph(const float* X, int64_t N, int D, int L,
                       const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                       double sigma, double lambda, int32_t* modes,
                       int max_outer, int max_inner, double tol,
                       double* Z, int32_t* labels, double* energy,
                       int* outer_done, int* inner_total);

/* ---- SLK-MS (modes via mean-shift, Section 3.1 "Mode updates", Algorithm 1) ----
 * Modes are vectors m_l in R^D (M: L x D row-major, double). */

/* Unary term with vector modes: a_{p,l} = k(x_p, m_l). */
int oracle_unary_vec(const float* X, int64_t N, int D, const double* M, int L,
                     double sigma, double* A);

/* Eq. (mean-shift) with the assignments fixed: every iteration replaces, for
 * every l, m_l by  sum_p z_{p,l} k(x_p, m_l) x_p / sum_p z_{p,l} k(x_p, m_l),
 * all labels from the same previous M.  z is given as logZ = log z_{p,l}
 * (N x L).  Stops when max_l ||m_l^new - m_l^old||_2 <= tol * sigma, or after
 * max_iters iterations; tol < 0 runs exactly max_iters.  M is in/out. */
int oracle_mean_shift(const float* X, int64_t N, int D, const double* logZ, int L,
                      double sigma, double* M, int max_iters, double tol,
                      int* iters_done, double* last_shift);

/* Eq. (1) at one-hot labels with vector modes:
 * -sum_p k(x_p, m_{labels[p]}) + lambda/2 sum_p sum_{q in row p} w_pq ||z_p - z_q||^2. */
double oracle_energy_vec(const float* X, int D, const int32_t* labels,
                         const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                         int64_t N, int L, const double* M, double sigma, double lambda);

/* Algorithm 1 (SLK-MS) on a given graph and kernel width.  Outer loop: a from
 * the modes, z = softmax(a), inner z-updates, mean-shift mode update, labels,
 * energy; stop when max_l ||m_l^new - m_l^old||_2 <= tol_outer * sigma or after
 * max_outer steps.  M (L x D) in: initial modes, out: final.  Returns 1 if
 * max_outer was hit without convergence. */
int oracle_solve_ms_graph(const float* X, int64_t N, int D, int L,
                          const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                          double sigma, double lambda, double* M,
                          int max_outer, int max_inner, double tol,
                          int max_ms, double tol_ms, double tol_outer,
                          double* Z, int32_t* labels, double* energy,
                          int* outer_done, int* inner_total, int* ms_total);

/* ---- Starting modes (Section 4.2: the starting mode of each cluster follows
 * the mode definition of Eq. (1) from the initial assignments) ----
 * assign[p] = argmin_l ||x_p - x_{seeds[l]}||^2 (ties to the smaller l); then
 * m_l = argmax_{y in X} sum_{p: assign[p] = l} k(x_p, y), ties to the smaller
 * index.  density_out [L, nullable] receives the maximum of each cluster's sum;
 * a cluster with no point keeps its seed (density 0). */
int oracle_initial_modes(const float* X, int64_t N, int D, const int32_t* seeds, int L,
                         double sigma, int32_t* modes_out, int32_t* assign_out,
                         double* density_out);

/* The cluster density sum_{p: assign[p] = l} k(x_p, x_y) at the given points y. */
int oracle_cluster_density(const float* X, int64_t N, int D, const int32_t* assign, int l,
                           double sigma, const int64_t* ys, int64_t ny, double* out);

/* ---- K-means++ seeds (Section 4.2 cites Arthur & Vassilvitskii 2007) ----
 * seeds[0] = first; seeds[i] = the first p whose running sum of
 * D(x_p)^2 (squared distance to the closest of seeds[0..i-1]) exceeds
 * u[i-1] * sum_p D(x_p)^2, the last point if none does; if every D(x)^2 is 0,
 * point floor(u[i-1] N).  u: L - 1 uniform draws in [0, 1). */
int oracle_kmeanspp(const float* X, int64_t N, int D, int L, int32_t first, const double* u,
                    int32_t* seeds);

/* ---- Symmetric affinity (Prop. 1 assumes a symmetric psd K) ----
 * K' = (K + K^t) / 2 of the CSR K (w = NULL: binary).  Row p of K' is the
 * union of row p and column p of K by increasing column, K'_pq =
 * (K_pq + K_qp) / 2 with missing entries 0.  Call once with out_col = NULL
 * for out_row_ptr[N + 1], then with out_col / out_w of out_row_ptr[N] slots. */
int oracle_symmetrize(const int64_t* row_ptr, const int32_t* col_idx, const double* w, int64_t N,
                      int64_t* out_row_ptr, int32_t* out_col, double* out_w, int64_t out_cap);

#ifdef __cplusplus
}
#endif
#endif
