/*
 * FP64 CPU oracle for Scalable Laplacian K-modes (SLK-BO).
 *
 * TEST INFRASTRUCTURE ONLY -- see slk_oracle.h.  Every function restates one
 * definition of the paper in plain loops; the comment above each names the
 * section / equation it follows.  No blocking, fusion or reordering beyond
 * what the definition states.
 */
#include "slk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the row-parallel loops.  Only loops whose iterations are
 * independent (one output row each, or a maximum) run in parallel, so the
 * results are bit-identical for every thread count. */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static int thread_index(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* ||x_p - x_q||^2 with every difference and product in double.  A float
 * difference is exact in double and so is its square (two 24-bit
 * significands), so only the running sum rounds. */
static double sqdist(const float* X, int D, int64_t p, int64_t q)
{
    const float* a = X + p * (int64_t)D;
    const float* b = X + q * (int64_t)D;
    double s = 0.0;
    for (int j = 0; j < D; ++j) {
        double d = (double)a[j] - (double)b[j];
        s += d * d;
    }
    return s;
}

/* Section 4.2: kNN affinity, N_p = the k nearest neighbours of x_p by
 * Euclidean distance.  The point itself is excluded; ties go to the smaller
 * index (the scan runs over increasing q and only a strictly smaller
 * distance displaces an earlier entry).  bd / bi hold the sorted list. */
static void knn_one_row(const float* X, int64_t N, int D, int k, int64_t p,
                        double* bd, int32_t* bi, int32_t* idx_out, double* d2_out)
{
    int count = 0;
    for (int64_t q = 0; q < N; ++q) {
        if (q == p) continue;
        double d = sqdist(X, D, p, q);
        if (count == k && !(d < bd[k - 1])) continue;
        /* insertion into the ascending list, after every entry <= d */
        int pos = count < k ? count : k - 1;
        while (pos > 0 && bd[pos - 1] > d) {
            if (pos < k) { bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; }
            --pos;
        }
        bd[pos] = d;
        bi[pos] = (int32_t)q;
        if (count < k) ++count;
    }
    memcpy(idx_out, bi, sizeof(int32_t) * (size_t)k);
    memcpy(d2_out, bd, sizeof(double) * (size_t)k);
}

int oracle_knn_rows(const float* X, int64_t N, int D, int k,
                    const int64_t* rows, int64_t nrows,
                    int32_t* idx_out, double* d2_out)
{
    if (!X || N < 2 || D < 1 || k < 1 || k > N - 1 || !rows || nrows < 0 || !idx_out || !d2_out)
        return -1;
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t p = rows[r];
        if (p < 0 || p >= N) return -1;
    }
    /* one sorted list per thread */
    int nt = oracle_threads(0);
    double* bd = (double*)malloc(sizeof(double) * (size_t)k * (size_t)nt);
    int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * (size_t)k * (size_t)nt);
    if (!bd || !bi) { free(bd); free(bi); return -2; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        int t = thread_index();
        knn_one_row(X, N, D, k, rows[r], bd + (size_t)t * k, bi + (size_t)t * k,
                    idx_out + r * k, d2_out + r * k);
    }
    free(bd);
    free(bi);
    return 0;
}

/* ||x_p - x_q||^2 (the sum of the kNN scan) for n given pairs. */
int oracle_pair_d2(const float* X, int64_t N, int D, const int64_t* p, const int64_t* q,
                   int64_t n, double* out)
{
    if (!X || N < 1 || D < 1 || !p || !q || n < 0 || !out) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (p[i] < 0 || p[i] >= N || q[i] < 0 || q[i] >= N) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = sqdist(X, D, p[i], q[i]);
    return 0;
}

int oracle_knn(const float* X, int64_t N, int D, int k, int32_t* idx_out, double* d2_out)
{
    if (N < 2) return -1;
    int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    if (!rows) return -2;
    for (int64_t p = 0; p < N; ++p) rows[p] = p;
    int rc = oracle_knn_rows(X, N, D, k, rows, N, idx_out, d2_out);
    free(rows);
    return rc;
}

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Section 4.2 kernel width.  rule 1 is the paper's estimator
 * sigma^2 = (1 / (N k)) sum_p sum_{q in N_p} ||x_p - x_q||^2; rule 0 takes the
 * median of the Euclidean kNN distances instead. */
double oracle_sigma(const double* d2, int64_t n, int rule)
{
    if (!d2 || n < 1) return -1.0;
    if (rule == 1) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += d2[i];
        return sqrt(s / (double)n);
    }
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    if (!v) return -1.0;
    for (int64_t i = 0; i < n; ++i) v[i] = sqrt(d2[i]);
    qsort(v, (size_t)n, sizeof(double), cmp_double);
    double med = (n % 2) ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
    free(v);
    return med;
}

/* Section 4.2: k(x, y) = exp(-||x - y||^2 / (2 sigma^2)). */
double oracle_gauss(double d2, double sigma)
{
    return exp(-d2 / (2.0 * sigma * sigma));
}

void oracle_heat_weights(const double* d2, int64_t nnz, double sigma, double* w)
{
    for (int64_t e = 0; e < nnz; ++e) w[e] = oracle_gauss(d2[e], sigma);
}

/* Eq. (general-second): a_{p,l} = k(x_p, m_l). */
int oracle_unary(const float* X, int64_t N, int D, const int32_t* modes, int L,
                 double sigma, double* A)
{
    if (!X || N < 1 || D < 1 || !modes || L < 1 || !(sigma > 0.0) || !A) return -1;
    for (int l = 0; l < L; ++l)
        if (modes[l] < 0 || modes[l] >= N) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p)
        for (int l = 0; l < L; ++l)
            A[p * L + l] = oracle_gauss(sqdist(X, D, p, modes[l]), sigma);
    return 0;
}

/* z_p = exp(s_p) / 1^t exp(s_p), evaluated as exp(s - max s) / sum exp(s - max s)
 * (the same ratio; the shift only keeps exp in range). */
void oracle_softmax_rows(const double* S, int64_t N, int L, double* Z)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        const double* s = S + p * L;
        double m = s[0];
        for (int l = 1; l < L; ++l) if (s[l] > m) m = s[l];
        double sum = 0.0;
        for (int l = 0; l < L; ++l) sum += exp(s[l] - m);
        for (int l = 0; l < L; ++l) Z[p * L + l] = exp(s[l] - m) / sum;
    }
}

/* Eq. (general-third): b_{p,l} = sum_q k(x_p, x_q) z_{q,l}, the sum running over
 * the non-zeros of row p of the sparse affinity matrix (w = NULL: all ones). */
void oracle_pairwise(const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                     int64_t N, int L, const double* Z, double* B)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        for (int l = 0; l < L; ++l) B[p * L + l] = 0.0;
        for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
            double kpq = w ? w[e] : 1.0;
            int64_t q = col_idx[e];
            for (int l = 0; l < L; ++l) B[p * L + l] += kpq * Z[q * L + l];
        }
    }
}

/* s_p = a_p + lambda b_p: the exponent of the soft-max update. */
void oracle_logits(const double* A, const int64_t* row_ptr, const int32_t* col_idx,
                   const double* w, int64_t N, int L, double lambda,
                   const double* Z, double* S)
{
    oracle_pairwise(row_ptr, col_idx, w, N, L, Z, S);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N * (int64_t)L; ++i) S[i] = A[i] + lambda * S[i];
}

/* Algorithm 1, inner loop: z_p^{i+1} = exp(a_p + lambda b_p^i) / 1^t exp(...),
 * all p from the same Z^i (the soft-max update, computed for every point in
 * parallel as Section 4.2 states), until convergence. */
int oracle_bound_iterate(const double* A, const int64_t* row_ptr, const int32_t* col_idx,
                         const double* w, int64_t N, int L, double lambda,
                         double* Z, int max_iters, double tol,
                         double* Zprev, int* iters_done, double* last_delta)
{
    if (!A || !row_ptr || !col_idx || N < 1 || L < 1 || !Z || max_iters < 0) return -1;
    size_t n = (size_t)N * (size_t)L;
    double* S = (double*)malloc(sizeof(double) * n);
    double* Znew = (double*)malloc(sizeof(double) * n);
    if (!S || !Znew) { free(S); free(Znew); return -2; }
    int it = 0;
    double delta = 0.0;
    while (it < max_iters) {
        oracle_logits(A, row_ptr, col_idx, w, N, L, lambda, Z, S);
        oracle_softmax_rows(S, N, L, Znew);
        delta = 0.0;
#pragma omp parallel for schedule(static) reduction(max : delta)
        for (size_t i = 0; i < n; ++i) {
            double d = fabs(Znew[i] - Z[i]);
            if (d > delta) delta = d;
        }
        if (Zprev) memcpy(Zprev, Z, sizeof(double) * n);
        memcpy(Z, Znew, sizeof(double) * n);
        ++it;
        if (tol >= 0.0 && delta <= tol) break;
    }
    if (iters_done) *iters_done = it;
    if (last_delta) *last_delta = delta;
    free(S);
    free(Znew);
    return 0;
}

/* log z_{q,l} of the soft-max of the logits S:
 * (s_l - m) - log(1 + sum_{j != j*} exp(s_j - m)), m = s_{j*} = max_j s_j,
 * the log1p form keeping full precision when z_{q,l} is close to 1. */
void oracle_log_z(const double* S, int64_t N, int L, double* logZ)
{
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < N; ++q) {
        const double* s = S + q * L;
        int jstar = 0;
        for (int j = 1; j < L; ++j) if (s[j] > s[jstar]) jstar = j;
        double r = 0.0;
        for (int j = 0; j < L; ++j) if (j != jstar) r += exp(s[j] - s[jstar]);
        double lse1 = log1p(r);
        for (int l = 0; l < L; ++l) logZ[q * L + l] = (s[l] - s[jstar]) - lse1;
    }
}

/* Eq. (mode_byproduct): m_l = x_p with p = argmax_q z_{q,l}; compared on
 * log z (a monotone map of z), ties to the smaller q. */
void oracle_mode_update(const double* S, int64_t N, int L, int32_t* modes_out, double* best_key)
{
    double* logZ = (double*)malloc(sizeof(double) * (size_t)N * (size_t)L);
    if (!logZ) return;
    oracle_log_z(S, N, L, logZ);
    for (int l = 0; l < L; ++l) {
        int64_t best = 0;
        for (int64_t q = 1; q < N; ++q)
            if (logZ[q * L + l] > logZ[best * L + l]) best = q;
        modes_out[l] = (int32_t)best;
        if (best_key) best_key[l] = logZ[best * L + l];
    }
    free(logZ);
}

/* Discrete assignment of point p: argmax_l z_{p,l} (= argmax_l s_{p,l}, the
 * soft-max being monotone within a row), ties to the smaller l. */
void oracle_labels(const double* S, int64_t N, int L, int32_t* labels)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int best = 0;
        for (int l = 1; l < L; ++l) if (S[p * L + l] > S[p * L + best]) best = l;
        labels[p] = best;
    }
}

/* Eq. (1) at one-hot z_p = e_{labels[p]}:
 * E = -sum_p sum_l z_{p,l} k(x_p, m_l) + lambda/2 sum_p sum_q k(x_p, x_q) ||z_p - z_q||^2,
 * with k(x_p, x_q) the sparse affinity (row p of the CSR). */
double oracle_energy(const float* X, int D, const int32_t* labels,
                     const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                     int64_t N, int L, const int32_t* modes, double sigma, double lambda)
{
    double unary = 0.0, pair = 0.0;
    for (int64_t p = 0; p < N; ++p) {
        for (int l = 0; l < L; ++l) {
            double zpl = (labels[p] == l) ? 1.0 : 0.0;
            if (zpl != 0.0) unary += zpl * oracle_gauss(sqdist(X, D, p, modes[l]), sigma);
        }
        for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
            int64_t q = col_idx[e];
            double kpq = w ? w[e] : 1.0;
            double n2 = 0.0;
            for (int l = 0; l < L; ++l) {
                double d = ((labels[p] == l) ? 1.0 : 0.0) - ((labels[q] == l) ? 1.0 : 0.0);
                n2 += d * d;
            }
            pair += kpq * n2;
        }
    }
    return -unary + 0.5 * lambda * pair;
}

/* Eq. (2): sum_p z_p^t log z_p - sum_{p,l} z_{p,l} a_{p,l}
 *          - lam_pair sum_{p,q} k(x_p, x_q) z_p^t z_q (0 log 0 = 0). */
double oracle_relaxed(const double* A, const double* Z, const int64_t* row_ptr,
                      const int32_t* col_idx, const double* w, int64_t N, int L,
                      double lam_pair)
{
    double ent = 0.0, un = 0.0, pair = 0.0;
    for (int64_t p = 0; p < N; ++p) {
        for (int l = 0; l < L; ++l) {
            double z = Z[p * L + l];
            if (z > 0.0) ent += z * log(z);
            un += z * A[p * L + l];
        }
        for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
            int64_t q = col_idx[e];
            double kpq = w ? w[e] : 1.0;
            double dot = 0.0;
            for (int l = 0; l < L; ++l) dot += Z[p * L + l] * Z[q * L + l];
            pair += kpq * dot;
        }
    }
    return ent - un - lam_pair * pair;
}

/* Algorithm 1 (SLK-BO), outer loop: modes fixed -> a; z = softmax(a); inner
 * z-updates; modes as by-products (Eq. mode_byproduct); repeat until the modes
 * do not change (Section 3's stopping rule). */
int oracle_solve_graph(const float* X, int64_t N, int D, int L,
                       const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                       double sigma, double lambda, int32_t* modes,
                       int max_outer, int max_inner, double tol,
                       double* Z, int32_t* labels, double* energy,
                       int* outer_done, int* inner_total)
{
    if (!X || N < 1 || D < 1 || L < 1 || L > N || !row_ptr || !col_idx || !(sigma > 0.0) ||
        !modes || max_outer < 1 || max_inner < 0 || !Z || !labels || !energy)
        return -1;
    size_t n = (size_t)N * (size_t)L;
    double* A = (double*)malloc(sizeof(double) * n);
    double* Zp = (double*)malloc(sizeof(double) * n);
    double* S = (double*)malloc(sizeof(double) * n);
    int32_t* newm = (int32_t*)malloc(sizeof(int32_t) * (size_t)L);
    if (!A || !Zp || !S || !newm) { free(A); free(Zp); free(S); free(newm); return -2; }
    int converged = 0, t = 0, total = 0;
    for (t = 0; t < max_outer && !converged; ++t) {
        oracle_unary(X, N, D, modes, L, sigma, A);
        oracle_softmax_rows(A, N, L, Z);
        int it = 0;
        double dl = 0.0;
        oracle_bound_iterate(A, row_ptr, col_idx, w, N, L, lambda, Z, max_inner, tol, Zp, &it, &dl);
        total += it;
        if (it > 0) oracle_logits(A, row_ptr, col_idx, w, N, L, lambda, Zp, S);
        else memcpy(S, A, sizeof(double) * n);
        oracle_mode_update(S, N, L, newm, NULL);
        oracle_labels(S, N, L, labels);
        *energy = oracle_energy(X, D, labels, row_ptr, col_idx, w, N, L, newm, sigma, lambda);
        converged = (memcmp(newm, modes, sizeof(int32_t) * (size_t)L) == 0);
        memcpy(modes, newm, sizeof(int32_t) * (size_t)L);
    }
    if (outer_done) *outer_done = t;
    if (inner_total) *inner_total = total;
    free(A); free(Zp); free(S); free(newm);
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------ SLK-MS */

/* ||x_p - m||^2 with x_p a float32 row and m a double vector. */
static double sqdist_vec(const float* X, int D, int64_t p, const double* m)
{
    double s = 0.0;
    for (int j = 0; j < D; ++j) {
        double d = (double)X[p * D + j] - m[j];
        s += d * d;
    }
    return s;
}

/* Eq. (general-second) with m_l a vector: a_{p,l} = k(x_p, m_l). */
int oracle_unary_vec(const float* X, int64_t N, int D, const double* M, int L,
                     double sigma, double* A)
{
    if (!X || N < 1 || D < 1 || !M || L < 1 || !(sigma > 0.0) || !A) return -1;
    for (int64_t p = 0; p < N; ++p)
        for (int l = 0; l < L; ++l)
            A[p * L + l] = oracle_gauss(sqdist_vec(X, D, p, M + (size_t)l * D), sigma);
    return 0;
}

/* Eq. (mean-shift).  The weight of point p for mode l is
 * z_{p,l} k(x_p, m_l) = exp(log z_{p,l} - ||x_p - m_l||^2 / (2 sigma^2)); every
 * weight of label l is multiplied by exp(-c_l), c_l the largest exponent of
 * that label, which cancels in the ratio and keeps the sums away from
 * underflow when a mode is far from every point. */
int oracle_mean_shift(const float* X, int64_t N, int D, const double* logZ, int L,
                      double sigma, double* M, int max_iters, double tol,
                      int* iters_done, double* last_shift)
{
    if (!X || N < 1 || D < 1 || !logZ || L < 1 || !(sigma > 0.0) || !M || max_iters < 0)
        return -1;
    double* Mn = (double*)malloc(sizeof(double) * (size_t)L * (size_t)D);
    double* ex = (double*)malloc(sizeof(double) * (size_t)N);
    if (!Mn || !ex) { free(Mn); free(ex); return -2; }
    int it = 0;
    double shift = 0.0;
    while (it < max_iters) {
        shift = 0.0;
        for (int l = 0; l < L; ++l) {
            const double* m = M + (size_t)l * D;
            double c = -INFINITY;
            for (int64_t p = 0; p < N; ++p) {
                ex[p] = logZ[p * L + l] - sqdist_vec(X, D, p, m) / (2.0 * sigma * sigma);
                if (ex[p] > c) c = ex[p];
            }
            double den = 0.0;
            double* mn = Mn + (size_t)l * D;
            for (int j = 0; j < D; ++j) mn[j] = 0.0;
            for (int64_t p = 0; p < N; ++p) {
                double wp = exp(ex[p] - c);
                den += wp;
                for (int j = 0; j < D; ++j) mn[j] += wp * (double)X[p * D + j];
            }
            double s2 = 0.0;
            for (int j = 0; j < D; ++j) {
                mn[j] /= den;
                s2 += (mn[j] - m[j]) * (mn[j] - m[j]);
            }
            if (sqrt(s2) > shift) shift = sqrt(s2);
        }
        memcpy(M, Mn, sizeof(double) * (size_t)L * (size_t)D);
        ++it;
        if (tol >= 0.0 && shift <= tol * sigma) break;
    }
    if (iters_done) *iters_done = it;
    if (last_shift) *last_shift = shift;
    free(Mn);
    free(ex);
    return 0;
}

/* Eq. (1) at one-hot labels, modes given as vectors. */
double oracle_energy_vec(const float* X, int D, const int32_t* labels,
                         const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                         int64_t N, int L, const double* M, double sigma, double lambda)
{
    double unary = 0.0, pair = 0.0;
    for (int64_t p = 0; p < N; ++p) {
        for (int l = 0; l < L; ++l)
            if (labels[p] == l) unary += oracle_gauss(sqdist_vec(X, D, p, M + (size_t)l * D), sigma);
        for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
            int64_t q = col_idx[e];
            double kpq = w ? w[e] : 1.0;
            double n2 = 0.0;
            for (int l = 0; l < L; ++l) {
                double d = ((labels[p] == l) ? 1.0 : 0.0) - ((labels[q] == l) ? 1.0 : 0.0);
                n2 += d * d;
            }
            pair += kpq * n2;
        }
    }
    return -unary + 0.5 * lambda * pair;
}

/* Algorithm 1 with the SLK-MS branch: modes from Eq. (mean-shift) run to
 * convergence with Z fixed after the inner z-updates. */
int oracle_solve_ms_graph(const float* X, int64_t N, int D, int L,
                          const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                          double sigma, double lambda, double* M,
                          int max_outer, int max_inner, double tol,
                          int max_ms, double tol_ms, double tol_outer,
                          double* Z, int32_t* labels, double* energy,
                          int* outer_done, int* inner_total, int* ms_total)
{
    if (!X || N < 1 || D < 1 || L < 1 || L > N || !row_ptr || !col_idx || !(sigma > 0.0) ||
        !M || max_outer < 1 || max_inner < 0 || max_ms < 0 || !Z || !labels || !energy)
        return -1;
    size_t n = (size_t)N * (size_t)L;
    double* A = (double*)malloc(sizeof(double) * n);
    double* Zp = (double*)malloc(sizeof(double) * n);
    double* S = (double*)malloc(sizeof(double) * n);
    double* LZ = (double*)malloc(sizeof(double) * n);
    double* M0 = (double*)malloc(sizeof(double) * (size_t)L * (size_t)D);
    if (!A || !Zp || !S || !LZ || !M0) {
        free(A); free(Zp); free(S); free(LZ); free(M0);
        return -2;
    }
    int converged = 0, t = 0, total = 0, mstotal = 0;
    for (t = 0; t < max_outer && !converged; ++t) {
        oracle_unary_vec(X, N, D, M, L, sigma, A);
        oracle_softmax_rows(A, N, L, Z);
        int it = 0;
        double dl = 0.0;
        oracle_bound_iterate(A, row_ptr, col_idx, w, N, L, lambda, Z, max_inner, tol, Zp, &it, &dl);
        total += it;
        if (it > 0) oracle_logits(A, row_ptr, col_idx, w, N, L, lambda, Zp, S);
        else memcpy(S, A, sizeof(double) * n);
        oracle_log_z(S, N, L, LZ);
        oracle_labels(S, N, L, labels);
        memcpy(M0, M, sizeof(double) * (size_t)L * (size_t)D);
        int ms = 0;
        double sh = 0.0;
        oracle_mean_shift(X, N, D, LZ, L, sigma, M, max_ms, tol_ms, &ms, &sh);
        mstotal += ms;
        *energy = oracle_energy_vec(X, D, labels, row_ptr, col_idx, w, N, L, M, sigma, lambda);
        double moved = 0.0;
        for (int l = 0; l < L; ++l) {
            double s2 = 0.0;
            for (int j = 0; j < D; ++j) {
                double d = M[(size_t)l * D + j] - M0[(size_t)l * D + j];
                s2 += d * d;
            }
            if (sqrt(s2) > moved) moved = sqrt(s2);
        }
        converged = (moved <= tol_outer * sigma);
    }
    if (outer_done) *outer_done = t;
    if (inner_total) *inner_total = total;
    if (ms_total) *ms_total = mstotal;
    free(A); free(Zp); free(S); free(LZ); free(M0);
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------ starting modes */

/* Initial assignment to the nearest seed, then the mode definition of
 * Eq. (1) with that one-hot z: the data point of largest cluster density. */
int oracle_initial_modes(const float* X, int64_t N, int D, const int32_t* seeds, int L,
                         double sigma, int32_t* modes_out, int32_t* assign_out,
                         double* density_out)
{
    if (!X || N < 1 || D < 1 || !seeds || L < 1 || !(sigma > 0.0) || !modes_out) return -1;
    for (int l = 0; l < L; ++l)
        if (seeds[l] < 0 || seeds[l] >= N) return -1;
    int32_t* assign = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    double* dens = (double*)malloc(sizeof(double) * (size_t)L);
    if (!assign || !dens) { free(assign); free(dens); return -2; }
    for (int64_t p = 0; p < N; ++p) {
        int best = 0;
        double bd = sqdist(X, D, p, seeds[0]);
        for (int l = 1; l < L; ++l) {
            double d = sqdist(X, D, p, seeds[l]);
            if (d < bd) { bd = d; best = l; }
        }
        assign[p] = best;
    }
    for (int l = 0; l < L; ++l) { modes_out[l] = seeds[l]; dens[l] = 0.0; }
    for (int l = 0; l < L; ++l) {
        int any = 0;
        for (int64_t p = 0; p < N && !any; ++p) any = (assign[p] == l);
        if (!any) continue;
        double best = -1.0;
        for (int64_t y = 0; y < N; ++y) {
            double f = 0.0;
            for (int64_t p = 0; p < N; ++p)
                if (assign[p] == l) f += oracle_gauss(sqdist(X, D, p, y), sigma);
            if (f > best) { best = f; modes_out[l] = (int32_t)y; }
        }
        dens[l] = best;
    }
    if (assign_out) memcpy(assign_out, assign, sizeof(int32_t) * (size_t)N);
    if (density_out) memcpy(density_out, dens, sizeof(double) * (size_t)L);
    free(assign);
    free(dens);
    return 0;
}

int oracle_cluster_density(const float* X, int64_t N, int D, const int32_t* assign, int l,
                           double sigma, const int64_t* ys, int64_t ny, double* out)
{
    if (!X || N < 1 || D < 1 || !assign || !(sigma > 0.0) || !ys || !out) return -1;
    for (int64_t i = 0; i < ny; ++i) {
        if (ys[i] < 0 || ys[i] >= N) return -1;
        double f = 0.0;
        for (int64_t p = 0; p < N; ++p)
            if (assign[p] == l) f += oracle_gauss(sqdist(X, D, p, ys[i]), sigma);
        out[i] = f;
    }
    return 0;
}

/* ------------------------------------------------------------------ K-means++ seeds */

/* K-means++ seeding (Section 4.2 takes its initial seeds from Arthur and
 * Vassilvitskii's K-means++): seed 0 is the given point `first`; seed i is
 * drawn with probability proportional to D(x)^2, the squared distance to the
 * closest seed so far.  The draw is made with the given uniform u[i-1] in
 * [0, 1): r = u[i-1] * sum_p D(x_p)^2, and the seed is the first p whose
 * running sum D(x_0)^2 + ... + D(x_p)^2 exceeds r (the last point if none
 * does).  When every D(x)^2 is zero the seed is point floor(u[i-1] N). */
int oracle_kmeanspp(const float* X, int64_t N, int D, int L, int32_t first, const double* u,
                    int32_t* seeds)
{
    if (!X || N < 1 || D < 1 || L < 1 || L > N || first < 0 || first >= N || (L > 1 && !u) || !seeds)
        return -1;
    double* closest = (double*)malloc(sizeof(double) * (size_t)N);
    if (!closest) return -2;
    for (int64_t p = 0; p < N; ++p) closest[p] = INFINITY;
    seeds[0] = first;
    for (int i = 1; i < L; ++i) {
        int64_t c = seeds[i - 1];
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < N; ++p) {
            double d = sqdist(X, D, p, c);
            if (d < closest[p]) closest[p] = d;
        }
        double total = 0.0;
        for (int64_t p = 0; p < N; ++p) total += closest[p];
        int64_t pick = N - 1;
        if (total > 0.0) {
            double r = u[i - 1] * total, run = 0.0;
            for (int64_t p = 0; p < N; ++p) {
                run += closest[p];
                if (run > r) { pick = p; break; }
            }
        } else {
            pick = (int64_t)(u[i - 1] * (double)N);
            if (pick > N - 1) pick = N - 1;
        }
        seeds[i] = (int32_t)pick;
    }
    free(closest);
    return 0;
}

/* ------------------------------------------------------------------ symmetric affinity */

/* The symmetric affinity K' = (K + K^t) / 2 of a sparse K (Prop. 1 assumes a
 * symmetric, psd K; the kNN affinity of Section 4.2 is directed).  Row p of
 * K' holds the union of row p of K and column p of K, by increasing column,
 * with K'_pq = (K_pq + K_qp) / 2, a missing entry counting 0 (w = NULL: K is
 * binary).  Two passes: out_row_ptr[N + 1] first (out_col / out_w may be
 * NULL), then the entries (out_cap >= out_row_ptr[N]). */
static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

int oracle_symmetrize(const int64_t* row_ptr, const int32_t* col_idx, const double* w, int64_t N,
                      int64_t* out_row_ptr, int32_t* out_col, double* out_w, int64_t out_cap)
{
    if (!row_ptr || !col_idx || N < 1 || !out_row_ptr) return -1;
    int64_t nnz = row_ptr[N];
    for (int64_t e = 0; e < nnz; ++e)
        if (col_idx[e] < 0 || col_idx[e] >= N) return -1;
    /* column p of K: the rows q with an entry (q, p), by increasing q */
    int64_t* cnt = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    int64_t* tq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    double* tw = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t* fill = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    /* per row: (column, weight) pairs before the merge */
    int64_t* keys = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? 2 * nnz : 1));
    if (!cnt || !tq || !tw || !fill || !keys) {
        free(cnt); free(tq); free(tw); free(fill); free(keys);
        return -2;
    }
    for (int64_t e = 0; e < nnz; ++e) cnt[col_idx[e] + 1]++;
    for (int64_t p = 0; p < N; ++p) cnt[p + 1] += cnt[p];
    for (int64_t q = 0; q < N; ++q)
        for (int64_t e = row_ptr[q]; e < row_ptr[q + 1]; ++e) {
            int64_t p = col_idx[e];
            int64_t slot = cnt[p] + fill[p]++;
            tq[slot] = q;
            tw[slot] = w ? w[e] : 1.0;
        }
    int rc = 0;
    out_row_ptr[0] = 0;
    for (int64_t p = 0; p < N; ++p) {
        /* candidate columns: row p of K and column p of K, sorted, duplicates once */
        int64_t m = 0;
        for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) keys[m++] = col_idx[e];
        for (int64_t t = cnt[p]; t < cnt[p + 1]; ++t) keys[m++] = tq[t];
        qsort(keys, (size_t)m, sizeof(int64_t), cmp_i64);
        int64_t u = 0;
        for (int64_t i = 0; i < m; ++i)
            if (i == 0 || keys[i] != keys[i - 1]) keys[u++] = keys[i];
        out_row_ptr[p + 1] = out_row_ptr[p] + u;
        if (!out_col) continue;
        if (out_row_ptr[p + 1] > out_cap) { rc = -1; break; }
        for (int64_t i = 0; i < u; ++i) {
            int64_t q = keys[i];
            double kpq = 0.0, kqp = 0.0;
            for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e)
                if (col_idx[e] == q) kpq += w ? w[e] : 1.0;
            for (int64_t t = cnt[p]; t < cnt[p + 1]; ++t)
                if (tq[t] == q) kqp += tw[t];
            out_col[out_row_ptr[p] + i] = (int32_t)q;
            if (out_w) out_w[out_row_ptr[p] + i] = 0.5 * (kpq + kqp);
        }
    }
    free(cnt); free(tq); free(tw); free(fill); free(keys);
    return rc;
}
