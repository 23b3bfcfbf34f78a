// Internal declarations shared by the CUDA translation units of the SLK
// library (never included by anything outside csrc/).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/slk.h"

// ---------------------------------------------------------------- context

struct slk_ctx {
    int device = 0;
    int num_sms = 0;
    int coop_supported = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // scratch workspace, grown on demand (cudaMalloc), freed by slk_destroy
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // small pinned host block for scalar results
    void* host_pin = nullptr;
    // small device block for scalar state (status words, sigma, energy)
    void* dev_small = nullptr;
    // phase profiling: recorded (phase, start, stop) event triples
    bool prof = false;
    long long launches = 0;
    struct Rec { int phase; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[SLK_PHASE_COUNT] = {};
    long long prof_calls[SLK_PHASE_COUNT] = {};
    // candidates recomputed exactly by the last starting-mode call
    long long init_candidates = 0;
    // the last kNN graph used bfloat16 candidates (its stage counters mean so)
    bool knn_last_bf16 = false;
    bool knn_last_two_term = false;   // ... and ran the two-term stage
    // auxiliary streams (batched graph building), created on first use
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_ev;
};

// Records start/stop events of one phase on the context stream (when
// profiling is enabled).
struct PhaseScope {
    slk_ctx* ctx;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseScope(slk_ctx* c, int ph);
    ~PhaseScope();
};

// Count kernel launches made by the library.
#define SLK_COUNT_LAUNCH(ctx, n) ((ctx)->launches += (n))

// Device-side status / scalar block (lives at ctx->dev_small).
struct DevState {
    unsigned int barrier_arrive;
    unsigned int barrier_gen;
    unsigned int error;          // bit 0: barrier timeout
    int iters_done;
    unsigned int delta_bits[3];  // float bits of max |dz| per update (ring of 3)
    float last_delta;
    int changed;
    float sigma;
    double energy;
    unsigned long long mode_best[SLK_MAX_L];  // packed (ordered key, ~index) per label
    // radix select state
    unsigned int sel_prefix;
    unsigned int sel_mask;
    unsigned long long sel_rank;
    unsigned int sel_hist[256];
    double sum_d2;
    long long fallback_count;
    unsigned int knn_max_norm_bits;   // float bits of max candidate-operand norm^2
    unsigned int knn_max_rho_bits;    // float bits of max rounding perturbation norm
    unsigned int knn_error;           // bit 1: a tensor-core pipeline wait timed out
    unsigned int knn_max_norm32_bits; // float bits of max float32-operand norm^2
    long long fallback2_count;        // rows left for the float32 stage after the two-term stage
    // one-launch median: grid barrier words, count of values <= the lower
    // middle order statistic, smallest value above it (bits)
    unsigned int sel_bar[4];
    unsigned long long sel_cnt;
    unsigned int sel_min_bits;
    unsigned int sym_error;           // bit 0: a row of the graph to symmetrise is too long
    unsigned int deg_mixed;           // 1: the rows of a CSR graph do not all have one degree
    unsigned int knn_max_norm_s_bits; // float bits of max two-term bfloat16 operand norm^2
    unsigned int knn_max_rho_s_bits;  // float bits of max two-term rounding perturbation norm
    unsigned int knn_max_kappa_bits;  // float bits of max rho_p / ||v_p|| (candidate operand)
    unsigned int knn_max_kappa_s_bits;// float bits of max rho_s_p / ||v_p|| (two-term operand)
    long long fallback3_count;        // rows left for the exact scan after the float32 stage
    unsigned long long knn_sweep;     // tiles issued by the tensor-core kNN kernel (sweep alignment)
};

enum : unsigned int { ERR_BARRIER_TIMEOUT = 1u };

// ---------------------------------------------------------------- helpers

slk_status set_err(slk_ctx* ctx, slk_status st, const char* fmt, ...);
slk_status cuda_err(slk_ctx* ctx, cudaError_t e, const char* where);
// Make sure ctx->ws holds at least `bytes`; returns SLK_OK or SLK_ERR_OOM.
slk_status ensure_ws(slk_ctx* ctx, size_t bytes);

#define SLK_CUDA_TRY(ctx, expr)                                                  \
    do {                                                                         \
        cudaError_t _e = (expr);                                                 \
        if (_e != cudaSuccess) return cuda_err((ctx), _e, #expr);                \
    } while (0)

#define SLK_LAUNCH_CHECK(ctx, name)                                              \
    do {                                                                         \
        cudaError_t _e = cudaGetLastError();                                     \
        if (_e != cudaSuccess) return cuda_err((ctx), _e, name);                 \
    } while (0)

static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over the workspace (256-byte aligned slices).
struct WsCarver {
    char* base;
    size_t off = 0;
    explicit WsCarver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

// Workspace needed by knn_graph_launch (bytes), and the launcher itself
// (device outputs only; no synchronisation).
size_t knn_ws_bytes(const slk_ctx* ctx, int64_t N, int D, int k, int precision);
slk_status knn_graph_launch(slk_ctx* ctx, const float* X, int64_t N, int D, int k,
                            int precision, int64_t* row_ptr, int32_t* col_idx, float* dist2,
                            void* ws, DevState* st);

// Centred float32 operand of the distance tiles: xt[p][j] = x_pj - mean_j
// (Np x Dp, zero padding), norms[p] = ||xt_p||^2, rho[p] = rounding norm.
slk_status knn_prep_fp32_launch(slk_ctx* ctx, const float* X, int64_t N, int D, int Dp, int64_t Np,
                                double* colsum, float* mu, float* xt, float* norms, float* rho,
                                DevState* st);

// Starting modes of Section 4.2 (nearest-seed assignment, then the mode
// definition of Eq. (1)): modes [L] device out, assign [N] device out
// (nullable), density [L] device float64 out (nullable); sigma from *sigma_dev.
size_t init_modes_ws_bytes(const slk_ctx* ctx, int64_t N, int D, int L);
slk_status init_modes_launch(slk_ctx* ctx, const float* X, int64_t N, int D, const int32_t* seeds,
                             int L, const float* sigma_dev, int32_t* modes, int32_t* assign,
                             double* density, void* ws, DevState* st);

// K' = (K + K^t) / 2 of a CSR graph whose rows hold at most SLK_MAX_K
// entries: out_row_ptr [N + 1], out_col / out_w [2 nnz at most].  A longer
// row sets bit 0 of *err.  Workspace: symmetrize_ws_bytes.
size_t symmetrize_ws_bytes(int64_t N, int64_t nnz);
slk_status symmetrize_launch(slk_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx,
                             const float* w, int64_t N, int64_t nnz, int64_t* out_row_ptr,
                             int32_t* out_col, float* out_w, void* ws, unsigned int* err);

// K-means++ seeds from the caller's draws (first, u_host [L - 1] host
// uniforms in [0, 1)) into seeds [L] (device); workspace kmeanspp_ws_bytes.
size_t kmeanspp_ws_bytes(int64_t N, int L);
slk_status kmeanspp_launch(slk_ctx* ctx, const float* X, int64_t N, int D, int L, int32_t first,
                           const double* u_host, int32_t* seeds, void* ws);

// weights w[e] = 1 (binary) or exp(-dist2[e] / (2 sigma^2)) with sigma read
// from *sigma_dev (heat).
slk_status weights_launch(slk_ctx* ctx, const float* dist2, int64_t nnz, int affinity,
                          const float* sigma_dev, float* w);

// sigma -> st->sigma (device); no synchronisation.
size_t sigma_ws_bytes(int64_t n);
slk_status sigma_launch(slk_ctx* ctx, const float* dist2, int64_t n, int rule, DevState* st);

// A and (optionally) Z0 from modes; sigma taken from *sigma_dev.  With M
// (L x D float32) the modes are those vectors and `modes` is ignored
// (SLK-MS); with Mlo as well, the modes are M + Mlo (a float64 state split
// into two floats by ms_split_launch).
slk_status unary_launch(slk_ctx* ctx, const float* X, int64_t N, int D, const int32_t* modes,
                        int L, const float* sigma_dev, float* A, float* Z0,
                        const float* M = nullptr, const float* Mlo = nullptr);

// Inner loop; the final iterate ends in Z, the previous one in Z_prev.
slk_status bound_launch(slk_ctx* ctx, const float* A, const int64_t* row_ptr,
                        const int32_t* col_idx, const float* w, int64_t N, int L, float lambda,
                        float* Z, float* Z_prev, int max_iters, float tol, DevState* st,
                        int kdeg = 0);   // kdeg > 0: every row has kdeg entries (row_ptr[p] = kdeg p)

// Degree shared by every row of a CSR graph (row_ptr[p] = k p), or 0 if the
// degrees differ or k > SLK_MAX_K.  Synchronises the stream.
slk_status uniform_degree(slk_ctx* ctx, const int64_t* row_ptr, int64_t N, DevState* st, int* kdeg);

// One block waits at the device-wide barrier of the persistent z-update
// kernels for a second block that is never launched; the wait gives up after
// timeout_ns and sets ERR_BARRIER_TIMEOUT in st->error.
slk_status barrier_probe_launch(slk_ctx* ctx, DevState* st, unsigned long long timeout_ns);

// Mode update (keys from A + lambda K Z_prev; Z_prev NULL or st->iters_done == 0
// when use_iters_flag: s = A).  Writes modes in place, labels, keys, st->changed.
// With orig (row -> original point index) mode ties go to the smaller
// original index, and inv (original -> row) maps the chosen points back to
// row indices: the result does not depend on the order of the rows.
slk_status mode_launch(slk_ctx* ctx, const float* A, const float* Z_prev,
                       const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                       int64_t N, int L, float lambda, int32_t* modes, int32_t* labels,
                       float* mode_key, bool use_iters_flag, DevState* st,
                       const int32_t* orig = nullptr, const int32_t* inv = nullptr);

// Row order for the z-updates (L2 locality): rows sorted by their argmax_l
// A[p][l] (a stable counting sort), perm[i] = original row of row i,
// inv[perm[i]] = i; then X, A, Z0 and the graph in that order.
size_t locality_ws_bytes(int64_t N, int L);
slk_status locality_perm_launch(slk_ctx* ctx, const float* A, int64_t N, int L, int32_t* perm,
                                int32_t* inv, void* ws);
slk_status permute_problem_launch(slk_ctx* ctx, const int32_t* perm, const int32_t* inv,
                                  int64_t N, int D, int L, int k, const float* X, const float* A,
                                  const float* Z0, const int32_t* col_idx, const float* w,
                                  float* Xp, float* Ap, float* Z0p, int32_t* colp, float* wp);
// out[l] = inv[modes[l]] (mode indices in the new row order).
slk_status map_modes_launch(slk_ctx* ctx, const int32_t* inv, const int32_t* modes, int L,
                            int32_t* out);
// Outputs back in the original order: Z[perm[i]] = Zp[i], labels likewise,
// modes[l] = perm[modes_p[l]].
slk_status unpermute_launch(slk_ctx* ctx, const int32_t* perm, int64_t N, int L, const float* Zp,
                            const int32_t* labels_p, const int32_t* modes_p, float* Z,
                            int32_t* labels, int32_t* modes);

// log z keys (N x L) and labels for the SLK-MS weights (logits as in mode_launch).
slk_status logz_launch(slk_ctx* ctx, const float* A, const float* Z_prev,
                       const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                       int64_t N, int L, float lambda, int32_t* labels, float* LZ,
                       bool use_iters_flag, const DevState* st);

// SLK-MS mode update, Eq. (mean-shift), with the assignments fixed (given as
// log z).  M64 (L x D float64, workspace) is the iteration state, in/out;
// M (L x D float32) receives the modes after every iteration.  Counters go
// to *ms (device).  Workspace: ms_ws_bytes.
struct MsStatus {
    unsigned arrive, gen, error;  // device-wide barrier words (error: bit 0 barrier, bit 1 copy timeout)
    unsigned stop;                // launch-per-phase path: the loop has stopped
    int iters_done;
    float last_shift;
    float moved;                  // max_l ||m_l after - m_l before|| of one call (ms_moved_launch)
    double shift2[3][SLK_MAX_L];
};
size_t ms_ws_bytes(const slk_ctx* ctx, int64_t N, int D, int L);
slk_status ms_launch(slk_ctx* ctx, const float* X, int64_t N, int D, const float* LZ, int L,
                     const float* sigma_dev, double* M64, float* M, int max_iters, float tol,
                     MsStatus* ms, void* ws);
// M[l] = X[idx[l]] (float32) and M64 = the same in float64.
slk_status ms_gather_launch(slk_ctx* ctx, const float* X, int D, const int32_t* idx, int L,
                            float* M, double* M64);
// M64 = (double) M.
slk_status ms_widen_launch(slk_ctx* ctx, const float* M, int64_t n, double* M64);
// Mhi = (float) M64, Mlo = (float) (M64 - Mhi).
slk_status ms_split_launch(slk_ctx* ctx, const double* M64, int64_t n, float* Mhi, float* Mlo);
// ms->moved = max_l ||M64[l] - M64_start[l]||_2.
slk_status ms_moved_launch(slk_ctx* ctx, const double* M64, const double* M64_start, int D, int L,
                           MsStatus* ms);

// Energy -> st->energy (device); sigma from *sigma_dev.  M / Mlo as in
// unary_launch.
slk_status energy_launch(slk_ctx* ctx, const float* X, int D, const int32_t* labels,
                         const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                         int64_t N, int L, const int32_t* modes, const float* sigma_dev,
                         float lambda, DevState* st, const float* M = nullptr,
                         const float* Mlo = nullptr);

// Set st->sigma from a host value (enqueued on the stream).
slk_status set_sigma_launch(slk_ctx* ctx, float sigma, DevState* st);

// ---------------------------------------------------------------- device helpers

#ifdef __CUDACC__
__device__ __forceinline__ unsigned int float_to_ordered(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
// (h, l) += (bh, bl) for unevaluated float pairs: 2Sum of the high parts
// (exact, and the same on both lanes of an xor-butterfly step), the low
// parts and the rounding error added to the low part.  A butterfly of such
// additions gives every lane the same pair, within a few u^2 of the exact sum.
__device__ __forceinline__ void fpair_add(float& h, float& l, float bh, float bl) {
    const float s = __fadd_rn(h, bh);
    const float bb = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    l = __fadd_rn(__fadd_rn(l, bl), e);
    h = s;
}
// Squared distance of two rows by the 32 lanes of a warp (lane-strided
// features; every lane returns the total): float32 differences, squares
// summed in float32 chunks of 8 per lane, chunks and lanes added as float
// pairs (as accurate as float64 here, off GB300's narrow float64 pipe).
// xl (nullable): low part of a float64 row split into xm + xl.
__device__ __forceinline__ double warp_sq_dist(const float* __restrict__ xp,
                                               const float* __restrict__ xm,
                                               const float* __restrict__ xl, int D, int lane) {
    float h = 0.f, lo = 0.f;
    // chunks of 8 lane-iterations (features lane + 32 i), their loads issued
    // together
    for (int j0 = lane; j0 < D; j0 += 256) {
        float a[8], b[8], c[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int j = j0 + 32 * t;
            a[t] = j < D ? xp[j] : 0.f;
            b[t] = j < D ? xm[j] : 0.f;
            c[t] = (xl && j < D) ? xl[j] : 0.f;
        }
        float part = 0.f;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (j0 + 32 * t < D) {
                float df = a[t] - b[t];
                if (xl) df -= c[t];
                part = fmaf(df, df, part);
            }
        }
        fpair_add(h, lo, part, 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        fpair_add(h, lo, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, lo, o));
    return (double)h + (double)lo;
}
// warp_sq_dist with 16-byte loads (D a multiple of 4, rows 16-byte aligned):
// a chunk covers 4 float4 per lane, one float32 accumulator per column of
// the lane's 4-column groups (at most 4 squares each, as accurate as the
// chunks of 8 above), the accumulators added as float pairs.
__device__ __forceinline__ double warp_sq_dist4(const float* __restrict__ xp,
                                                const float* __restrict__ xm,
                                                const float* __restrict__ xl, int D, int lane) {
    const int D4 = D >> 2;
    const float4* p4 = reinterpret_cast<const float4*>(xp);
    const float4* m4 = reinterpret_cast<const float4*>(xm);
    const float4* l4 = reinterpret_cast<const float4*>(xl);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float h = 0.f, lo = 0.f;
    for (int j0 = lane; j0 < D4; j0 += 128) {
        float4 a[4], b[4], c[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = j0 + 32 * t;
            a[t] = j < D4 ? p4[j] : z4;
            b[t] = j < D4 ? m4[j] : z4;
            c[t] = (xl && j < D4) ? l4[j] : z4;
        }
        float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float dx = a[t].x - b[t].x, dy = a[t].y - b[t].y, dz = a[t].z - b[t].z,
                  dw = a[t].w - b[t].w;
            if (xl) { dx -= c[t].x; dy -= c[t].y; dz -= c[t].z; dw -= c[t].w; }
            q0 = fmaf(dx, dx, q0);
            q1 = fmaf(dy, dy, q1);
            q2 = fmaf(dz, dz, q2);
            q3 = fmaf(dw, dw, q3);
        }
        fpair_add(h, lo, q0, 0.f);
        fpair_add(h, lo, q1, 0.f);
        fpair_add(h, lo, q2, 0.f);
        fpair_add(h, lo, q3, 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        fpair_add(h, lo, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, lo, o));
    return (double)h + (double)lo;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#endif
