// C-ABI entry points of include/slk.h: context management, argument checks,
// and the host drivers of Algorithm 1 (SLK-BO and SLK-MS).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "slk_internal.cuh"

// ---------------------------------------------------------------- helpers

slk_status set_err(slk_ctx* ctx, slk_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

slk_status cuda_err(slk_ctx* ctx, cudaError_t e, const char* where) {
    const slk_status st = (e == cudaErrorMemoryAllocation) ? SLK_ERR_OOM : SLK_ERR_CUDA;
    return set_err(ctx, st, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

slk_status ensure_ws(slk_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return SLK_OK;
    if (ctx->ws) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "workspace resize sync");
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    const size_t want = align_up(bytes + bytes / 8, 1 << 20);
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        ctx->ws = nullptr;
        cudaGetLastError();
        return set_err(ctx, SLK_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    ctx->ws_bytes = want;
    return SLK_OK;
}

static cudaEvent_t take_event(slk_ctx* ctx) {
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

PhaseScope::PhaseScope(slk_ctx* c, int ph) : ctx(c), phase(ph) {
    if (ctx->prof && (a = take_event(ctx)) != nullptr) cudaEventRecord(a, ctx->stream);
}

PhaseScope::~PhaseScope() {
    if (!a) return;
    cudaEvent_t b = take_event(ctx);
    if (!b) {
        ctx->pool.push_back(a);
        return;
    }
    cudaEventRecord(b, ctx->stream);
    ctx->recs.push_back({phase, a, b});
}

// Fold recorded event pairs into the totals (caller has synchronised).
static void fold_profile(slk_ctx* ctx) {
    for (auto& r : ctx->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ctx->prof_ms[r.phase] += ms;
            ctx->prof_calls[r.phase] += 1;
        } else {
            cudaGetLastError();
        }
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
}

namespace {

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(const slk_ctx* ctx) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != ctx->device) ok = (cudaSetDevice(ctx->device) == cudaSuccess);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

DevState* dstate(slk_ctx* ctx) { return static_cast<DevState*>(ctx->dev_small); }

slk_status sync_and_check(slk_ctx* ctx) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "stream synchronize");
    return SLK_OK;
}

// Copy the device status block to pinned host memory and wait for it.
slk_status read_state(slk_ctx* ctx, DevState* out) {
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->host_pin, ctx->dev_small, sizeof(DevState),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    slk_status r = sync_and_check(ctx);
    if (r != SLK_OK) return r;
    memcpy(out, ctx->host_pin, sizeof(DevState));
    return SLK_OK;
}

#define CHECK_ARG(cond, ...)                                                   \
    do {                                                                       \
        if (!(cond)) return set_err(ctx, SLK_ERR_INVALID_ARG, __VA_ARGS__);    \
    } while (0)

#define BEGIN_CALL(ctx_)                                                       \
    if (!(ctx_)) return SLK_ERR_INVALID_ARG;                                   \
    (ctx_)->err.clear();                                                       \
    DeviceGuard _guard(ctx_);                                                  \
    if (!_guard.ok) return set_err(ctx_, SLK_ERR_CUDA, "cannot select device %d", (ctx_)->device)

slk_status check_graph(slk_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx, int64_t N) {
    CHECK_ARG(row_ptr && col_idx, "row_ptr and col_idx must not be NULL");
    CHECK_ARG(N >= 1 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    return SLK_OK;
}

}  // namespace

// ---------------------------------------------------------------- context

extern "C" const char* slk_version(void) { return "slk-gb300 0.1 sm_103a"; }

extern "C" slk_status slk_create(slk_ctx** out, int device, void* stream) {
    if (!out) return SLK_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
        cudaGetLastError();
        return SLK_ERR_NO_DEVICE;
    }
    if (device < 0 || device >= count) return SLK_ERR_NO_DEVICE;
    slk_ctx* ctx = new (std::nothrow) slk_ctx();
    if (!ctx) return SLK_ERR_OOM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->coop_supported, cudaDevAttrCooperativeLaunch, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dev_small, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMemset(ctx->dev_small, 0, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->host_pin, sizeof(DevState) + 256);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->dev_small) cudaFree(ctx->dev_small);
        delete ctx;
        return (e == cudaErrorMemoryAllocation) ? SLK_ERR_OOM : SLK_ERR_NO_DEVICE;
    }
    *out = ctx;
    return SLK_OK;
}

extern "C" slk_status slk_destroy(slk_ctx* ctx) {
    if (!ctx) return SLK_OK;
    {
        DeviceGuard g(ctx);
        cudaStreamSynchronize(ctx->stream);
        for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : ctx->pool) cudaEventDestroy(e);
        for (auto e : ctx->aux_ev) cudaEventDestroy(e);
        for (auto a : ctx->aux) cudaStreamDestroy(a);
        if (ctx->ws) cudaFree(ctx->ws);
        if (ctx->dev_small) cudaFree(ctx->dev_small);
        if (ctx->host_pin) cudaFreeHost(ctx->host_pin);
    }
    delete ctx;
    return SLK_OK;
}

extern "C" slk_status slk_set_stream(slk_ctx* ctx, void* stream) {
    if (!ctx) return SLK_ERR_INVALID_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return SLK_OK;
}

extern "C" const char* slk_last_error(const slk_ctx* ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" slk_status slk_profile(slk_ctx* ctx, int32_t enable) {
    BEGIN_CALL(ctx);
    slk_status r = sync_and_check(ctx);
    if (r != SLK_OK) return r;
    fold_profile(ctx);
    if (enable) {
        for (int i = 0; i < SLK_PHASE_COUNT; ++i) { ctx->prof_ms[i] = 0.0; ctx->prof_calls[i] = 0; }
        ctx->launches = 0;
    }
    ctx->prof = enable != 0;
    return SLK_OK;
}

extern "C" slk_status slk_profile_read(slk_ctx* ctx, double* ms, int64_t* calls,
                                       int64_t* kernel_launches) {
    BEGIN_CALL(ctx);
    slk_status r = sync_and_check(ctx);
    if (r != SLK_OK) return r;
    fold_profile(ctx);
    for (int i = 0; i < SLK_PHASE_COUNT; ++i) {
        if (ms) ms[i] = ctx->prof_ms[i];
        if (calls) calls[i] = ctx->prof_calls[i];
    }
    if (kernel_launches) *kernel_launches = ctx->launches;
    return SLK_OK;
}

extern "C" void slk_default_params(slk_params* p) {
    if (!p) return;
    p->max_outer = 50;
    p->max_inner = 100;
    p->tol_inner = 1e-6f;
    p->sigma_rule = SLK_SIGMA_MEDIAN;
    p->affinity = SLK_AFFINITY_BINARY;
    p->knn_precision = SLK_KNN_FP32;
    p->refine_init = 0;
    p->reorder = -1;
    p->max_ms = 100;
    p->tol_ms = 1e-5f;
    p->tol_modes = 1e-3f;
    p->symmetrize = 0;
}

// ---------------------------------------------------------------- steps

extern "C" slk_status slk_knn_graph(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t k,
                                    int32_t affinity, int32_t precision, float sigma,
                                    int64_t* row_ptr, int32_t* col_idx, float* dist2, float* w,
                                    int64_t* fallback_rows) {
    BEGIN_CALL(ctx);
    CHECK_ARG(X && row_ptr && col_idx && dist2, "X, row_ptr, col_idx and dist2 must not be NULL");
    CHECK_ARG(N >= 2 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    CHECK_ARG(D >= 1, "D=%d must be >= 1", D);
    CHECK_ARG(k >= 1 && k <= SLK_MAX_K && k <= N - 1, "k=%d must be in [1, min(%d, N-1)]", k, SLK_MAX_K);
    CHECK_ARG(affinity == SLK_AFFINITY_BINARY || affinity == SLK_AFFINITY_HEAT, "bad affinity %d", affinity);
    CHECK_ARG(precision == SLK_KNN_FP32 || precision == SLK_KNN_BF16_RERANK, "bad precision %d", precision);
    CHECK_ARG(affinity != SLK_AFFINITY_HEAT || (w && sigma > 0.f), "HEAT needs w and sigma > 0");
    slk_status r = ensure_ws(ctx, knn_ws_bytes(ctx, N, D, k, precision));
    if (r != SLK_OK) return r;
    DevState* st = dstate(ctx);
    r = knn_graph_launch(ctx, X, N, D, k, precision, row_ptr, col_idx, dist2, ctx->ws, st);
    if (r != SLK_OK) return r;
    if (w) {
        if (affinity == SLK_AFFINITY_HEAT) {
            r = set_sigma_launch(ctx, sigma, st);
            if (r != SLK_OK) return r;
        }
        r = weights_launch(ctx, dist2, N * (int64_t)k, affinity, &st->sigma, w);
        if (r != SLK_OK) return r;
    }
    DevState hs;
    r = read_state(ctx, &hs);
    if (r != SLK_OK) return r;
    if (hs.knn_error)
        return set_err(ctx, SLK_ERR_TIMEOUT, "a wait of the tensor-core kNN pipeline timed out");
    if (fallback_rows) *fallback_rows = hs.fallback_count;
    return SLK_OK;
}

extern "C" slk_status slk_knn_stage_rows(slk_ctx* ctx, int64_t* rows) {
    BEGIN_CALL(ctx);
    CHECK_ARG(rows, "rows must not be NULL");
    DevState hs;
    const slk_status r = read_state(ctx, &hs);
    if (r != SLK_OK) return r;
    rows[0] = hs.fallback_count;
    rows[1] = ctx->knn_last_two_term ? hs.fallback2_count
                                     : (ctx->knn_last_bf16 ? hs.fallback_count : 0);
    rows[2] = ctx->knn_last_bf16 ? hs.fallback3_count : hs.fallback_count;
    return SLK_OK;
}

extern "C" slk_status slk_sigma(slk_ctx* ctx, const float* dist2, int64_t n, int32_t rule,
                                float* sigma_out) {
    BEGIN_CALL(ctx);
    CHECK_ARG(dist2 && sigma_out, "dist2 and sigma_out must not be NULL");
    CHECK_ARG(n >= 1, "n=%lld must be >= 1", (long long)n);
    CHECK_ARG(rule == SLK_SIGMA_MEDIAN || rule == SLK_SIGMA_MEANSQ, "bad rule %d", rule);
    DevState* st = dstate(ctx);
    slk_status r = sigma_launch(ctx, dist2, n, rule, st);
    if (r != SLK_OK) return r;
    DevState hs;
    r = read_state(ctx, &hs);
    if (r != SLK_OK) return r;
    *sigma_out = hs.sigma;
    return SLK_OK;
}

extern "C" slk_status slk_unary(slk_ctx* ctx, const float* X, int64_t N, int32_t D,
                                const int32_t* mode_idx, int32_t L, float sigma, float* A,
                                float* Z0) {
    BEGIN_CALL(ctx);
    CHECK_ARG(X && mode_idx && A, "X, mode_idx and A must not be NULL");
    CHECK_ARG(N >= 1 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    CHECK_ARG(D >= 1, "D=%d must be >= 1", D);
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L && L <= N, "L=%d must be in [1, min(%d, N)]", L, SLK_MAX_L);
    CHECK_ARG(sigma > 0.f, "sigma must be > 0");
    DevState* st = dstate(ctx);
    slk_status r = set_sigma_launch(ctx, sigma, st);
    if (r != SLK_OK) return r;
    return unary_launch(ctx, X, N, D, mode_idx, L, &st->sigma, A, Z0);
}

extern "C" slk_status slk_bound_iterate(slk_ctx* ctx, const float* A, const int64_t* row_ptr,
                                        const int32_t* col_idx, const float* w, int64_t N,
                                        int32_t L, float lambda, float* Z, float* Z_prev,
                                        int32_t max_iters, float tol, int32_t* iters_done,
                                        float* last_delta) {
    BEGIN_CALL(ctx);
    CHECK_ARG(A && Z && Z_prev, "A, Z and Z_prev must not be NULL");
    CHECK_ARG(Z != Z_prev, "Z and Z_prev must be distinct buffers");
    slk_status r = check_graph(ctx, row_ptr, col_idx, N);
    if (r != SLK_OK) return r;
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L, "L=%d must be in [1, %d]", L, SLK_MAX_L);
    CHECK_ARG(max_iters >= 0, "max_iters must be >= 0");
    DevState* st = dstate(ctx);
    // a kNN-shaped graph (every row the same degree) takes the kernels that
    // know the degree: cached operands, or the staged pipeline at large N
    int kdeg = 0;
    r = uniform_degree(ctx, row_ptr, N, st, &kdeg);
    if (r != SLK_OK) return r;
    r = bound_launch(ctx, A, row_ptr, col_idx, w, N, L, lambda, Z, Z_prev, max_iters, tol, st, kdeg);
    if (r != SLK_OK) return r;
    DevState hs;
    r = read_state(ctx, &hs);
    if (r != SLK_OK) return r;
    if (hs.error & ERR_BARRIER_TIMEOUT)
        return set_err(ctx, SLK_ERR_TIMEOUT, "device-wide barrier of the bound kernel timed out");
    if (iters_done) *iters_done = hs.iters_done;
    if (last_delta) *last_delta = hs.last_delta;
    return SLK_OK;
}

extern "C" slk_status slk_barrier_selftest(slk_ctx* ctx, int32_t timeout_ms) {
    BEGIN_CALL(ctx);
    CHECK_ARG(timeout_ms >= 1 && timeout_ms <= 2000, "timeout_ms=%d must be in [1, 2000]", timeout_ms);
    DevState* st = dstate(ctx);
    slk_status r = barrier_probe_launch(ctx, st, (unsigned long long)timeout_ms * 1000000ull);
    if (r != SLK_OK) return r;
    DevState hs;
    r = read_state(ctx, &hs);
    if (r != SLK_OK) return r;
    if (hs.error & ERR_BARRIER_TIMEOUT)
        return set_err(ctx, SLK_ERR_TIMEOUT, "device-wide barrier of the bound kernel timed out");
    return set_err(ctx, SLK_ERR_CUDA, "the barrier wait did not give up");
}

extern "C" slk_status slk_mode_update(slk_ctx* ctx, const float* A, const float* Z_prev,
                                      const int64_t* row_ptr, const int32_t* col_idx,
                                      const float* w, int64_t N, int32_t L, float lambda,
                                      int32_t* mode_idx, int32_t* labels, float* mode_key,
                                      int32_t* changed) {
    BEGIN_CALL(ctx);
    CHECK_ARG(A && mode_idx, "A and mode_idx must not be NULL");
    if (Z_prev) {
        slk_status r = check_graph(ctx, row_ptr, col_idx, N);
        if (r != SLK_OK) return r;
    }
    CHECK_ARG(N >= 1 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L && L <= N, "L=%d must be in [1, min(%d, N)]", L, SLK_MAX_L);
    DevState* st = dstate(ctx);
    slk_status r = mode_launch(ctx, A, Z_prev, row_ptr, col_idx, w, N, L, lambda, mode_idx, labels,
                               mode_key, false, st);
    if (r != SLK_OK) return r;
    if (changed) {
        DevState hs;
        r = read_state(ctx, &hs);
        if (r != SLK_OK) return r;
        *changed = hs.changed;
    }
    return SLK_OK;
}

extern "C" slk_status slk_energy(slk_ctx* ctx, const float* X, int32_t D, const int32_t* labels,
                                 const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                                 int64_t N, int32_t L, const int32_t* mode_idx, float sigma,
                                 float lambda, double* E) {
    BEGIN_CALL(ctx);
    CHECK_ARG(X && labels && mode_idx && E, "X, labels, mode_idx and E must not be NULL");
    slk_status r = check_graph(ctx, row_ptr, col_idx, N);
    if (r != SLK_OK) return r;
    CHECK_ARG(D >= 1, "D must be >= 1");
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L && L <= N, "L=%d must be in [1, min(%d, N)]", L, SLK_MAX_L);
    CHECK_ARG(sigma > 0.f, "sigma must be > 0");
    DevState* st = dstate(ctx);
    r = set_sigma_launch(ctx, sigma, st);
    if (r != SLK_OK) return r;
    r = energy_launch(ctx, X, D, labels, row_ptr, col_idx, w, N, L, mode_idx, &st->sigma, lambda, st);
    if (r != SLK_OK) return r;
    DevState hs;
    r = read_state(ctx, &hs);
    if (r != SLK_OK) return r;
    *E = hs.energy;
    return SLK_OK;
}

// ---------------------------------------------------------------- solve

namespace {

constexpr int64_t kReorderBytes = 64ll << 20;   // Z above this: sorted row order

bool use_reorder(const slk_params& p, int64_t N, int L) {
    if (p.symmetrize) return false;   // rows of variable degree stay in the given order
    return p.reorder > 0 || (p.reorder < 0 && N * (int64_t)L * 4 > kReorderBytes);
}

struct SolveBufs {
    void* init_ws;   // starting-mode scratch (refine_init), else NULL
    // sorted row order (reorder): permutation, problem copies, sort scratch
    int32_t* perm;
    int32_t* inv;
    float* Xp;
    float* Ap;
    float* Zc;
    int32_t* colp;
    float* wp;
    int32_t* labp;
    int32_t* modp;
    void* loc_ws;
    float* A;
    float* Zp;
    float* dist2;
    int64_t* row_ptr;
    int32_t* col_idx;
    float* w;
    float* mode_key;
    void* knn_ws;
    // symmetric affinity (symmetrize): CSR of (K + K^t) / 2 and its scratch
    int64_t* srow_ptr;
    int32_t* scol;
    float* sw;
    void* sym_ws;
};

size_t solve_ws_bytes(const slk_ctx* ctx, int64_t N, int D, int L, int k, const slk_params& p) {
    size_t b = 0;
    b += 2 * align_up(sizeof(float) * (size_t)N * L, 256);
    b += 3 * align_up(sizeof(float) * (size_t)N * k, 256);
    b += align_up(sizeof(int64_t) * (size_t)(N + 1), 256);
    b += align_up(sizeof(float) * (size_t)L, 256);
    b += knn_ws_bytes(ctx, N, D, k, p.knn_precision) + 512;
    if (p.refine_init) b += init_modes_ws_bytes(ctx, N, D, L) + 512;
    if (p.symmetrize)
        b += align_up(sizeof(int64_t) * (size_t)(N + 1), 256) +
             2 * align_up(sizeof(float) * (size_t)N * k * 2, 256) + symmetrize_ws_bytes(N, N * k) + 512;
    if (use_reorder(p, N, L))
        b += 3 * align_up(sizeof(int32_t) * (size_t)N, 256) + align_up(sizeof(float) * (size_t)N * D, 256) +
             2 * align_up(sizeof(float) * (size_t)N * L, 256) + 2 * align_up(sizeof(float) * (size_t)N * k, 256) +
             align_up(sizeof(int32_t) * L, 256) + locality_ws_bytes(N, L) + 2048;
    return b;
}

SolveBufs carve_solve(WsCarver& wc, const slk_ctx* ctx, int64_t N, int D, int L, int k,
                      const slk_params& p) {
    SolveBufs b{};
    b.A = wc.take<float>((size_t)N * L);
    b.Zp = wc.take<float>((size_t)N * L);
    b.dist2 = wc.take<float>((size_t)N * k);
    b.col_idx = wc.take<int32_t>((size_t)N * k);
    b.w = wc.take<float>((size_t)N * k);
    b.row_ptr = wc.take<int64_t>((size_t)N + 1);
    b.mode_key = wc.take<float>((size_t)L);
    b.knn_ws = wc.take<unsigned char>(knn_ws_bytes(ctx, N, D, k, p.knn_precision));
    b.init_ws = p.refine_init ? wc.take<unsigned char>(init_modes_ws_bytes(ctx, N, D, L)) : nullptr;
    if (p.symmetrize) {
        b.srow_ptr = wc.take<int64_t>((size_t)N + 1);
        b.scol = wc.take<int32_t>((size_t)N * k * 2);
        b.sw = wc.take<float>((size_t)N * k * 2);
        b.sym_ws = wc.take<unsigned char>(symmetrize_ws_bytes(N, N * k));
    }
    if (use_reorder(p, N, L)) {
        b.perm = wc.take<int32_t>(N);
        b.inv = wc.take<int32_t>(N);
        b.Xp = wc.take<float>((size_t)N * D);
        b.Ap = wc.take<float>((size_t)N * L);
        b.Zc = wc.take<float>((size_t)N * L);
        b.colp = wc.take<int32_t>((size_t)N * k);
        b.wp = wc.take<float>((size_t)N * k);
        b.labp = wc.take<int32_t>(N);
        b.modp = wc.take<int32_t>(L);
        b.loc_ws = wc.take<unsigned char>(locality_ws_bytes(N, L));
    }
    return b;
}

slk_status check_solve_args(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L, int32_t k,
                            const int32_t* init_modes, const slk_params& p, const void* Z,
                            const int32_t* labels, const int32_t* modes, bool host) {
    CHECK_ARG(X && init_modes && labels && modes && (Z || host), "required pointer is NULL");
    CHECK_ARG(N >= 2 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    CHECK_ARG(D >= 1, "D must be >= 1");
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L && L <= N, "L=%d must be in [1, min(%d, N)]", L, SLK_MAX_L);
    CHECK_ARG(k >= 1 && k <= SLK_MAX_K && k <= N - 1, "k=%d must be in [1, min(%d, N-1)]", k, SLK_MAX_K);
    CHECK_ARG(p.max_outer >= 1 && p.max_inner >= 1, "max_outer and max_inner must be >= 1");
    CHECK_ARG(p.sigma_rule == SLK_SIGMA_MEDIAN || p.sigma_rule == SLK_SIGMA_MEANSQ, "bad sigma_rule");
    CHECK_ARG(p.affinity == SLK_AFFINITY_BINARY || p.affinity == SLK_AFFINITY_HEAT, "bad affinity");
    CHECK_ARG(p.knn_precision == SLK_KNN_FP32 || p.knn_precision == SLK_KNN_BF16_RERANK,
              "bad knn_precision");
    CHECK_ARG(p.symmetrize == 0 || p.symmetrize == 1, "symmetrize must be 0 or 1");
    return SLK_OK;
}

// Algorithm 1 on device buffers; sb carved from the workspace.
slk_status solve_device(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L, int32_t k,
                        float lambda, float sigma, const int32_t* init_modes, const slk_params& p,
                        float* Z, int32_t* labels, int32_t* modes, slk_stats* stats,
                        const SolveBufs& b) {
    DevState* st = dstate(ctx);
    cudaStream_t s = ctx->stream;
    slk_status r = knn_graph_launch(ctx, X, N, D, k, p.knn_precision, b.row_ptr, b.col_idx, b.dist2,
                                    b.knn_ws, st);
    if (r != SLK_OK) return r;
    r = (sigma > 0.f) ? set_sigma_launch(ctx, sigma, st)
                      : sigma_launch(ctx, b.dist2, N * (int64_t)k, p.sigma_rule, st);
    if (r != SLK_OK) return r;
    const float* w = nullptr;
    if (p.affinity == SLK_AFFINITY_HEAT) {
        r = weights_launch(ctx, b.dist2, N * (int64_t)k, SLK_AFFINITY_HEAT, &st->sigma, b.w);
        if (r != SLK_OK) return r;
        w = b.w;
    }
    // the graph the z-updates, modes and energy use: the directed kNN graph
    // (k entries a row), or its symmetric form (K + K^t) / 2 (variable degree)
    const int64_t* rp_it = b.row_ptr;
    const int32_t* col_it = b.col_idx;
    int kdeg_it = k;
    if (p.symmetrize) {
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->sym_error, 0, sizeof(unsigned int), s));
        r = symmetrize_launch(ctx, b.row_ptr, b.col_idx, w, N, N * (int64_t)k, b.srow_ptr, b.scol,
                              b.sw, b.sym_ws, &st->sym_error);
        if (r != SLK_OK) return r;
        rp_it = b.srow_ptr;
        col_it = b.scol;
        w = b.sw;
        kdeg_it = 0;
    }
    if (p.refine_init) {
        r = init_modes_launch(ctx, X, N, D, init_modes, L, &st->sigma, modes, nullptr, nullptr,
                              b.init_ws, st);
        if (r != SLK_OK) return r;
    } else if (modes != init_modes) {
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(modes, init_modes, sizeof(int32_t) * L,
                                          cudaMemcpyDeviceToDevice, s));
    }
    // The iteration may run on the rows sorted by their nearest initial mode
    // (neighbours then sit close in memory and the z-update gathers hit L2).
    // Every row keeps its edge order and mode ties go to the smaller original
    // index, so the results are the same bits as in the given order.
    const bool reorder = use_reorder(p, N, L);
    const float* Xc = X;
    float* Ac = b.A;
    float* Zc = Z;
    const int32_t* colc = col_it;
    int32_t* labc = labels;
    int32_t* modc = modes;
    DevState hs;
    int outer = 0, inner_total = 0, converged = 0;
    for (outer = 0; outer < p.max_outer;) {
        r = unary_launch(ctx, Xc, N, D, modc, L, &st->sigma, Ac, Zc);
        if (r != SLK_OK) return r;
        if (reorder && outer == 0) {
            r = locality_perm_launch(ctx, b.A, N, L, b.perm, b.inv, b.loc_ws);
            if (r != SLK_OK) return r;
            r = permute_problem_launch(ctx, b.perm, b.inv, N, D, L, k, X, b.A, Z, b.col_idx, w, b.Xp,
                                       b.Ap, b.Zc, b.colp, b.wp);
            if (r != SLK_OK) return r;
            r = map_modes_launch(ctx, b.inv, modes, L, b.modp);
            if (r != SLK_OK) return r;
            Xc = b.Xp;
            Ac = b.Ap;
            Zc = b.Zc;
            colc = b.colp;
            if (w) w = b.wp;
            labc = b.labp;
            modc = b.modp;
        }
        r = bound_launch(ctx, Ac, rp_it, colc, w, N, L, lambda, Zc, b.Zp, p.max_inner,
                         p.tol_inner, st, kdeg_it);
        if (r != SLK_OK) return r;
        r = mode_launch(ctx, Ac, b.Zp, rp_it, colc, w, N, L, lambda, modc, labc, b.mode_key,
                        true, st, reorder ? b.perm : nullptr, reorder ? b.inv : nullptr);
        if (r != SLK_OK) return r;
        r = energy_launch(ctx, Xc, D, labc, rp_it, colc, w, N, L, modc, &st->sigma, lambda, st);
        if (r != SLK_OK) return r;
        r = read_state(ctx, &hs);
        if (r != SLK_OK) return r;
        if (hs.error & ERR_BARRIER_TIMEOUT)
            return set_err(ctx, SLK_ERR_TIMEOUT, "device-wide barrier of the bound kernel timed out");
        if (hs.knn_error)
            return set_err(ctx, SLK_ERR_TIMEOUT, "a wait of the tensor-core kNN pipeline timed out");
        ++outer;
        inner_total += hs.iters_done;
        if (!hs.changed) { converged = 1; break; }
    }
    if (reorder && outer > 0) {
        r = unpermute_launch(ctx, b.perm, N, L, Zc, labc, modc, Z, labels, modes);
        if (r != SLK_OK) return r;
        r = sync_and_check(ctx);
        if (r != SLK_OK) return r;
    }
    if (stats) {
        stats->outer_iters = outer;
        stats->inner_iters_total = inner_total;
        stats->converged = converged;
        stats->sigma = hs.sigma;
        stats->energy = hs.energy;
        stats->knn_fallback_rows = hs.fallback_count;
        stats->knn_float32_rows = ctx->knn_last_two_term ? hs.fallback2_count
                                  : (ctx->knn_last_bf16 ? hs.fallback_count : 0);
        stats->knn_exact_rows = p.knn_precision == SLK_KNN_BF16_RERANK ? hs.fallback3_count
                                                                      : hs.fallback_count;
    }
    return converged ? SLK_OK : SLK_NOT_CONVERGED;
}

}  // namespace

extern "C" slk_status slk_solve(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L,
                                int32_t k, float lambda, float sigma, const int32_t* init_modes,
                                const slk_params* params, float* Z, int32_t* labels,
                                int32_t* modes, slk_stats* stats) {
    BEGIN_CALL(ctx);
    slk_params p;
    if (params) p = *params; else slk_default_params(&p);
    slk_status r = check_solve_args(ctx, X, N, D, L, k, init_modes, p, Z, labels, modes, false);
    if (r != SLK_OK) return r;
    r = ensure_ws(ctx, solve_ws_bytes(ctx, N, D, L, k, p));
    if (r != SLK_OK) return r;
    WsCarver wc(ctx->ws);
    const SolveBufs b = carve_solve(wc, ctx, N, D, L, k, p);
    return solve_device(ctx, X, N, D, L, k, lambda, sigma, init_modes, p, Z, labels, modes, stats, b);
}

extern "C" slk_status slk_solve_host(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L,
                                     int32_t k, float lambda, float sigma,
                                     const int32_t* init_modes, const slk_params* params,
                                     float* Z, int32_t* labels, int32_t* modes, slk_stats* stats) {
    BEGIN_CALL(ctx);
    slk_params p;
    if (params) p = *params; else slk_default_params(&p);
    slk_status r = check_solve_args(ctx, X, N, D, L, k, init_modes, p, Z, labels, modes, true);
    if (r != SLK_OK) return r;
    size_t need = solve_ws_bytes(ctx, N, D, L, k, p);
    need += align_up(sizeof(float) * (size_t)N * D, 256) + align_up(sizeof(float) * (size_t)N * L, 256) +
            align_up(sizeof(int32_t) * (size_t)N, 256) + 2 * align_up(sizeof(int32_t) * (size_t)L, 256) + 1024;
    r = ensure_ws(ctx, need);
    if (r != SLK_OK) return r;
    WsCarver wc(ctx->ws);
    float* dX = wc.take<float>((size_t)N * D);
    float* dZ = wc.take<float>((size_t)N * L);
    int32_t* dlab = wc.take<int32_t>((size_t)N);
    int32_t* dinit = wc.take<int32_t>((size_t)L);
    int32_t* dmodes = wc.take<int32_t>((size_t)L);
    const SolveBufs b = carve_solve(wc, ctx, N, D, L, k, p);
    cudaStream_t s = ctx->stream;
    {
        PhaseScope ps(ctx, SLK_PHASE_TRANSFER);
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(dX, X, sizeof(float) * (size_t)N * D, cudaMemcpyHostToDevice, s));
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(dinit, init_modes, sizeof(int32_t) * L, cudaMemcpyHostToDevice, s));
    }
    const slk_status rs = solve_device(ctx, dX, N, D, L, k, lambda, sigma, dinit, p, dZ, dlab, dmodes,
                                       stats, b);
    if (rs != SLK_OK && rs != SLK_NOT_CONVERGED) return rs;
    {
        PhaseScope ps(ctx, SLK_PHASE_TRANSFER);
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(labels, dlab, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost, s));
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(modes, dmodes, sizeof(int32_t) * L, cudaMemcpyDeviceToHost, s));
        if (Z)
            SLK_CUDA_TRY(ctx, cudaMemcpyAsync(Z, dZ, sizeof(float) * (size_t)N * L, cudaMemcpyDeviceToHost, s));
    }
    r = sync_and_check(ctx);
    if (r != SLK_OK) return r;
    return rs;
}

// ---------------------------------------------------------------- SLK-MS

namespace {

// Scratch of the mean-shift mode update: status words, float64 modes (the
// iteration state and its value at the start of a call), log z.
struct MsBufs {
    MsStatus* ms;
    double* M64;
    double* M64_start;
    float* Mhi;     // M64 split into two floats for the unary term and the energy
    float* Mlo;
    float* LZ;
    void* ms_ws;
};

size_t ms_bufs_bytes(const slk_ctx* ctx, int64_t N, int D, int L) {
    return align_up(sizeof(MsStatus), 256) + 2 * align_up(sizeof(double) * (size_t)L * D, 256) +
           2 * align_up(sizeof(float) * (size_t)L * D, 256) +
           align_up(sizeof(float) * (size_t)N * L, 256) + ms_ws_bytes(ctx, N, D, L) + 1024;
}

MsBufs carve_ms(WsCarver& wc, const slk_ctx* ctx, int64_t N, int D, int L) {
    MsBufs b{};
    b.ms = wc.take<MsStatus>(1);
    b.M64 = wc.take<double>((size_t)L * D);
    b.M64_start = wc.take<double>((size_t)L * D);
    b.Mhi = wc.take<float>((size_t)L * D);
    b.Mlo = wc.take<float>((size_t)L * D);
    b.LZ = wc.take<float>((size_t)N * L);
    b.ms_ws = wc.take<unsigned char>(ms_ws_bytes(ctx, N, D, L));
    return b;
}

// Head of MsStatus (barrier words, counters, moves) next to the DevState copy.
struct MsHead {
    unsigned arrive, gen, error, stop;
    int iters_done;
    float last_shift;
    float moved;
};

slk_status read_state_ms(slk_ctx* ctx, DevState* out, const MsStatus* ms, MsHead* head) {
    char* hp = static_cast<char*>(ctx->host_pin);
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(hp, ctx->dev_small, sizeof(DevState), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(hp + sizeof(DevState), ms, sizeof(MsHead),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    slk_status r = sync_and_check(ctx);
    if (r != SLK_OK) return r;
    memcpy(out, hp, sizeof(DevState));
    memcpy(head, hp + sizeof(DevState), sizeof(MsHead));
    return SLK_OK;
}

slk_status ms_errors(slk_ctx* ctx, const DevState& hs, const MsHead& mh) {
    if (hs.error & ERR_BARRIER_TIMEOUT)
        return set_err(ctx, SLK_ERR_TIMEOUT, "device-wide barrier of the bound kernel timed out");
    if (hs.knn_error)
        return set_err(ctx, SLK_ERR_TIMEOUT, "a wait of the tensor-core kNN pipeline timed out");
    if (mh.error)
        return set_err(ctx, SLK_ERR_TIMEOUT, "a wait of the mean-shift kernel timed out (%u)", mh.error);
    return SLK_OK;
}

}  // namespace

extern "C" slk_status slk_unary_vec(slk_ctx* ctx, const float* X, int64_t N, int32_t D,
                                    const float* M, int32_t L, float sigma, float* A, float* Z0) {
    BEGIN_CALL(ctx);
    CHECK_ARG(X && M && A, "X, M and A must not be NULL");
    CHECK_ARG(N >= 1 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    CHECK_ARG(D >= 1, "D=%d must be >= 1", D);
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L, "L=%d must be in [1, %d]", L, SLK_MAX_L);
    CHECK_ARG(sigma > 0.f, "sigma must be > 0");
    DevState* st = dstate(ctx);
    slk_status r = set_sigma_launch(ctx, sigma, st);
    if (r != SLK_OK) return r;
    return unary_launch(ctx, X, N, D, nullptr, L, &st->sigma, A, Z0, M);
}

extern "C" slk_status slk_mean_shift(slk_ctx* ctx, const float* X, int32_t D, const float* A,
                                     const float* Z_prev, const int64_t* row_ptr,
                                     const int32_t* col_idx, const float* w, int64_t N, int32_t L,
                                     float lambda, float sigma, float* M, int32_t max_iters,
                                     float tol, int32_t* labels, int32_t* iters_done,
                                     float* last_shift) {
    BEGIN_CALL(ctx);
    CHECK_ARG(X && A && M, "X, A and M must not be NULL");
    if (Z_prev) {
        slk_status r = check_graph(ctx, row_ptr, col_idx, N);
        if (r != SLK_OK) return r;
    }
    CHECK_ARG(N >= 1 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    CHECK_ARG(D >= 1 && D <= SLK_MS_MAX_D, "D=%d must be in [1, %d]", D, SLK_MS_MAX_D);
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L, "L=%d must be in [1, %d]", L, SLK_MAX_L);
    CHECK_ARG(sigma > 0.f, "sigma must be > 0");
    CHECK_ARG(max_iters >= 0, "max_iters must be >= 0");
    slk_status r = ensure_ws(ctx, ms_bufs_bytes(ctx, N, D, L));
    if (r != SLK_OK) return r;
    WsCarver wc(ctx->ws);
    const MsBufs b = carve_ms(wc, ctx, N, D, L);
    DevState* st = dstate(ctx);
    r = set_sigma_launch(ctx, sigma, st);
    if (r != SLK_OK) return r;
    r = ms_widen_launch(ctx, M, (int64_t)L * D, b.M64);
    if (r != SLK_OK) return r;
    r = logz_launch(ctx, A, Z_prev, row_ptr, col_idx, w, N, L, lambda, labels, b.LZ, false, st);
    if (r != SLK_OK) return r;
    r = ms_launch(ctx, X, N, D, b.LZ, L, &st->sigma, b.M64, M, max_iters, tol, b.ms, b.ms_ws);
    if (r != SLK_OK) return r;
    DevState hs;
    MsHead mh;
    r = read_state_ms(ctx, &hs, b.ms, &mh);
    if (r != SLK_OK) return r;
    r = ms_errors(ctx, hs, mh);
    if (r != SLK_OK) return r;
    if (iters_done) *iters_done = mh.iters_done;
    if (last_shift) *last_shift = mh.last_shift;
    return SLK_OK;
}

extern "C" slk_status slk_energy_vec(slk_ctx* ctx, const float* X, int32_t D, const int32_t* labels,
                                     const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                                     int64_t N, int32_t L, const float* M, float sigma, float lambda,
                                     double* E) {
    BEGIN_CALL(ctx);
    CHECK_ARG(X && labels && M && E, "X, labels, M and E must not be NULL");
    slk_status r = check_graph(ctx, row_ptr, col_idx, N);
    if (r != SLK_OK) return r;
    CHECK_ARG(D >= 1, "D must be >= 1");
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L, "L=%d must be in [1, %d]", L, SLK_MAX_L);
    CHECK_ARG(sigma > 0.f, "sigma must be > 0");
    DevState* st = dstate(ctx);
    r = set_sigma_launch(ctx, sigma, st);
    if (r != SLK_OK) return r;
    r = energy_launch(ctx, X, D, labels, row_ptr, col_idx, w, N, L, nullptr, &st->sigma, lambda, st, M);
    if (r != SLK_OK) return r;
    DevState hs;
    r = read_state(ctx, &hs);
    if (r != SLK_OK) return r;
    *E = hs.energy;
    return SLK_OK;
}

extern "C" slk_status slk_solve_ms(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L,
                                   int32_t k, float lambda, float sigma, const int32_t* init_modes,
                                   const slk_params* params, float* Z, int32_t* labels, float* M,
                                   slk_stats* stats) {
    BEGIN_CALL(ctx);
    slk_params p;
    if (params) p = *params; else slk_default_params(&p);
    CHECK_ARG(M, "M must not be NULL");
    slk_status r = check_solve_args(ctx, X, N, D, L, k, init_modes, p, Z, labels, init_modes, false);
    if (r != SLK_OK) return r;
    CHECK_ARG(D <= SLK_MS_MAX_D, "D=%d must be <= %d", D, SLK_MS_MAX_D);
    CHECK_ARG(p.max_ms >= 1, "max_ms must be >= 1");
    r = ensure_ws(ctx, solve_ws_bytes(ctx, N, D, L, k, p) + ms_bufs_bytes(ctx, N, D, L) + 1024);
    if (r != SLK_OK) return r;
    WsCarver wc(ctx->ws);
    const SolveBufs b = carve_solve(wc, ctx, N, D, L, k, p);
    const MsBufs mb = carve_ms(wc, ctx, N, D, L);
    DevState* st = dstate(ctx);
    cudaStream_t s = ctx->stream;
    r = knn_graph_launch(ctx, X, N, D, k, p.knn_precision, b.row_ptr, b.col_idx, b.dist2, b.knn_ws, st);
    if (r != SLK_OK) return r;
    r = (sigma > 0.f) ? set_sigma_launch(ctx, sigma, st)
                      : sigma_launch(ctx, b.dist2, N * (int64_t)k, p.sigma_rule, st);
    if (r != SLK_OK) return r;
    const float* w = nullptr;
    if (p.affinity == SLK_AFFINITY_HEAT) {
        r = weights_launch(ctx, b.dist2, N * (int64_t)k, SLK_AFFINITY_HEAT, &st->sigma, b.w);
        if (r != SLK_OK) return r;
        w = b.w;
    }
    const int64_t* rp_it = b.row_ptr;
    const int32_t* col_it = b.col_idx;
    int kdeg_it = k;
    if (p.symmetrize) {
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->sym_error, 0, sizeof(unsigned int), s));
        r = symmetrize_launch(ctx, b.row_ptr, b.col_idx, w, N, N * (int64_t)k, b.srow_ptr, b.scol,
                              b.sw, b.sym_ws, &st->sym_error);
        if (r != SLK_OK) return r;
        rp_it = b.srow_ptr;
        col_it = b.scol;
        w = b.sw;
        kdeg_it = 0;
    }
    const int32_t* start = init_modes;
    if (p.refine_init) {
        int32_t* refined = wc.take<int32_t>(L);
        r = init_modes_launch(ctx, X, N, D, init_modes, L, &st->sigma, refined, nullptr, nullptr,
                              b.init_ws, st);
        if (r != SLK_OK) return r;
        start = refined;
    }
    r = ms_gather_launch(ctx, X, D, start, L, M, mb.M64);
    if (r != SLK_OK) return r;
    DevState hs;
    MsHead mh{};
    int outer = 0, inner_total = 0, ms_total = 0, converged = 0;
    for (outer = 0; outer < p.max_outer;) {
        r = ms_split_launch(ctx, mb.M64, (int64_t)L * D, mb.Mhi, mb.Mlo);
        if (r != SLK_OK) return r;
        r = unary_launch(ctx, X, N, D, nullptr, L, &st->sigma, b.A, Z, mb.Mhi, mb.Mlo);
        if (r != SLK_OK) return r;
        r = bound_launch(ctx, b.A, rp_it, col_it, w, N, L, lambda, Z, b.Zp, p.max_inner,
                         p.tol_inner, st, kdeg_it);
        if (r != SLK_OK) return r;
        r = logz_launch(ctx, b.A, b.Zp, rp_it, col_it, w, N, L, lambda, labels, mb.LZ, true, st);
        if (r != SLK_OK) return r;
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(mb.M64_start, mb.M64, sizeof(double) * (size_t)L * D,
                                          cudaMemcpyDeviceToDevice, s));
        r = ms_launch(ctx, X, N, D, mb.LZ, L, &st->sigma, mb.M64, M, p.max_ms, p.tol_ms, mb.ms,
                      mb.ms_ws);
        if (r != SLK_OK) return r;
        r = ms_moved_launch(ctx, mb.M64, mb.M64_start, D, L, mb.ms);
        if (r != SLK_OK) return r;
        r = ms_split_launch(ctx, mb.M64, (int64_t)L * D, mb.Mhi, mb.Mlo);
        if (r != SLK_OK) return r;
        r = energy_launch(ctx, X, D, labels, rp_it, col_it, w, N, L, nullptr, &st->sigma,
                          lambda, st, mb.Mhi, mb.Mlo);
        if (r != SLK_OK) return r;
        r = read_state_ms(ctx, &hs, mb.ms, &mh);
        if (r != SLK_OK) return r;
        r = ms_errors(ctx, hs, mh);
        if (r != SLK_OK) return r;
        ++outer;
        inner_total += hs.iters_done;
        ms_total += mh.iters_done;
        if (mh.moved <= p.tol_modes * hs.sigma) { converged = 1; break; }
    }
    if (stats) {
        stats->outer_iters = outer;
        stats->inner_iters_total = inner_total;
        stats->converged = converged;
        stats->sigma = hs.sigma;
        stats->energy = hs.energy;
        stats->knn_fallback_rows = hs.fallback_count;
        stats->knn_float32_rows = ctx->knn_last_two_term ? hs.fallback2_count
                                  : (ctx->knn_last_bf16 ? hs.fallback_count : 0);
        stats->knn_exact_rows = p.knn_precision == SLK_KNN_BF16_RERANK ? hs.fallback3_count
                                                                      : hs.fallback_count;
        stats->ms_iters_total = ms_total;
    }
    return converged ? SLK_OK : SLK_NOT_CONVERGED;
}

// ---------------------------------------------------------------- starting modes

extern "C" slk_status slk_symmetrize(slk_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx,
                                     const float* w, int64_t N, int64_t* out_row_ptr,
                                     int32_t* out_col, float* out_w, int64_t* out_nnz) {
    BEGIN_CALL(ctx);
    slk_status r = check_graph(ctx, row_ptr, col_idx, N);
    if (r != SLK_OK) return r;
    CHECK_ARG(out_row_ptr && out_col && out_w, "out_row_ptr, out_col and out_w must not be NULL");
    int64_t nnz = 0;
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(&nnz, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    r = sync_and_check(ctx);
    if (r != SLK_OK) return r;
    CHECK_ARG(nnz >= 0 && nnz <= (int64_t)0x3fffffff, "row_ptr[N]=%lld out of range", (long long)nnz);
    r = ensure_ws(ctx, symmetrize_ws_bytes(N, nnz));
    if (r != SLK_OK) return r;
    DevState* st = dstate(ctx);
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->sym_error, 0, sizeof(unsigned int), ctx->stream));
    r = symmetrize_launch(ctx, row_ptr, col_idx, w, N, nnz, out_row_ptr, out_col, out_w, ctx->ws,
                          &st->sym_error);
    if (r != SLK_OK) return r;
    DevState hs;
    r = read_state(ctx, &hs);
    if (r != SLK_OK) return r;
    CHECK_ARG(hs.sym_error == 0, "a row of the graph has more than %d entries", SLK_MAX_K);
    if (out_nnz) {
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(out_nnz, out_row_ptr + N, sizeof(int64_t),
                                          cudaMemcpyDeviceToHost, ctx->stream));
        return sync_and_check(ctx);
    }
    return SLK_OK;
}

extern "C" slk_status slk_kmeanspp(slk_ctx* ctx, const float* X, int64_t N, int32_t D, int32_t L,
                                   int32_t first, const double* u, int32_t* seeds) {
    BEGIN_CALL(ctx);
    CHECK_ARG(X && seeds, "X and seeds must not be NULL");
    CHECK_ARG(N >= 1 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    CHECK_ARG(D >= 1, "D=%d must be >= 1", D);
    CHECK_ARG(L >= 1 && L <= N, "L=%d must be in [1, N]", L);
    CHECK_ARG(first >= 0 && first < N, "first=%d must be a point index", first);
    CHECK_ARG(L == 1 || u, "u must not be NULL when L > 1");
    for (int i = 0; i + 1 < L; ++i)
        CHECK_ARG(u[i] >= 0.0 && u[i] < 1.0, "u[%d] must lie in [0, 1)", i);
    slk_status r = ensure_ws(ctx, kmeanspp_ws_bytes(N, L));
    if (r != SLK_OK) return r;
    r = kmeanspp_launch(ctx, X, N, D, L, first, u, seeds, ctx->ws);
    if (r != SLK_OK) return r;
    // the draws are read from host memory by an asynchronous copy
    return sync_and_check(ctx);
}

extern "C" slk_status slk_initial_modes(slk_ctx* ctx, const float* X, int64_t N, int32_t D,
                                        const int32_t* seeds, int32_t L, float sigma,
                                        int32_t* modes, int32_t* assign, double* density,
                                        int64_t* candidates) {
    BEGIN_CALL(ctx);
    CHECK_ARG(X && seeds && modes, "X, seeds and modes must not be NULL");
    CHECK_ARG(N >= 1 && N < (int64_t)0x7fffffff, "N=%lld out of range", (long long)N);
    CHECK_ARG(D >= 1, "D=%d must be >= 1", D);
    CHECK_ARG(L >= 1 && L <= SLK_MAX_L && L <= N, "L=%d must be in [1, min(%d, N)]", L, SLK_MAX_L);
    CHECK_ARG(sigma > 0.f, "sigma must be > 0");
    const size_t need = init_modes_ws_bytes(ctx, N, D, L) + align_up(sizeof(double) * L, 256) + 512;
    slk_status r = ensure_ws(ctx, need);
    if (r != SLK_OK) return r;
    WsCarver wc(ctx->ws);
    double* ddens = wc.take<double>(L);
    void* iws = wc.take<unsigned char>(init_modes_ws_bytes(ctx, N, D, L));
    DevState* st = dstate(ctx);
    r = set_sigma_launch(ctx, sigma, st);
    if (r != SLK_OK) return r;
    r = init_modes_launch(ctx, X, N, D, seeds, L, &st->sigma, modes, assign, ddens, iws, st);
    if (r != SLK_OK) return r;
    if (density)
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(density, ddens, sizeof(double) * L, cudaMemcpyDeviceToHost,
                                          ctx->stream));
    if (candidates) *candidates = ctx->init_candidates;
    return sync_and_check(ctx);
}
