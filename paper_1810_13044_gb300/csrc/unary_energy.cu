// Unary term, kNN-edge weights and the discrete energy.
//
// Unary, Eq. (general-second) with the Gaussian kernel of Section 4.2:
//   a_{p,l} = exp(-||x_p - m_l||^2 / (2 sigma^2)),  z_p^0 = softmax(a_p) (Algorithm 1),
// m_l = x_{modes[l]} (SLK-BO) or a row of the mode vectors M (SLK-MS).
// Energy, Eq. (1) at one-hot z:
//   E = -sum_p k(x_p, m_{l_p}) + (lambda/2) sum_p sum_{e in row p} w_e ||z_p - z_q||^2.
#include <math.h>

#include "slk_internal.cuh"

namespace {

constexpr int kUPG = 128;      // points per point group (4 per lane)
constexpr int kUDC = 32;       // feature chunk staged in shared memory (float32 partial sums)
constexpr int kUThreads = 256;

// Row stride of the staged mode values: 4 G rounded up to 4 x odd, so that
// 16-byte rows stay aligned and the staging stores are at most 4-way
// bank-conflicted.
__host__ __device__ inline int unary_mode_stride(int G) { return 4 * (G | 1); }

// 4-byte asynchronous global -> shared copy; n = 0 fills the word with zero
// (the source is then not read).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int n) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Thread tile: 4 points (lane + 32 i) x 4 labels.  A warp covers one point
// group of 128 and one label group of 4; a block holds PG point groups and G
// label groups (G PG warps), and loops over passes of 4 G labels.  Features
// go in chunks of 32: X staged [point][33] (conflict-free per point), the
// pass's mode values [feature][S] (S = 4 x odd: one 16-byte broadcast per
// label group), two buffers filled by asynchronous copies so that the next
// chunk (of this pass or the next) loads while this one is summed.  Each
// pair's squared differences over a chunk are summed in float32 in feature
// order; the chunk sums are added as an unevaluated pair of floats (2Sum:
// about as accurate as a float64 sum and off the slow float64 pipe).  Vector
// modes (SLK-MS) come as M (float32) or as a float64 state split into
// M + Mlo: (x - m_hi) - m_lo keeps the difference accurate to float32
// relative to itself, not to |m|.  Z0's softmax rows are read back from A
// once the block has written it.
__global__ void __launch_bounds__(kUThreads, 2)
unary_kernel(const float* __restrict__ X, int64_t N, int D, const int32_t* __restrict__ modes,
             const float* __restrict__ M, const float* __restrict__ Mlo, int L, int G, int PG,
             const float* __restrict__ sigma_dev, float* __restrict__ A, float* __restrict__ Z0) {
    constexpr int PPL = kUPG / 32;   // points per lane
    extern __shared__ __align__(16) float sm[];
    const int S = unary_mode_stride(G), npts = PG * kUPG;
    const int nthr = blockDim.x;
    const size_t xbuf = (size_t)npts * (kUDC + 1), mbuf = (size_t)kUDC * S;
    float* xs = sm;                                    // 2 x [npts][kUDC + 1]
    float* mh = xs + 2 * xbuf;                         // 2 x [kUDC][S]
    float* mlo = mh + 2 * mbuf;                        // 2 x [kUDC][S] (Mlo only)
    __shared__ int mrow[SLK_MAX_L];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int g = warp % G, pg = warp / G;
    const int64_t p0 = (int64_t)blockIdx.x * npts;
    if (M == nullptr)
        for (int l = t; l < L; l += nthr) mrow[l] = modes[l];
    __syncthreads();
    const float sg = *sigma_dev;
    const float inv2s2 = 1.0f / (2.0f * sg * sg);
    const int nch = (D + kUDC - 1) / kUDC;
    const int nsteps = ((L + 4 * G - 1) / (4 * G)) * nch;   // (pass, chunk) pairs
    // Step s: pass s / nch (labels l0 = 4 G (s / nch) ..), chunk s % nch, buffer s & 1.
    auto stage = [&](int s) {
        const int d0 = (s % nch) * kUDC, l0 = (s / nch) * 4 * G, b = s & 1;
        const int dc = min(kUDC, D - d0);
        float* xb = xs + b * xbuf;
        for (int i = t; i < npts * kUDC; i += nthr) {
            const int r = i / kUDC, c = i % kUDC;
            const int64_t p = p0 + r;
            const bool ok = p < N && c < dc;
            cp_async4(xb + r * (kUDC + 1) + c, ok ? X + p * D + d0 + c : X, ok ? 4 : 0);
        }
        float* hb = mh + b * mbuf;
        float* lb = mlo + b * mbuf;
        for (int i = t; i < 4 * G * kUDC; i += nthr) {
            const int r = i / kUDC, c = i % kUDC;   // label l0 + r, feature d0 + c
            const int l = l0 + r;
            const bool ok = l < L && c < dc;
            const float* src = !ok ? X : M ? M + (int64_t)l * D + d0 + c
                                          : X + (int64_t)mrow[l] * D + d0 + c;
            cp_async4(hb + c * S + r, src, ok ? 4 : 0);
            if (Mlo) cp_async4(lb + c * S + r, ok ? Mlo + (int64_t)l * D + d0 + c : Mlo, ok ? 4 : 0);
        }
        cp_async_commit();
    };
    stage(0);
    float hi[PPL][4], lo[PPL][4];   // chunk sums added as an unevaluated float pair (2Sum)
    for (int s = 0; s < nsteps; ++s) {
        const int k = s % nch, l0 = (s / nch) * 4 * G, b = s & 1;
        const int dc = min(kUDC, D - k * kUDC);
        if (k == 0) {
#pragma unroll
            for (int i = 0; i < PPL; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    hi[i][j] = 0.f;
                    lo[i][j] = 0.f;
                }
        }
        if (s + 1 < nsteps) stage(s + 1);
        else cp_async_commit();          // an empty group keeps the wait count uniform
        cp_async_wait1();                // this thread's copies of step s have landed
        __syncthreads();                 // ... and every thread's
        const float* xrow = xs + b * xbuf + (size_t)(pg * kUPG + lane) * (kUDC + 1);
        const float* hb = mh + b * mbuf + 4 * g;
        const float* lb = mlo + b * mbuf + 4 * g;
        float part[PPL][4];
#pragma unroll
        for (int i = 0; i < PPL; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
        for (int c = 0; c < dc; ++c) {
            float x[PPL];
#pragma unroll
            for (int i = 0; i < PPL; ++i) x[i] = xrow[32 * i * (kUDC + 1) + c];
            const float4 h4 = *reinterpret_cast<const float4*>(hb + c * S);
            const float m[4] = {h4.x, h4.y, h4.z, h4.w};
            float ml[4] = {0.f, 0.f, 0.f, 0.f};
            if (Mlo) {
                const float4 l4 = *reinterpret_cast<const float4*>(lb + c * S);
                ml[0] = l4.x; ml[1] = l4.y; ml[2] = l4.z; ml[3] = l4.w;
            }
#pragma unroll
            for (int i = 0; i < PPL; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float df = x[i] - m[j];
                    if (Mlo) df -= ml[j];
                    part[i][j] = fmaf(df, df, part[i][j]);
                }
        }
#pragma unroll
        for (int i = 0; i < PPL; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // 2Sum (Knuth): s + e == hi + part exactly
                const float sum = __fadd_rn(hi[i][j], part[i][j]);
                const float bb = __fsub_rn(sum, hi[i][j]);
                const float e = __fadd_rn(__fsub_rn(hi[i][j], __fsub_rn(sum, bb)),
                                          __fsub_rn(part[i][j], bb));
                lo[i][j] = __fadd_rn(lo[i][j], e);
                hi[i][j] = sum;
            }
        if (k == nch - 1) {
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                const int64_t p = p0 + pg * kUPG + lane + 32 * i;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int l = l0 + 4 * g + j;
                    if (p < N && l < L) A[p * L + l] = expf(-__fadd_rn(hi[i][j], lo[i][j]) * inv2s2);
                }
            }
        }
        __syncthreads();                 // buffer b is free for step s + 2
    }
    if (Z0 == nullptr) return;
    for (int r = t; r < npts; r += nthr) {   // the block's rows of A are written (last barrier)
        if (p0 + r >= N) break;
        const float* ar = A + (p0 + r) * L;
        float m = ar[0];
        for (int l = 1; l < L; ++l) m = fmaxf(m, ar[l]);
        float s = 0.f;
        for (int l = 0; l < L; ++l) s += expf(ar[l] - m);
        float* zr = Z0 + (p0 + r) * L;
        for (int l = 0; l < L; ++l) zr[l] = expf(ar[l] - m) / s;
    }
}

__global__ void weights_kernel(const float* __restrict__ dist2, int64_t nnz, int heat,
                               const float* __restrict__ sigma_dev, float* __restrict__ w) {
    const float sg = heat ? *sigma_dev : 1.f;
    const float inv2s2 = 1.0f / (2.0f * sg * sg);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        w[e] = heat ? expf(-dist2[e] * inv2s2) : 1.f;
}

__global__ void set_sigma_kernel(float sigma, DevState* st) { st->sigma = sigma; }

// One warp per point: squared distance to its mode (warp_sq_dist) and the
// cut edges of its row (weights summed as float pairs).  Lane i keeps the
// distance and cut of the warp's points i, i + 32, ... until it has to add
// them, so that the float64 kernel value exp(-d2 / (2 sigma^2)) is one
// warp-wide instruction sequence per 32 points rather than one single-lane
// sequence per point.  V4: 16-byte row loads (warp_sq_dist4).
template <bool V4>
__global__ void __launch_bounds__(256, 4)
energy_kernel(const float* __restrict__ X, int D, const int32_t* __restrict__ labels,
              const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
              const float* __restrict__ w, int64_t N, const int32_t* __restrict__ modes,
              const float* __restrict__ M, const float* __restrict__ Mlo,
              const float* __restrict__ sigma_dev, float lambda, DevState* st) {
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double sg = (double)*sigma_dev;
    const double inv2s2 = 1.0 / (2.0 * sg * sg);
    double acc = 0.0;  // per-lane partial of E
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    double my_d2 = 0.0, my_cut = 0.0;
    bool mine = false;
    int slot = 0;   // lane that keeps the current point
    for (int64_t p = (int64_t)blockIdx.x * 8 + warp; p < N; p += nwarps) {
        const int lp = labels[p];
        const float* xp = X + p * D;
        const float* xm = M ? M + (int64_t)lp * D : X + (int64_t)modes[lp] * D;
        const float* xl = Mlo ? Mlo + (int64_t)lp * D : nullptr;
        const double d2 = V4 ? warp_sq_dist4(xp, xm, xl, D, lane) : warp_sq_dist(xp, xm, xl, D, lane);
        float ch = 0.f, cl = 0.f;
        for (int64_t e = row_ptr[p] + lane; e < row_ptr[p + 1]; e += 32) {
            const int q = col_idx[e];
            if (labels[q] != lp) fpair_add(ch, cl, w ? w[e] : 1.f, 0.f);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            fpair_add(ch, cl, __shfl_xor_sync(0xffffffffu, ch, o), __shfl_xor_sync(0xffffffffu, cl, o));
        if (lane == slot) {
            my_d2 = d2;
            my_cut = (double)ch + (double)cl;
            mine = true;
        }
        if (++slot == 32) {
            // ||z_p - z_q||^2 = 2 for every cut edge
            if (mine) acc += -exp(-my_d2 * inv2s2) + 0.5 * (double)lambda * 2.0 * my_cut;
            mine = false;
            slot = 0;
        }
    }
    if (mine) acc += -exp(-my_d2 * inv2s2) + 0.5 * (double)lambda * 2.0 * my_cut;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += red[i];
        atomicAdd(&st->energy, s);
    }
}

}  // namespace

slk_status unary_launch(slk_ctx* ctx, const float* X, int64_t N, int D, const int32_t* modes,
                        int L, const float* sigma_dev, float* A, float* Z0, const float* M,
                        const float* Mlo) {
    PhaseScope ps(ctx, SLK_PHASE_UNARY);
    SLK_COUNT_LAUNCH(ctx, 1);
    // label groups of 4: up to 8 warps per pass, the passes balanced
    const int gtot = (L + 3) / 4;
    const int passes = (gtot + 7) / 8;
    const int G = (gtot + passes - 1) / passes;
    const int PG = G <= 2 ? 2 : 1;
    const size_t smem = 2 * sizeof(float) * ((size_t)PG * kUPG * (kUDC + 1) +
                                             (Mlo ? 2 : 1) * (size_t)kUDC * unary_mode_stride(G));
    SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(unary_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    const int64_t npts = (int64_t)PG * kUPG;
    const unsigned grid = (unsigned)((N + npts - 1) / npts);
    unary_kernel<<<grid, 32 * G * PG, smem, ctx->stream>>>(X, N, D, modes, M, Mlo, L, G, PG,
                                                            sigma_dev, A, Z0);
    SLK_LAUNCH_CHECK(ctx, "unary_kernel");
    return SLK_OK;
}

slk_status weights_launch(slk_ctx* ctx, const float* dist2, int64_t nnz, int affinity,
                          const float* sigma_dev, float* w) {
    SLK_COUNT_LAUNCH(ctx, 1);
    int64_t grid = (nnz + 255) / 256;
    if (grid > (int64_t)ctx->num_sms * 16) grid = (int64_t)ctx->num_sms * 16;
    if (grid < 1) grid = 1;
    weights_kernel<<<(unsigned)grid, 256, 0, ctx->stream>>>(
        dist2, nnz, affinity == SLK_AFFINITY_HEAT ? 1 : 0, sigma_dev, w);
    SLK_LAUNCH_CHECK(ctx, "weights_kernel");
    return SLK_OK;
}

slk_status set_sigma_launch(slk_ctx* ctx, float sigma, DevState* st) {
    SLK_COUNT_LAUNCH(ctx, 1);
    set_sigma_kernel<<<1, 1, 0, ctx->stream>>>(sigma, st);
    SLK_LAUNCH_CHECK(ctx, "set_sigma_kernel");
    return SLK_OK;
}

slk_status energy_launch(slk_ctx* ctx, const float* X, int D, const int32_t* labels,
                         const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                         int64_t N, int L, const int32_t* modes, const float* sigma_dev,
                         float lambda, DevState* st, const float* M, const float* Mlo) {
    (void)L;
    PhaseScope ps(ctx, SLK_PHASE_ENERGY);
    SLK_COUNT_LAUNCH(ctx, 1);
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->energy, 0, sizeof(double), ctx->stream));
    int64_t grid = (N + 7) / 8;   // one wave: 4 CTAs per SM (launch bounds)
    if (grid > (int64_t)ctx->num_sms * 4) grid = (int64_t)ctx->num_sms * 4;
    auto al16 = [](const float* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    const bool v4 = D % 4 == 0 && al16(X) && (M == nullptr || al16(M)) && (Mlo == nullptr || al16(Mlo));
    if (v4)
        energy_kernel<true><<<(unsigned)grid, 256, 0, ctx->stream>>>(
            X, D, labels, row_ptr, col_idx, w, N, modes, M, Mlo, sigma_dev, lambda, st);
    else
        energy_kernel<false><<<(unsigned)grid, 256, 0, ctx->stream>>>(
            X, D, labels, row_ptr, col_idx, w, N, modes, M, Mlo, sigma_dev, lambda, st);
    SLK_LAUNCH_CHECK(ctx, "energy_kernel");
    return SLK_OK;
}
