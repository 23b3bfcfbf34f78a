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

constexpr int kUTP = 32;       // points per block
constexpr int kUDC = 32;       // feature chunk staged in shared memory
constexpr int kUThreads = 256;

// Block: 32 points x all L labels.  Thread t owns point t % 32 and labels
// t / 32 + 8 j.  X and mode rows are staged 32 features at a time; each
// chunk's squared differences are summed in float32, chunk sums in float64.
// Vector modes (SLK-MS) come as M (float32) or as a float64 state split into
// Mhi + Mlo (two floats): (x - m_hi) - m_lo keeps the difference accurate to
// float32 relative to itself, not to |m|.
template <int LPT>
__global__ void __launch_bounds__(kUThreads)
unary_kernel(const float* __restrict__ X, int64_t N, int D, const int32_t* __restrict__ modes,
             const float* __restrict__ M, const float* __restrict__ Mlo, int L,
             const float* __restrict__ sigma_dev, float* __restrict__ A, float* __restrict__ Z0) {
    extern __shared__ float sm[];
    float* xs = sm;                                  // [kUTP][kUDC + 1]
    float* ms = xs + kUTP * (kUDC + 1);              // [L][kUDC + 1]
    float* ml = ms + (size_t)L * (kUDC + 1);         // [L][kUDC + 1] (Mlo only)
    float* at = ml + (Mlo ? (size_t)L * (kUDC + 1) : 0);   // [kUTP][L]
    __shared__ int mrow[SLK_MAX_L];
    const int t = threadIdx.x;
    const int pl = t % kUTP, lb = t / kUTP;
    const int64_t p0 = (int64_t)blockIdx.x * kUTP;
    if (M == nullptr)
        for (int l = t; l < L; l += kUThreads) mrow[l] = modes[l];
    double acc[LPT];
#pragma unroll
    for (int j = 0; j < LPT; ++j) acc[j] = 0.0;
    __syncthreads();
    for (int d0 = 0; d0 < D; d0 += kUDC) {
        const int dc = min(kUDC, D - d0);
        for (int i = t; i < kUTP * kUDC; i += kUThreads) {
            const int r = i / kUDC, c = i % kUDC;
            const int64_t p = p0 + r;
            xs[r * (kUDC + 1) + c] = (p < N && c < dc) ? X[p * D + d0 + c] : 0.f;
        }
        for (int i = t; i < L * kUDC; i += kUThreads) {
            const int r = i / kUDC, c = i % kUDC;
            if (M) {
                ms[r * (kUDC + 1) + c] = (c < dc) ? M[(int64_t)r * D + d0 + c] : 0.f;
                if (Mlo) ml[r * (kUDC + 1) + c] = (c < dc) ? Mlo[(int64_t)r * D + d0 + c] : 0.f;
            } else {
                ms[r * (kUDC + 1) + c] = (c < dc) ? X[(int64_t)mrow[r] * D + d0 + c] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int l = lb + 8 * j;
            if (l < L) {
                float part = 0.f;
                if (Mlo) {
                    for (int c = 0; c < dc; ++c) {
                        const float df = (xs[pl * (kUDC + 1) + c] - ms[l * (kUDC + 1) + c]) -
                                         ml[l * (kUDC + 1) + c];
                        part = fmaf(df, df, part);
                    }
                } else {
                    for (int c = 0; c < dc; ++c) {
                        const float df = xs[pl * (kUDC + 1) + c] - ms[l * (kUDC + 1) + c];
                        part = fmaf(df, df, part);
                    }
                }
                acc[j] += (double)part;
            }
        }
        __syncthreads();
    }
    const float sg = *sigma_dev;
    const float inv2s2 = 1.0f / (2.0f * sg * sg);
    const int64_t p = p0 + pl;
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        const int l = lb + 8 * j;
        if (l < L) {
            const float a = expf(-(float)acc[j] * inv2s2);
            at[pl * L + l] = a;
            if (p < N) A[p * L + l] = a;
        }
    }
    if (Z0 == nullptr) return;
    __syncthreads();
    if (t < kUTP && p0 + t < N) {
        const float* ar = at + t * L;
        float m = ar[0];
        for (int l = 1; l < L; ++l) m = fmaxf(m, ar[l]);
        float s = 0.f;
        for (int l = 0; l < L; ++l) s += expf(ar[l] - m);
        float* zr = Z0 + (p0 + t) * L;
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

// One warp per point: squared distance to its mode (lanes over features,
// float32 differences, squares summed in float32 chunks of 8 and the chunks
// in float64), float64 kernel value, and the cut edges of its row.
__global__ void __launch_bounds__(256)
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
    for (int64_t p = (int64_t)blockIdx.x * 8 + warp; p < N; p += nwarps) {
        const int lp = labels[p];
        const float* xp = X + p * D;
        const float* xm = M ? M + (int64_t)lp * D : X + (int64_t)modes[lp] * D;
        const double d2 = warp_sq_dist(xp, xm, Mlo ? Mlo + (int64_t)lp * D : nullptr, D, lane);
        double cut = 0.0;
        for (int64_t e = row_ptr[p] + lane; e < row_ptr[p + 1]; e += 32) {
            const int q = col_idx[e];
            if (labels[q] != lp) cut += w ? (double)w[e] : 1.0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cut += __shfl_xor_sync(0xffffffffu, cut, o);
        // ||z_p - z_q||^2 = 2 for every cut edge
        if (lane == 0) acc += -exp(-d2 * inv2s2) + 0.5 * (double)lambda * 2.0 * cut;
    }
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
    const size_t smem = sizeof(float) * ((size_t)kUTP * (kUDC + 1) +
                                         (Mlo ? 2 : 1) * (size_t)L * (kUDC + 1) + (size_t)kUTP * L);
    const unsigned grid = (unsigned)((N + kUTP - 1) / kUTP);
    const int lpt = (L + 7) / 8;
#define SLK_UNARY(LPT_)                                                                     \
    {                                                                                       \
        auto kern = unary_kernel<LPT_>;                                                     \
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                               (int)smem));                                 \
        kern<<<grid, kUThreads, smem, ctx->stream>>>(X, N, D, modes, M, Mlo, L, sigma_dev, A, Z0); \
    }
    if (lpt <= 1) { SLK_UNARY(1) }
    else if (lpt <= 2) { SLK_UNARY(2) }
    else if (lpt <= 4) { SLK_UNARY(4) }
    else if (lpt <= 8) { SLK_UNARY(8) }
    else if (lpt <= 16) { SLK_UNARY(16) }
    else { SLK_UNARY(32) }
#undef SLK_UNARY
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
    int64_t grid = (N + 7) / 8;
    if (grid > (int64_t)ctx->num_sms * 8) grid = (int64_t)ctx->num_sms * 8;
    energy_kernel<<<(unsigned)grid, 256, 0, ctx->stream>>>(X, D, labels, row_ptr, col_idx, w, N,
                                                          modes, M, Mlo, sigma_dev, lambda, st);
    SLK_LAUNCH_CHECK(ctx, "energy_kernel");
    return SLK_OK;
}
