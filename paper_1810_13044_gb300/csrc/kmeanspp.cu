// K-means++ seeding on the GPU (the initial seeds of Section 4.2, which
// cites Arthur & Vassilvitskii 2007 for them), with the random draws made
// by the caller: seed 0 is the point `first`; seed i is the first point p
// whose running sum D(x_0)^2 + ... + D(x_p)^2 exceeds u_i * sum_q D(x_q)^2,
// D(x)^2 the squared distance to the closest seed chosen so far (the last
// point if no running sum does; point floor(u_i N) if every D^2 is 0).
//
// Per seed, two launches:
//   kpp_min_dist_kernel  one warp per point: ||x_p - c||^2 in float64 from
//                        exact float64 differences, min into closest[p]
//                        (an HBM pass over X; the float64 FMAs bound it)
//   kpp_select_kernel    one block: 1024 contiguous chunks of closest[]
//                        summed in index order, their offsets accumulated
//                        in index order by one thread, then the chunk that
//                        holds u_i * total rescanned in index order.  Every
//                        running sum is offset + (running sum inside the
//                        chunk), the same additions that produced the
//                        offsets, so the sums are non-decreasing and the
//                        point is found in that chunk.
#include <math.h>
#include <stdint.h>

#include "slk_internal.cuh"

namespace {

constexpr int kSelThreads = 1024;

template <bool VEC4>
__global__ void __launch_bounds__(256)
kpp_min_dist_kernel(const float* __restrict__ X, int64_t N, int D, const int32_t* __restrict__ seeds,
                    int i, int first_pass, double* __restrict__ closest) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float* c = X + (int64_t)seeds[i - 1] * D;
    for (int64_t p = warp; p < N; p += nwarps) {
        const float* x = X + p * D;
        double acc = 0.0;
        if (VEC4) {
            const float4* x4 = reinterpret_cast<const float4*>(x);
            const float4* c4 = reinterpret_cast<const float4*>(c);
            for (int j = lane; j < (D >> 2); j += 32) {
                const float4 a = __ldg(x4 + j), b = __ldg(c4 + j);
                const double d0 = (double)a.x - (double)b.x, d1 = (double)a.y - (double)b.y;
                const double d2 = (double)a.z - (double)b.z, d3 = (double)a.w - (double)b.w;
                acc = fma(d0, d0, acc);
                acc = fma(d1, d1, acc);
                acc = fma(d2, d2, acc);
                acc = fma(d3, d3, acc);
            }
        } else {
            for (int j = lane; j < D; j += 32) {
                const double d = (double)__ldg(x + j) - (double)__ldg(c + j);
                acc = fma(d, d, acc);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) closest[p] = first_pass ? acc : fmin(closest[p], acc);
    }
}

__global__ void __launch_bounds__(kSelThreads)
kpp_select_kernel(const double* __restrict__ closest, int64_t N, const double* __restrict__ u, int i,
                  int32_t* __restrict__ seeds) {
    __shared__ double ssum[kSelThreads];
    __shared__ double soff[kSelThreads];
    __shared__ double stotal;
    __shared__ int sowner;
    const int t = threadIdx.x;
    const int64_t chunk = (N + kSelThreads - 1) / kSelThreads;
    const int64_t b = (int64_t)t * chunk, e = (b + chunk < N) ? b + chunk : N;
    double s = 0.0;
    for (int64_t j = b; j < e; ++j) s += closest[j];
    ssum[t] = s;
    __syncthreads();
    const double r_u = u[i - 1];
    if (t == 0) {
        double run = 0.0;
        for (int c = 0; c < kSelThreads; ++c) {
            soff[c] = run;
            run += ssum[c];
        }
        stotal = run;
        sowner = -1;
        if (run > 0.0) {
            const double r = r_u * run;
            for (int c = 0; c < kSelThreads; ++c)
                if (soff[c] + ssum[c] > r) { sowner = c; break; }
        }
    }
    __syncthreads();
    if (t == 0 && !(stotal > 0.0)) {
        int64_t pick = (int64_t)(r_u * (double)N);
        seeds[i] = (int32_t)(pick < N - 1 ? pick : N - 1);
        return;
    }
    if (t == 0 && sowner < 0) seeds[i] = (int32_t)(N - 1);
    if (t != sowner) return;
    const double r = r_u * stotal, off = soff[t];
    double run = 0.0;
    int64_t pick = e - 1;
    for (int64_t j = b; j < e; ++j) {
        run += closest[j];
        if (off + run > r) { pick = j; break; }
    }
    seeds[i] = (int32_t)pick;
}

__global__ void kpp_first_kernel(int32_t first, int32_t* seeds) { seeds[0] = first; }

}  // namespace

size_t kmeanspp_ws_bytes(int64_t N, int L) {
    return align_up(sizeof(double) * (size_t)N, 256) + align_up(sizeof(double) * (size_t)L, 256);
}

slk_status kmeanspp_launch(slk_ctx* ctx, const float* X, int64_t N, int D, int L, int32_t first,
                           const double* u_host, int32_t* seeds, void* ws) {
    WsCarver wc(ws);
    double* closest = wc.take<double>((size_t)N);
    double* u = wc.take<double>((size_t)(L > 1 ? L - 1 : 1));
    if (L > 1)
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(u, u_host, sizeof(double) * (size_t)(L - 1),
                                          cudaMemcpyHostToDevice, ctx->stream));
    SLK_COUNT_LAUNCH(ctx, 1 + 2 * (L - 1));
    kpp_first_kernel<<<1, 1, 0, ctx->stream>>>(first, seeds);
    SLK_LAUNCH_CHECK(ctx, "kpp_first_kernel");
    const bool vec4 = (D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    int64_t grid = (N + 7) / 8;
    if (grid > (int64_t)ctx->num_sms * 16) grid = (int64_t)ctx->num_sms * 16;
    for (int i = 1; i < L; ++i) {
        if (vec4)
            kpp_min_dist_kernel<true><<<(unsigned)grid, 256, 0, ctx->stream>>>(X, N, D, seeds, i,
                                                                                i == 1, closest);
        else
            kpp_min_dist_kernel<false><<<(unsigned)grid, 256, 0, ctx->stream>>>(X, N, D, seeds, i,
                                                                                 i == 1, closest);
        SLK_LAUNCH_CHECK(ctx, "kpp_min_dist_kernel");
        kpp_select_kernel<<<1, kSelThreads, 0, ctx->stream>>>(closest, N, u, i, seeds);
        SLK_LAUNCH_CHECK(ctx, "kpp_select_kernel");
    }
    return SLK_OK;
}
