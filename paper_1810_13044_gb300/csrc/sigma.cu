// Kernel width of Section 4.2 from the kNN squared distances.
//
// MEDIAN: sigma = median of sqrt(dist2).  sqrt is monotone, so the order
// statistics are selected on dist2 itself: non-negative floats order like
// their bit patterns, and a most-significant-byte-first radix select (four
// passes of a 256-bin histogram) finds the element of a given rank exactly.
// MEANSQ: sigma^2 = mean of dist2 (the paper's estimator), summed in float64.
#include <math.h>

#include "slk_internal.cuh"

namespace {

__global__ void radix_hist_kernel(const float* __restrict__ v, int64_t n, int shift,
                                  DevState* st) {
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const unsigned prefix = st->sel_prefix, mask = st->sel_mask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned key = __float_as_uint(v[i]);
        if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&st->sel_hist[i], h[i]);
}

// Pick the bucket holding the wanted rank, narrow prefix/mask, clear the histogram.
__global__ void radix_pick_kernel(int shift, DevState* st) {
    if (threadIdx.x == 0) {
        unsigned long long rank = st->sel_rank, cum = 0;
        int b = 0;
        for (; b < 255; ++b) {
            if (cum + st->sel_hist[b] > rank) break;
            cum += st->sel_hist[b];
        }
        st->sel_rank = rank - cum;
        st->sel_prefix |= ((unsigned)b) << shift;
        st->sel_mask |= 255u << shift;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) st->sel_hist[i] = 0u;
}

__global__ void radix_init_kernel(unsigned long long rank, DevState* st) {
    st->sel_prefix = 0u;
    st->sel_mask = 0u;
    st->sel_rank = rank;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) st->sel_hist[i] = 0u;
}

// slot 0: store the first order statistic's sqrt in sum_d2; slot 1: average it
// with the second one and store sigma.
__global__ void radix_store_kernel(int slot, int even, DevState* st) {
    const double v = sqrt((double)__uint_as_float(st->sel_prefix));
    if (slot == 0) {
        st->sum_d2 = v;
        if (!even) st->sigma = (float)v;
    } else {
        st->sigma = (float)(0.5 * (st->sum_d2 + v));
    }
}

__global__ void sum_kernel(const float* __restrict__ v, int64_t n, DevState* st) {
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (double)v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        atomicAdd(&st->sum_d2, t);
    }
}

__global__ void meansq_finish_kernel(int64_t n, DevState* st) {
    st->sigma = (float)sqrt(st->sum_d2 / (double)n);
}

}  // namespace

size_t sigma_ws_bytes(int64_t) { return 0; }

slk_status sigma_launch(slk_ctx* ctx, const float* dist2, int64_t n, int rule, DevState* st) {
    PhaseScope ps(ctx, SLK_PHASE_SIGMA);
    int64_t grid = (n + 255) / 256;
    if (grid > (int64_t)ctx->num_sms * 4) grid = (int64_t)ctx->num_sms * 4;
    if (grid < 1) grid = 1;
    if (rule == SLK_SIGMA_MEANSQ) {
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->sum_d2, 0, sizeof(double), ctx->stream));
        SLK_COUNT_LAUNCH(ctx, 2);
        sum_kernel<<<(unsigned)grid, 256, 0, ctx->stream>>>(dist2, n, st);
        SLK_LAUNCH_CHECK(ctx, "sum_kernel");
        meansq_finish_kernel<<<1, 1, 0, ctx->stream>>>(n, st);
        SLK_LAUNCH_CHECK(ctx, "meansq_finish_kernel");
        return SLK_OK;
    }
    const bool even = (n % 2) == 0;
    const int nsel = even ? 2 : 1;
    for (int s = 0; s < nsel; ++s) {
        const unsigned long long rank = even ? (unsigned long long)(n / 2 - 1 + s)
                                             : (unsigned long long)(n / 2);
        SLK_COUNT_LAUNCH(ctx, 2 + 2 * 4);
        radix_init_kernel<<<1, 256, 0, ctx->stream>>>(rank, st);
        for (int shift = 24; shift >= 0; shift -= 8) {
            radix_hist_kernel<<<(unsigned)grid, 256, 0, ctx->stream>>>(dist2, n, shift, st);
            radix_pick_kernel<<<1, 256, 0, ctx->stream>>>(shift, st);
        }
        radix_store_kernel<<<1, 1, 0, ctx->stream>>>(s, even ? 1 : 0, st);
    }
    SLK_LAUNCH_CHECK(ctx, "radix select");
    return SLK_OK;
}
