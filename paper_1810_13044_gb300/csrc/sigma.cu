// Kernel width of Section 4.2 from the kNN squared distances.
//
// MEDIAN: sigma = median of sqrt(dist2).  sqrt is monotone, so the order
// statistics are selected on dist2 itself: non-negative floats order like
// their bit patterns, and a most-significant-byte-first radix select (four
// passes of a 256-bin histogram) finds the element of a given rank exactly.
// MEANSQ: sigma^2 = mean of dist2 (the paper's estimator), summed in float64.
#include <math.h>

#include "slk_internal.cuh"
#include "sync.cuh"

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

// The median in one cooperative launch: the four histogram passes of the
// radix select are separated by grid barriers whose last arriving block picks
// the bucket (the same steps as radix_hist / radix_pick); for an even count
// the upper middle statistic is the lower one again when more than r + 1
// values are <= it, else the smallest value above it (one more pass).  sigma
// is then computed as radix_store_kernel does.  A barrier wait that times
// out sets the barrier-timeout bit of st->error and returns.
__global__ void __launch_bounds__(256)
median_coop_kernel(const float* __restrict__ v, int64_t n, unsigned long long rank, int even,
                   DevState* st) {
    __shared__ unsigned int h[256];
    __shared__ unsigned int s_min;
    __shared__ unsigned long long s_cnt;
    GridBarrier* gb = reinterpret_cast<GridBarrier*>(st->sel_bar);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
        __syncthreads();
        const unsigned prefix = ld_acq(&st->sel_prefix), mask = ld_acq(&st->sel_mask);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const unsigned key = __float_as_uint(v[i]);
            if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 256; i += blockDim.x)
            if (h[i]) atomicAdd(&st->sel_hist[i], h[i]);
        const int r = grid_barrier(gb, gridDim.x, [&]() {
            unsigned long long rk = st->sel_rank, cum = 0;
            int b = 0;
            for (; b < 255; ++b) {
                if (cum + st->sel_hist[b] > rk) break;
                cum += st->sel_hist[b];
            }
            st->sel_rank = rk - cum;
            st->sel_prefix |= ((unsigned)b) << shift;
            st->sel_mask |= 255u << shift;
            for (int i = 0; i < 256; ++i) st->sel_hist[i] = 0u;
            return false;
        });
        if (r < 0) {
            if (threadIdx.x == 0) atomicOr(&st->error, ERR_BARRIER_TIMEOUT);
            return;
        }
    }
    const unsigned xr = ld_acq(&st->sel_prefix);   // bits of the lower middle statistic
    if (even) {
        if (threadIdx.x == 0) {
            s_min = 0xffffffffu;
            s_cnt = 0ull;
        }
        __syncthreads();
        unsigned my_min = 0xffffffffu;
        unsigned long long my_cnt = 0ull;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const unsigned key = __float_as_uint(v[i]);
            if (key <= xr) ++my_cnt;
            else my_min = min(my_min, key);
        }
        atomicMin(&s_min, my_min);
        atomicAdd(&s_cnt, my_cnt);
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicMin(&st->sel_min_bits, s_min);
            atomicAdd(&st->sel_cnt, s_cnt);
        }
        const int r = grid_barrier(gb, gridDim.x, [&]() {
            const double lo = sqrt((double)__uint_as_float(xr));
            const unsigned up = (st->sel_cnt >= rank + 2) ? xr : st->sel_min_bits;
            st->sum_d2 = lo;
            st->sigma = (float)(0.5 * (lo + sqrt((double)__uint_as_float(up))));
            return false;
        });
        if (r < 0) {
            if (threadIdx.x == 0) atomicOr(&st->error, ERR_BARRIER_TIMEOUT);
            return;
        }
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double lo = sqrt((double)__uint_as_float(xr));
        st->sum_d2 = lo;
        st->sigma = (float)lo;
    }
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
    if (ctx->coop_supported) {
        // one cooperative launch (lower middle rank, and the upper one if even)
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->sel_bar[0], 0, sizeof(st->sel_bar), ctx->stream));
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->sel_cnt, 0, sizeof(st->sel_cnt), ctx->stream));
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->sel_min_bits, 0xff, sizeof(st->sel_min_bits), ctx->stream));
        const unsigned long long rank =
            even ? (unsigned long long)(n / 2 - 1) : (unsigned long long)(n / 2);
        SLK_COUNT_LAUNCH(ctx, 2);
        radix_init_kernel<<<1, 256, 0, ctx->stream>>>(rank, st);
        SLK_LAUNCH_CHECK(ctx, "radix_init_kernel");
        int per_sm = 0;
        SLK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, median_coop_kernel, 256, 0));
        int64_t cgrid = (n + 2047) / 2048;
        if (cgrid > (int64_t)ctx->num_sms * (per_sm < 1 ? 1 : per_sm)) cgrid = (int64_t)ctx->num_sms * per_sm;
        if (cgrid > (int64_t)ctx->num_sms) cgrid = ctx->num_sms;
        if (cgrid < 1) cgrid = 1;
        const float* v_ = dist2;
        int64_t n_ = n;
        unsigned long long rk_ = rank;
        int ev_ = even ? 1 : 0;
        DevState* st_ = st;
        void* args[] = {&v_, &n_, &rk_, &ev_, &st_};
        const cudaError_t e = cudaLaunchCooperativeKernel((const void*)median_coop_kernel,
                                                          dim3((unsigned)cgrid), dim3(256), args, 0,
                                                          ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "median_coop_kernel");
        return SLK_OK;
    }
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
