// The symmetric affinity K' = (K + K^t) / 2 of the directed kNN graph
// (Prop. 1 assumes a symmetric K; the kNN affinity of Section 4.2 is not).
// Row p of K' is the union of row p of K (its out-neighbours) and column p
// of K (the points that list p), by increasing column; K'_pq =
// (K_pq + K_qp) / 2 with a missing entry counting 0.
//
//   sym_in_count_kernel   in-degrees (atomic counts)
//   scan (3 launches)     in-list offsets
//   sym_in_fill_kernel    sources of every column (atomic cursors: any order)
//   sym_rows_kernel<0>    per row: sort its in-list by source, sort a copy of
//                         its out-list by column, count the union
//   scan                  row offsets of K'
//   sym_rows_kernel<1>    per row: merge into K' (deterministic: both lists
//                         sorted), weights 0.5 (w_pq + w_qp)
// One thread per row; in-lists are short except at hubs, where the
// insertion sort is the cost.
#include <stdint.h>

#include "slk_internal.cuh"

namespace {

constexpr int kScanBlock = 1024;

__global__ void sym_in_count_kernel(const int64_t* __restrict__ row_ptr,
                                    const int32_t* __restrict__ col_idx, int64_t N,
                                    int64_t* __restrict__ cnt) {
    const int64_t nnz = row_ptr[N];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(cnt + col_idx[e]), 1ull);
}

// Exclusive scan of v[0..n) into out[0..n] (out[n] = total), in three steps:
// per-block inclusive scans with block totals, a one-block scan of the
// totals, the block offsets added.
__global__ void __launch_bounds__(kScanBlock)
scan_blocks_kernel(const int64_t* __restrict__ v, int64_t n, int64_t* __restrict__ out,
                   int64_t* __restrict__ block_tot) {
    __shared__ int64_t s[kScanBlock];
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    s[threadIdx.x] = (i < n) ? v[i] : 0;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        const int64_t t = (threadIdx.x >= o) ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i + 1] = s[threadIdx.x];   // inclusive -> exclusive shifted by one
    if (threadIdx.x == kScanBlock - 1) block_tot[blockIdx.x] = s[threadIdx.x];
}

__global__ void scan_totals_kernel(int64_t* __restrict__ block_tot, int nb) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t run = 0;
        for (int b = 0; b < nb; ++b) {
            const int64_t t = block_tot[b];
            block_tot[b] = run;   // exclusive offsets of the blocks
            run += t;
        }
    }
}

__global__ void __launch_bounds__(kScanBlock)
scan_add_kernel(int64_t n, int64_t* __restrict__ out, const int64_t* __restrict__ block_off) {
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
    if (i < n) out[i + 1] += block_off[blockIdx.x];
}

__global__ void sym_in_fill_kernel(const int64_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ col_idx,
                                   const float* __restrict__ w, int64_t N,
                                   const int64_t* __restrict__ in_ptr, int64_t* __restrict__ cursor,
                                   int32_t* __restrict__ in_src, float* __restrict__ in_w) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N;
         q += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t e = row_ptr[q]; e < row_ptr[q + 1]; ++e) {
            const int32_t p = col_idx[e];
            const int64_t slot =
                in_ptr[p] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(cursor + p), 1ull);
            in_src[slot] = (int32_t)q;
            in_w[slot] = w ? w[e] : 1.f;
        }
    }
}

// WRITE = 0: sort row p's in-list (by source, then weight for a repeated
// source) and store the size of the union with its out-list in cnt[p];
// WRITE = 1: write row p of K' from the two sorted lists.
template <int WRITE>
__global__ void sym_rows_kernel(const int64_t* __restrict__ row_ptr,
                                const int32_t* __restrict__ col_idx, const float* __restrict__ w,
                                int64_t N, const int64_t* __restrict__ in_ptr,
                                int32_t* __restrict__ in_src, float* __restrict__ in_w,
                                int64_t* __restrict__ cnt, const int64_t* __restrict__ out_ptr,
                                int32_t* __restrict__ out_col, float* __restrict__ out_w,
                                unsigned int* __restrict__ err) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = in_ptr[p], i1 = in_ptr[p + 1];
        if (!WRITE) {
            for (int64_t a = i0 + 1; a < i1; ++a) {   // insertion sort by (source, weight)
                const int32_t ks = in_src[a];
                const float kw = in_w[a];
                int64_t b = a - 1;
                while (b >= i0 && (in_src[b] > ks || (in_src[b] == ks && in_w[b] > kw))) {
                    in_src[b + 1] = in_src[b];
                    in_w[b + 1] = in_w[b];
                    --b;
                }
                in_src[b + 1] = ks;
                in_w[b + 1] = kw;
            }
        }
        // out-list sorted by column (a kNN row: at most SLK_MAX_K entries; a
        // longer row is refused with the error bit and left empty)
        const int64_t o0 = row_ptr[p], o1 = row_ptr[p + 1];
        const int64_t no = o1 - o0;
        if (no > SLK_MAX_K || no < 0) {
            if (!WRITE) {
                atomicOr(err, 1u);
                cnt[p] = 0;
            }
            continue;
        }
        int32_t oc[SLK_MAX_K];
        float ow[SLK_MAX_K];
        const int nk = (int)no;
        for (int a = 0; a < nk; ++a) {
            int32_t c = col_idx[o0 + a];
            float x = w ? w[o0 + a] : 1.f;
            int b = a - 1;
            while (b >= 0 && (oc[b] > c || (oc[b] == c && ow[b] > x))) {
                oc[b + 1] = oc[b];
                ow[b + 1] = ow[b];
                --b;
            }
            oc[b + 1] = c;
            ow[b + 1] = x;
        }
        // merge: each distinct column once, K_pq and K_qp summed over repeats
        int a = 0;
        int64_t t = i0, u = 0;
        const int64_t base = WRITE ? out_ptr[p] : 0;
        while (a < nk || t < i1) {
            const int32_t ca = (a < nk) ? oc[a] : 0x7fffffff;
            const int32_t ct = (t < i1) ? in_src[t] : 0x7fffffff;
            const int32_t c = ca < ct ? ca : ct;
            float kpq = 0.f, kqp = 0.f;
            while (a < nk && oc[a] == c) kpq += ow[a++];
            while (t < i1 && in_src[t] == c) kqp += in_w[t++];
            if (WRITE) {
                out_col[base + u] = c;
                out_w[base + u] = 0.5f * (kpq + kqp);
            }
            ++u;
        }
        if (!WRITE) cnt[p] = u;
    }
}

slk_status scan_launch(slk_ctx* ctx, const int64_t* v, int64_t n, int64_t* out, int64_t* block_tot) {
    const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
    SLK_COUNT_LAUNCH(ctx, 3);
    scan_blocks_kernel<<<nb > 0 ? nb : 1, kScanBlock, 0, ctx->stream>>>(v, n, out, block_tot);
    scan_totals_kernel<<<1, 32, 0, ctx->stream>>>(block_tot, nb > 0 ? nb : 1);
    scan_add_kernel<<<nb > 0 ? nb : 1, kScanBlock, 0, ctx->stream>>>(n, out, block_tot);
    SLK_LAUNCH_CHECK(ctx, "scan kernels");
    return SLK_OK;
}

}  // namespace

size_t symmetrize_ws_bytes(int64_t N, int64_t nnz) {
    const int64_t nb = (N + kScanBlock - 1) / kScanBlock + 1;
    return 3 * align_up(sizeof(int64_t) * (size_t)(N + 1), 256) +
           align_up(sizeof(int64_t) * (size_t)nb, 256) +
           align_up(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), 256) +
           align_up(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1), 256) + 1024;
}

slk_status symmetrize_launch(slk_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx,
                             const float* w, int64_t N, int64_t nnz, int64_t* out_row_ptr,
                             int32_t* out_col, float* out_w, void* ws, unsigned int* err) {
    WsCarver wc(ws);
    int64_t* cnt = wc.take<int64_t>((size_t)N + 1);
    int64_t* in_ptr = wc.take<int64_t>((size_t)N + 1);
    int64_t* cursor = wc.take<int64_t>((size_t)N + 1);
    int64_t* btot = wc.take<int64_t>((size_t)((N + kScanBlock - 1) / kScanBlock + 1));
    int32_t* in_src = wc.take<int32_t>((size_t)(nnz > 0 ? nnz : 1));
    float* in_w = wc.take<float>((size_t)(nnz > 0 ? nnz : 1));
    cudaStream_t s = ctx->stream;
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (size_t)N, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(cursor, 0, sizeof(int64_t) * (size_t)N, s));
    int64_t g = (N + 255) / 256;
    if (g > (int64_t)ctx->num_sms * 8) g = (int64_t)ctx->num_sms * 8;
    if (g < 1) g = 1;
    SLK_COUNT_LAUNCH(ctx, 4);
    sym_in_count_kernel<<<(unsigned)g, 256, 0, s>>>(row_ptr, col_idx, N, cnt);
    SLK_LAUNCH_CHECK(ctx, "sym_in_count_kernel");
    slk_status r = scan_launch(ctx, cnt, N, in_ptr, btot);
    if (r != SLK_OK) return r;
    sym_in_fill_kernel<<<(unsigned)g, 256, 0, s>>>(row_ptr, col_idx, w, N, in_ptr, cursor, in_src, in_w);
    SLK_LAUNCH_CHECK(ctx, "sym_in_fill_kernel");
    sym_rows_kernel<0><<<(unsigned)g, 256, 0, s>>>(row_ptr, col_idx, w, N, in_ptr, in_src, in_w, cnt,
                                                   nullptr, nullptr, nullptr, err);
    SLK_LAUNCH_CHECK(ctx, "sym_rows_kernel<0>");
    r = scan_launch(ctx, cnt, N, out_row_ptr, btot);
    if (r != SLK_OK) return r;
    sym_rows_kernel<1><<<(unsigned)g, 256, 0, s>>>(row_ptr, col_idx, w, N, in_ptr, in_src, in_w, cnt,
                                                   out_row_ptr, out_col, out_w, err);
    SLK_LAUNCH_CHECK(ctx, "sym_rows_kernel<1>");
    return SLK_OK;
}
