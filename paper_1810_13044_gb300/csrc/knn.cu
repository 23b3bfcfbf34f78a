// Exact kNN affinity graph of Section 4.2 (k nearest neighbours q != p by
// Euclidean distance, ascending by (distance, index)), brute force.
//
// Pipeline
//  1. prep: centre the features (x - mu, mu the column mean: distances are
//     translation invariant) and round them to the candidate operand type
//     (float32 or bfloat16).  Per point keep ||xt_p||^2 and the rounding
//     perturbation rho_p >= ||xt_p - (x_p - mu)|| (float32 lane sums with
//     their rounding bounds, lanes added as 2Sum float pairs).
//  2. candidates: a distance-tile kernel evaluates
//     dt(p, q) = ||xt_p||^2 + ||xt_q||^2 - 2 xt_p . xt_q for all pairs and keeps,
//     per row and per column split, the KC smallest (KC > k), sorted.
//  3. rerank + certificate (one warp per row): merge the splits' sorted lists,
//     recompute exactly in float32, from the original features, the distances
//     of the candidates whose lower bound can still reach the k nearest, keep
//     the k smallest.  With T the KC-th smallest dt, every other point q
//     satisfies dt(p,q) >= T, hence (rounding bounds below) its true distance
//     is at least LB = (sqrt(T - delta) - rho_p - rho_max)^2.  The row is
//     certified when the k-th exact distance, inflated by its own rounding
//     bound, is below LB; then the row equals a full float32 scan.
//  4. fallback: with bfloat16 candidates, the rows that fail the certificate
//     first get float32 candidate tiles and the same rerank under the float32
//     certificate; rows that fail that (or the float32 certificate of a
//     float32 pass) are rescanned exactly.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <stdint.h>

#include "slk_internal.cuh"

int knn_tc_tile_cols();
int knn_tc_lists_per_split(int kc, int ew);

namespace {

constexpr int BM = 128, BN = 128, BK = 16, KT = 256;
constexpr int QC = 32;      // per-row insertion queue of the candidate kernel
constexpr int MAXE = 16;    // merge entries per lane (splits * KC <= 512)
#define kInf __int_as_float(0x7f800000)
constexpr int kNoIdx = 0x7fffffff;

__device__ __forceinline__ bool lex_less(float d, int i, float d2, int i2) {
    return d < d2 || (d == d2 && i < i2);
}

// -------------------------------------------------------------------- prep

// Column sums (the centring mean mu only has to be some float vector:
// distances are translation invariant): float32 sums of 64 rows, added in
// float64.  Each lane sums V adjacent columns (V = 4: 16-byte loads, when D
// is a multiple of 4 and X is 16-byte aligned); the rows and their order do
// not depend on V.
template <int V>
__global__ void col_sum_kernel(const float* __restrict__ X, int64_t N, int D,
                               double* __restrict__ colsum) {
    __shared__ double sm[8][32 * V + 1];
    const int DV = D / V;
    const int c = blockIdx.x * 32 + threadIdx.x;   // column group
    const int64_t per = (N + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = (int64_t)blockIdx.y * per;
    const int64_t r1 = (r0 + per < N) ? r0 + per : N;
    double acc[V];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = 0.0;
    if (c < DV) {
        // rows r0 + y, r0 + y + 8, ... in increasing order; each chunk of 64
        // of them summed in float32 (8 loads in flight), the chunks in
        // float64 outside the inner loops (a float64 add predicated into
        // every iteration would occupy GB300's narrow float64 pipe)
        for (int64_t cb = r0 + threadIdx.y; cb < r1; cb += 512) {
            float part[V];
#pragma unroll
            for (int q = 0; q < V; ++q) part[q] = 0.f;
#pragma unroll 2
            for (int b = 0; b < 8; ++b) {
                float v[8][V];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int64_t r = cb + 64 * b + 8 * t;
                    if constexpr (V == 4) {
                        const float4 w = (r < r1) ? __ldg(reinterpret_cast<const float4*>(X + r * D) + c)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                        v[t][0] = w.x; v[t][1] = w.y; v[t][2] = w.z; v[t][3] = w.w;
                    } else {
                        v[t][0] = (r < r1) ? X[r * D + c] : 0.f;
                    }
                }
#pragma unroll
                for (int t = 0; t < 8; ++t)
#pragma unroll
                    for (int q = 0; q < V; ++q) part[q] += v[t][q];
            }
#pragma unroll
            for (int q = 0; q < V; ++q) acc[q] += (double)part[q];
        }
    }
#pragma unroll
    for (int q = 0; q < V; ++q) sm[threadIdx.y][threadIdx.x * V + q] = acc[q];
    __syncthreads();
    if (threadIdx.y == 0 && c < DV) {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            double t = 0.0;
            for (int i = 0; i < 8; ++i) t += sm[i][threadIdx.x * V + q];
            atomicAdd(&colsum[c * V + q], t);
        }
    }
}

// Column means of the centring: mu_j = (float)(colsum_j / N).
__global__ void mu_kernel(const double* __restrict__ colsum, int64_t N, int D, float* __restrict__ mu) {
    const double inv_n = 1.0 / (double)N;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D; j += gridDim.x * blockDim.x)
        mu[j] = (float)(colsum[j] * inv_n);
}

// One warp per padded row: xt = round(v), v = fl(x - mu), with
//   norms[p] = ||xt_p||^2: lane sums of xt^2 in float32, lanes added as float
//     pairs (within a few u^2 of the exact sum);
//   rho[p] >= ||xt_p - (x_p - mu)||: with e = xt - v (exact in float32) and
//     |v - (x - mu)| <= u |v|, rho <= ||e|| + u ||v||, both norms from float32
//     lane sums inflated by their summation bound and rounded up.
// Every square of a lane sum passes through at most Dp/32 roundings (u =
// 2^-24): V = 1 sums the lane's Dp/32 columns in one accumulator; V = 4
// (16-byte loads, D a multiple of 4, X 16-byte aligned, Dp >= 128) keeps one
// accumulator per column of its 4-column groups, ceil(Dp/128) terms each,
// added pairwise at the end: ceil(Dp/128) + 2 <= Dp/32 roundings.  Each
// bfloat16 square is exact.
// The row maxima go to st with one atomic per block.
template <int V>
__global__ void __launch_bounds__(256)
prep_rows_kernel(const float* __restrict__ X, int64_t N, int D, int Dp,
                 int64_t Np, const float* __restrict__ mu, int to_bf16,
                 float* __restrict__ xt32, __nv_bfloat16* __restrict__ xt16,
                 float* __restrict__ norms, float* __restrict__ rho,
                 float* __restrict__ norms32, DevState* st) {
    __shared__ unsigned bmax_n, bmax_r, bmax_n32;
    if (threadIdx.x == 0) { bmax_n = 0u; bmax_r = 0u; bmax_n32 = 0u; }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const double bound = 1.0 + (double)(Dp / 32 + 2) * 5.9604644775390625e-08;
    unsigned my_n = 0u, my_r = 0u, my_n32 = 0u;
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < Np;
         p += nw) {
        float n2v[V], e2v[V], v2v[V];
#pragma unroll
        for (int q = 0; q < V; ++q) { n2v[q] = 0.f; e2v[q] = 0.f; v2v[q] = 0.f; }
#pragma unroll 4
        for (int j = lane * V; j < Dp; j += 32 * V) {
            float v[V], vv[V];
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = 0.f;
            if (p < N && j < D) {
                if constexpr (V == 4) {
                    const float4 x = __ldg(reinterpret_cast<const float4*>(X + p * D + j));
                    const float4 m = __ldg(reinterpret_cast<const float4*>(mu + j));
                    v[0] = x.x - m.x; v[1] = x.y - m.y; v[2] = x.z - m.z; v[3] = x.w - m.w;
                } else {
                    v[0] = X[p * D + j] - __ldg(mu + j);
                }
            }
            if (to_bf16) {
                if constexpr (V == 4) {
                    const __nv_bfloat162 b01 = __floats2bfloat162_rn(v[0], v[1]);
                    const __nv_bfloat162 b23 = __floats2bfloat162_rn(v[2], v[3]);
                    uint2 w;
                    w.x = *reinterpret_cast<const unsigned*>(&b01);
                    w.y = *reinterpret_cast<const unsigned*>(&b23);
                    *reinterpret_cast<uint2*>(xt16 + p * Dp + j) = w;
                    vv[0] = __low2float(b01); vv[1] = __high2float(b01);
                    vv[2] = __low2float(b23); vv[3] = __high2float(b23);
                } else {
                    const __nv_bfloat16 b = __float2bfloat16_rn(v[0]);
                    xt16[p * Dp + j] = b;
                    vv[0] = __bfloat162float(b);
                }
            } else {
                if constexpr (V == 4)
                    *reinterpret_cast<float4*>(xt32 + p * Dp + j) = make_float4(v[0], v[1], v[2], v[3]);
                else
                    xt32[p * Dp + j] = v[0];
#pragma unroll
                for (int q = 0; q < V; ++q) vv[q] = v[q];
            }
#pragma unroll
            for (int q = 0; q < V; ++q) {
                n2v[q] = fmaf(vv[q], vv[q], n2v[q]);
                const float e = vv[q] - v[q];
                e2v[q] = fmaf(e, e, e2v[q]);
                v2v[q] = fmaf(v[q], v[q], v2v[q]);
            }
        }
        float n2 = n2v[0], e2 = e2v[0], v2 = v2v[0];
        if constexpr (V == 4) {
            n2 = (n2v[0] + n2v[1]) + (n2v[2] + n2v[3]);
            e2 = (e2v[0] + e2v[1]) + (e2v[2] + e2v[3]);
            v2 = (v2v[0] + v2v[1]) + (v2v[2] + v2v[3]);
        }
        // butterfly sums of the lane sums as unevaluated float pairs (2Sum):
        // within a few u^2 of the exact sum, and off the slow float64 pipe
        float nh = n2, nl = 0.f, eh = e2, el = 0.f, vh = v2, vl = 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fpair_add(nh, nl, __shfl_xor_sync(0xffffffffu, nh, o), __shfl_xor_sync(0xffffffffu, nl, o));
            fpair_add(eh, el, __shfl_xor_sync(0xffffffffu, eh, o), __shfl_xor_sync(0xffffffffu, el, o));
            fpair_add(vh, vl, __shfl_xor_sync(0xffffffffu, vh, o), __shfl_xor_sync(0xffffffffu, vl, o));
        }
        if (lane == 0) {
            const double dn = (double)nh + (double)nl, de = (double)eh + (double)el,
                         dv = (double)vh + (double)vl;
            const float nf = (float)dn;
            const double r = sqrt(de * bound) + 5.9604644775390625e-08 * sqrt(dv * bound);
            const float rf = __double2float_ru(r * (1.0 + 1e-12));
            // padding rows get an infinite norm: no distance to them can pass a filter
            norms[p] = (p < N) ? nf : __int_as_float(0x7f800000);
            rho[p] = rf;
            const float n32 = (float)dv;   // ||v||^2 of the float32 operand v
            if (norms32) norms32[p] = (p < N) ? n32 : __int_as_float(0x7f800000);
            if (p < N) {
                my_n = max(my_n, __float_as_uint(nf));
                my_r = max(my_r, __float_as_uint(rf));
                my_n32 = max(my_n32, __float_as_uint(n32));
            }
        }
    }
    if (lane == 0) {
        atomicMax(&bmax_n, my_n);
        atomicMax(&bmax_r, my_r);
        atomicMax(&bmax_n32, my_n32);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&st->knn_max_norm_bits, bmax_n);
        atomicMax(&st->knn_max_rho_bits, bmax_r);
        atomicMax(&st->knn_max_norm32_bits, bmax_n32);
    }
}

// ------------------------------------------------------- fp32 candidate tiles

// Shared-memory layout of the candidate kernel (dynamic).
template <int KC>
struct CandSmem {
    float As[2][BK][BM];
    float Bs[2][BK][BN];
    float list_d[BM][KC];
    int list_i[BM][KC];
    float q_d[BM][QC];
    int q_i[BM][QC];
    int q_cnt[BM];
    float thr[BM];
    float nrow[BM];
    float ncol[BN];
};

// Merge the queued entries of row r (owner thread) into its sorted list.
template <int KC>
__device__ __forceinline__ void merge_queue(CandSmem<KC>& s, int r) {
    const int n = min(s.q_cnt[r], QC);
    for (int e = 0; e < n; ++e) {
        const float d = s.q_d[r][e];
        const int i = s.q_i[r][e];
        if (!lex_less(d, i, s.list_d[r][KC - 1], s.list_i[r][KC - 1])) continue;
        int pos = KC - 1;
        while (pos > 0 && lex_less(d, i, s.list_d[r][pos - 1], s.list_i[r][pos - 1])) {
            s.list_d[r][pos] = s.list_d[r][pos - 1];
            s.list_i[r][pos] = s.list_i[r][pos - 1];
            --pos;
        }
        s.list_d[r][pos] = d;
        s.list_i[r][pos] = i;
    }
    s.q_cnt[r] = 0;
    s.thr[r] = s.list_d[r][KC - 1];
}

// Grid: (row blocks of 128, column splits).  Thread (ty, tx) = (t / 16, t % 16)
// owns rows {4ty..4ty+3, 64+4ty..64+4ty+3} and the same pattern of columns.
template <int KC>
__global__ void __launch_bounds__(KT, 2)
knn_cand_fp32_kernel(const float* __restrict__ xt, const float* __restrict__ norms, int64_t N,
                     int Dp, int n_tiles, int64_t Np, float* __restrict__ cand_d,
                     int32_t* __restrict__ cand_i) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CandSmem<KC>& s = *reinterpret_cast<CandSmem<KC>*>(smem_raw);
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int sp = blockIdx.y, splits = gridDim.y;
    const int tile0 = (int)((int64_t)sp * n_tiles / splits);
    const int tile1 = (int)((int64_t)(sp + 1) * n_tiles / splits);
    if (t < BM) {
        for (int j = 0; j < KC; ++j) { s.list_d[t][j] = kInf; s.list_i[t][j] = kNoIdx; }
        s.q_cnt[t] = 0;
        s.thr[t] = kInf;
        s.nrow[t] = norms[row0 + t];
    }
    const int nk = Dp / BK;
    // load mapping: element idx = t + 256 i (i = 0, 1) -> row idx % 128, k-quad idx / 128
    const int lr0 = t & 127, lq0 = t >> 7;          // i = 0: quads 0, 1
    const int lq1 = lq0 + 2;                        // i = 1: quads 2, 3
    for (int tile = tile0; tile < tile1; ++tile) {
        const int64_t col0 = (int64_t)tile * BN;
        __syncthreads();  // previous epilogue finished with ncol / buffers
        if (t < BN) s.ncol[t] = norms[col0 + t];
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        const float* pa = xt + (row0 + lr0) * Dp;
        const float* pb = xt + (col0 + lr0) * Dp;
        float4 ra0 = __ldg(reinterpret_cast<const float4*>(pa + 4 * lq0));
        float4 ra1 = __ldg(reinterpret_cast<const float4*>(pa + 4 * lq1));
        float4 rb0 = __ldg(reinterpret_cast<const float4*>(pb + 4 * lq0));
        float4 rb1 = __ldg(reinterpret_cast<const float4*>(pb + 4 * lq1));
        auto stash = [&](int buf) {
            s.As[buf][4 * lq0 + 0][lr0] = ra0.x; s.As[buf][4 * lq0 + 1][lr0] = ra0.y;
            s.As[buf][4 * lq0 + 2][lr0] = ra0.z; s.As[buf][4 * lq0 + 3][lr0] = ra0.w;
            s.As[buf][4 * lq1 + 0][lr0] = ra1.x; s.As[buf][4 * lq1 + 1][lr0] = ra1.y;
            s.As[buf][4 * lq1 + 2][lr0] = ra1.z; s.As[buf][4 * lq1 + 3][lr0] = ra1.w;
            s.Bs[buf][4 * lq0 + 0][lr0] = rb0.x; s.Bs[buf][4 * lq0 + 1][lr0] = rb0.y;
            s.Bs[buf][4 * lq0 + 2][lr0] = rb0.z; s.Bs[buf][4 * lq0 + 3][lr0] = rb0.w;
            s.Bs[buf][4 * lq1 + 0][lr0] = rb1.x; s.Bs[buf][4 * lq1 + 1][lr0] = rb1.y;
            s.Bs[buf][4 * lq1 + 2][lr0] = rb1.z; s.Bs[buf][4 * lq1 + 3][lr0] = rb1.w;
        };
        stash(0);
        __syncthreads();
        for (int kt = 0; kt < nk; ++kt) {
            const int buf = kt & 1;
            if (kt + 1 < nk) {
                const int k0 = (kt + 1) * BK;
                ra0 = __ldg(reinterpret_cast<const float4*>(pa + k0 + 4 * lq0));
                ra1 = __ldg(reinterpret_cast<const float4*>(pa + k0 + 4 * lq1));
                rb0 = __ldg(reinterpret_cast<const float4*>(pb + k0 + 4 * lq0));
                rb1 = __ldg(reinterpret_cast<const float4*>(pb + k0 + 4 * lq1));
            }
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4*>(&s.As[buf][kk][4 * ty]);
                const float4 a1 = *reinterpret_cast<const float4*>(&s.As[buf][kk][64 + 4 * ty]);
                const float4 b0 = *reinterpret_cast<const float4*>(&s.Bs[buf][kk][4 * tx]);
                const float4 b1 = *reinterpret_cast<const float4*>(&s.Bs[buf][kk][64 + 4 * tx]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            if (kt + 1 < nk) stash(buf ^ 1);
            __syncthreads();
        }
        // ---- epilogue: dt = n_p + n_q - 2 dot, filter against the row thresholds
        unsigned long long pend = 0ull;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + (i - 4);
            const int64_t p = row0 + r;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = (j < 4) ? 4 * tx + j : 64 + 4 * tx + (j - 4);
                const int64_t q = col0 + c;
                const float d = fmaf(-2.f, acc[i][j], s.nrow[r] + s.ncol[c]);
                acc[i][j] = d;
                if (p < N && q < N && q != p && d <= s.thr[r]) pend |= 1ull << (i * 8 + j);
            }
        }
        while (__syncthreads_or(pend != 0ull)) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + (i - 4);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (pend & (1ull << (i * 8 + j))) {
                        const int slot = atomicAdd(&s.q_cnt[r], 1);
                        if (slot < QC) {
                            const int c = (j < 4) ? 4 * tx + j : 64 + 4 * tx + (j - 4);
                            s.q_d[r][slot] = acc[i][j];
                            s.q_i[r][slot] = (int)(col0 + c);
                            pend &= ~(1ull << (i * 8 + j));
                        }
                    }
                }
            }
            __syncthreads();
            if (t < BM) merge_queue<KC>(s, t);
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + (i - 4);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if ((pend & (1ull << (i * 8 + j))) && !(acc[i][j] <= s.thr[r]))
                        pend &= ~(1ull << (i * 8 + j));
            }
        }
    }
    __syncthreads();
    if (t < BM) {
        const int64_t o = ((int64_t)sp * Np + row0 + t) * KC;
        for (int j = 0; j < KC; ++j) {
            cand_d[o + j] = s.list_d[t][j];
            cand_i[o + j] = s.list_i[t][j] == kNoIdx ? -1 : s.list_i[t][j];
        }
    }
}

// Float32 distance tiles for listed query rows (the rows the bfloat16
// certificate left open): rows fb_list[f], f < *count, against every point.
// Both operands are centred on the fly, v = fl(x - mu) -- the float32
// operand the float32 path would hold -- and the norms are its norms.  Work
// items (query row block, column split) are taken persistently, so the
// grid does not depend on the count; lists go to ((split N + f) KC).
template <int KC>
__global__ void __launch_bounds__(KT, 2)
knn_cand_query_kernel(const float* __restrict__ X, int64_t N, int D, int Dp,
                      const float* __restrict__ mu, const float* __restrict__ norms32,
                      const int32_t* __restrict__ fb_list, const long long* count_ptr, int splits,
                      int n_tiles, float* __restrict__ cand_d, int32_t* __restrict__ cand_i) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CandSmem<KC>& s = *reinterpret_cast<CandSmem<KC>*>(smem_raw);
    __shared__ int64_t prow[BM];
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const long long F = *(const volatile long long*)count_ptr;
    const int64_t items = (F + BM - 1) / BM * splits;
    const int nk = Dp / BK;
    const int lr0 = t & 127, lq0 = t >> 7, lq1 = lq0 + 2;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t rb = item / splits;
        const int sp = (int)(item % splits);
        const int tile0 = (int)((int64_t)sp * n_tiles / splits);
        const int tile1 = (int)((int64_t)(sp + 1) * n_tiles / splits);
        __syncthreads();   // the previous item is done with the lists
        if (t < BM) {
            const int64_t f = rb * BM + t;
            const int64_t p = (f < F) ? (int64_t)fb_list[f] : -1;
            prow[t] = p;
            for (int j = 0; j < KC; ++j) { s.list_d[t][j] = kInf; s.list_i[t][j] = kNoIdx; }
            s.q_cnt[t] = 0;
            s.thr[t] = kInf;
            s.nrow[t] = (p >= 0) ? norms32[p] : kInf;
        }
        __syncthreads();
        const int64_t pa_row = prow[lr0];
        for (int tile = tile0; tile < tile1; ++tile) {
            const int64_t col0 = (int64_t)tile * BN;
            __syncthreads();  // previous epilogue finished with ncol / buffers
            if (t < BN) s.ncol[t] = (col0 + t < N) ? norms32[col0 + t] : kInf;
            const int64_t qb_row = (col0 + lr0 < N) ? col0 + lr0 : -1;
            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            float ra[8], rbv[8];
            // 16-byte loads when every row starts on a 16-byte boundary and the
            // four features of a chunk are all inside the row (D % 4 == 0)
            const bool v4 = (D & 3) == 0 && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
            auto fetch = [&](int k0) {
                if (v4) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int d = k0 + 4 * (h == 0 ? lq0 : lq1);
                        const bool in = d < D;
                        const float4 m4 = in ? __ldg(reinterpret_cast<const float4*>(mu + d))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 xa = (pa_row >= 0 && in)
                                              ? __ldg(reinterpret_cast<const float4*>(X + pa_row * D + d))
                                              : m4;
                        const float4 xb = (qb_row >= 0 && in)
                                              ? __ldg(reinterpret_cast<const float4*>(X + qb_row * D + d))
                                              : m4;
                        ra[4 * h + 0] = xa.x - m4.x; ra[4 * h + 1] = xa.y - m4.y;
                        ra[4 * h + 2] = xa.z - m4.z; ra[4 * h + 3] = xa.w - m4.w;
                        rbv[4 * h + 0] = xb.x - m4.x; rbv[4 * h + 1] = xb.y - m4.y;
                        rbv[4 * h + 2] = xb.z - m4.z; rbv[4 * h + 3] = xb.w - m4.w;
                    }
                    return;
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int d = k0 + 4 * (c < 4 ? lq0 : lq1) + (c & 3);
                    const float m = (d < D) ? mu[d] : 0.f;
                    ra[c] = (pa_row >= 0 && d < D) ? X[pa_row * D + d] - m : 0.f;
                    rbv[c] = (qb_row >= 0 && d < D) ? X[qb_row * D + d] - m : 0.f;
                }
            };
            auto stash = [&](int buf) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int kk = 4 * (c < 4 ? lq0 : lq1) + (c & 3);
                    s.As[buf][kk][lr0] = ra[c];
                    s.Bs[buf][kk][lr0] = rbv[c];
                }
            };
            fetch(0);
            stash(0);
            __syncthreads();
            for (int kt = 0; kt < nk; ++kt) {
                const int buf = kt & 1;
                if (kt + 1 < nk) fetch((kt + 1) * BK);
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    const float4 a0 = *reinterpret_cast<const float4*>(&s.As[buf][kk][4 * ty]);
                    const float4 a1 = *reinterpret_cast<const float4*>(&s.As[buf][kk][64 + 4 * ty]);
                    const float4 b0 = *reinterpret_cast<const float4*>(&s.Bs[buf][kk][4 * tx]);
                    const float4 b1 = *reinterpret_cast<const float4*>(&s.Bs[buf][kk][64 + 4 * tx]);
                    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
                }
                if (kt + 1 < nk) stash(buf ^ 1);
                __syncthreads();
            }
            // ---- epilogue: dt = n_p + n_q - 2 dot, filter against the row thresholds
            unsigned long long pend = 0ull;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + (i - 4);
                const int64_t p = prow[r];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = (j < 4) ? 4 * tx + j : 64 + 4 * tx + (j - 4);
                    const int64_t q = col0 + c;
                    const float d = fmaf(-2.f, acc[i][j], s.nrow[r] + s.ncol[c]);
                    acc[i][j] = d;
                    if (p >= 0 && q < N && q != p && d <= s.thr[r]) pend |= 1ull << (i * 8 + j);
                }
            }
            while (__syncthreads_or(pend != 0ull)) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + (i - 4);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (pend & (1ull << (i * 8 + j))) {
                            const int slot = atomicAdd(&s.q_cnt[r], 1);
                            if (slot < QC) {
                                const int c = (j < 4) ? 4 * tx + j : 64 + 4 * tx + (j - 4);
                                s.q_d[r][slot] = acc[i][j];
                                s.q_i[r][slot] = (int)(col0 + c);
                                pend &= ~(1ull << (i * 8 + j));
                            }
                        }
                    }
                }
                __syncthreads();
                if (t < BM) merge_queue<KC>(s, t);
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + (i - 4);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if ((pend & (1ull << (i * 8 + j))) && !(acc[i][j] <= s.thr[r]))
                            pend &= ~(1ull << (i * 8 + j));
                }
            }
        }
        __syncthreads();
        if (t < BM) {
            const int64_t f = rb * BM + t;
            if (f < F) {
                const int64_t o = ((int64_t)sp * N + f) * KC;
                for (int j = 0; j < KC; ++j) {
                    cand_d[o + j] = s.list_d[t][j];
                    cand_i[o + j] = s.list_i[t][j] == kNoIdx ? -1 : s.list_i[t][j];
                }
            }
        }
    }
}

// ------------------------------------------------------ rerank + certificate

// Exact float32 squared distance, lane-strided over features, xor-butterfly
// sum: every lane gets the same bits, and the fallback scan uses the same
// formula so both paths agree bit for bit.
__device__ __forceinline__ float exact_d2(const float* __restrict__ xp,
                                          const float* __restrict__ xq, int D, int lane) {
    float part = 0.f;
    for (int j = lane; j < D; j += 32) {
        const float df = xp[j] - xq[j];
        part = fmaf(df, df, part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    return part;
}

// Rerank + certificate, one warp per row.  Lists hold KC entries each; the
// SEL best of their union (SEL >= KC: several lists of a split together, as
// the two column halves of the 8-warp tensor-core kernel) are the candidates
// whose last one bounds the rest.  Q = false: every row p < N, the lists of
// the candidate kernels at ((list Np + p) KC), failures appended to
// fb_list.  Q = true: the rows fb_in[f], f < *count_in, left open by the
// bfloat16 stage, their float32 query lists at ((split N + f) KC), norms of
// the float32 operand (rho <= u ||v||), failures appended to fb_list /
// *count_out.
template <int KC, bool Q, int E = MAXE, int SEL = KC>
__global__ void __launch_bounds__(256, 4)
knn_rerank_kernel(const float* __restrict__ X, int64_t N, int D, int Dp, int k, int splits,
                  int64_t Np, const float* __restrict__ cand_d, const int32_t* __restrict__ cand_i,
                  const float* __restrict__ norms, const float* __restrict__ rho, float u_acc,
                  int64_t* __restrict__ row_ptr, int32_t* __restrict__ col_idx,
                  float* __restrict__ dist2, int32_t* __restrict__ fb_list, DevState* st,
                  const int32_t* __restrict__ fb_in = nullptr, const long long* count_in = nullptr,
                  long long* count_out = nullptr) {
    __shared__ float s_d[8][32 * E];   // each warp's staged lists (256 threads)
    __shared__ int s_i[8][32 * E];
    __shared__ float s_od[8][SEL];     // and its SEL selected candidates
    __shared__ int s_oi[8][SEL];
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const double u = 5.9604644775390625e-08;  // 2^-24
    const double nmax = (double)__uint_as_float(Q ? st->knn_max_norm32_bits : st->knn_max_norm_bits);
    const double rmax = Q ? u * sqrt(nmax) * (1.0 + 1e-6)
                          : (double)__uint_as_float(st->knn_max_rho_bits);
    const double g = (double)Dp * (double)u_acc;
    const double gam = g / (1.0 - g);
    const double err_exact = 1.01 * (double)(D + 8) * u;
    // float32 copies of the bound's constants for the candidate pruning
    // (margins of 1e-6 .. 1e-5 cover the float rounding of the bounds)
    const float coef_f = (float)((gam + (double)(Dp / 32 + 5) * u) * (1.0 + 1e-6));
    const float rmax_f = (float)(rmax * (1.0 + 1e-6));
    const float snmax_f = (float)(sqrt(nmax) * (1.0 + 1e-6));
    const float keep_f = (float)((1.0 + 2.02 * err_exact) / (1.0 - 2.02 * err_exact) * (1.0 + 1e-5));
    const int64_t rows = Q ? (int64_t)(*(const volatile long long*)count_in) : N;
    const int64_t stride = Q ? N : Np;
    if (!Q && blockIdx.x == 0 && threadIdx.x == 0) row_ptr[N] = N * (int64_t)k;
    for (int64_t f = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < rows;
         f += nw) {
        const int64_t p = Q ? (int64_t)fb_in[f] : f;
        if (!Q && lane == 0) row_ptr[p] = p * (int64_t)k;
        // The splits' lists are sorted by (distance, index) and cover
        // disjoint columns, so the position of an entry in their union is its
        // position in its own list plus, for every other list, the number of
        // that list's entries ordered before it (a binary search; equal keys
        // count from earlier lists only, so positions stay distinct).  Empty
        // slots are (+inf, no index) and follow every entry.
        const int wib = threadIdx.x >> 5;
        float* sd = s_d[wib];
        int* si = s_i[wib];
        const int total = splits * KC;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = lane + 32 * m;
            if (e < total) {
                const int64_t o = ((int64_t)(e / KC) * stride + f) * KC + (e % KC);
                const int i = cand_i[o];
                sd[e] = i >= 0 ? cand_d[o] : kInf;
                si[e] = i >= 0 ? i : kNoIdx;
            }
        }
        __syncwarp();
        int rk[E];   // E >= ceil(splits KC / 32) entries per lane
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = lane + 32 * m;
            rk[m] = 0x7fffffff;
            if (e >= total) continue;
            const float xd = sd[e];
            const int xi = si[e];
            if (xi == kNoIdx) continue;   // empty slots are never selected
            const int l = e / KC;
            int r = 0;
            for (int l2 = 0; l2 < splits; ++l2) {
                int c;
                if (l2 == l) {
                    c = e % KC;
                } else {
                    const float* bd = sd + l2 * KC;
                    const int* bi = si + l2 * KC;
                    const bool eq = l2 < l;
                    c = 0;
#pragma unroll
                    for (int w = KC / 2; w > 0; w >>= 1) {
                        const float od = bd[c + w - 1];
                        const int oi = bi[c + w - 1];
                        if (lex_less(od, oi, xd, xi) || (eq && od == xd && oi == xi)) c += w;
                    }
                    const float od = bd[c];
                    const int oi = bi[c];
                    if (lex_less(od, oi, xd, xi) || (eq && od == xd && oi == xi)) ++c;
                }
                r += c;
            }
            rk[m] = r;
        }
        // the row itself is not a neighbour: entries after it move up one
        int self_rank = 0x7fffffff;
#pragma unroll
        for (int m = 0; m < E; ++m)
            if (lane + 32 * m < total && si[lane + 32 * m] == (int)p) self_rank = rk[m];
        self_rank = __reduce_min_sync(0xffffffffu, self_rank);
        float* od_ = s_od[wib];
        int* oi_ = s_oi[wib];
        int nv = 0;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = lane + 32 * m;
            const int xi = e < total ? si[e] : kNoIdx;
            const bool valid = xi != kNoIdx && xi != (int)p;
            nv += __popc(__ballot_sync(0xffffffffu, valid));
            const int r = rk[m] - (rk[m] > self_rank ? 1 : 0);
            if (valid && r < SEL) {
                od_[r] = sd[e];
                oi_[r] = xi;
            }
        }
        __syncwarp();
        // candidate c lives on lane c % 32, slot c / 32
        constexpr int CPL = (SEL + 31) / 32;
        const int nc = nv < SEL ? nv : SEL;
        int ci[CPL];
        float cd[CPL];
#pragma unroll
        for (int h = 0; h < CPL; ++h) {
            const int c = lane + 32 * h;
            ci[h] = c < nc ? oi_[c] : kNoIdx;
            cd[h] = c < nc ? od_[c] : kInf;
        }
        float T = nc == SEL ? od_[SEL - 1] : kInf;
        __syncwarp();   // read before the next row's lists are staged
        // Lower bound T on dt of every point that is not a candidate: a column
        // a split rejected has dt >= that split's last list entry (when its
        // list is full); an entry of the union left out has dt >= the SEL-th
        // selected one.
        {
            float ts = kInf;
            if (lane < splits) {
                const int64_t o = ((int64_t)lane * stride + f) * KC + (KC - 1);
                if (cand_i[o] >= 0) ts = cand_d[o];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ts = fminf(ts, __shfl_xor_sync(0xffffffffu, ts, o));
            T = fminf(T, ts);
        }
        // Candidates that cannot be among the k nearest need no exact
        // distance.  With |dt - |xt_p - xt_q|^2| <= delta_q =
        // coef (|xt_p| + |xt_q|)^2 and |xt - (x - mu)| <= rho, the exact
        // distance of candidate c = q lies in
        // [lb_c, ub_c] = [(sqrt(dt - delta_q) - rho_p - rho_q)^2,
        // (sqrt(dt + delta_q) + rho_p + rho_q)^2].  Every ub_c is at most the
        // same bound taken with the largest norm and rho of all rows, which
        // grows with dt, and the candidates come in increasing dt, so the
        // k-th smallest ub is at most that bound of candidate k - 1 (U); a
        // candidate whose own lb exceeds U (by more than the float32
        // rounding of the exact sums) is beaten by k candidates whatever the
        // rounding.  Skipped candidates keep an infinite distance, so they
        // rank after every computed one and the k nearest, their distances
        // and the certificate are unchanged.
        unsigned need[CPL];
        {
            const float npf = norms[p];
            const float rp = Q ? 5.9604645e-08f * 1.000001f * sqrtf(npf) : rho[p] * 1.000001f;
            const float snp = sqrtf(npf) * 1.000001f;   // the row's own terms
            const float rr = rp + rmax_f;
            const float snf = snp + snmax_f;
            const float dl = coef_f * snf * snf;
            float U = kInf;
            if (nc >= k) {
                float dkt = kInf;
#pragma unroll
                for (int h = 0; h < CPL; ++h)
                    if ((k - 1) / 32 == h) dkt = __shfl_sync(0xffffffffu, cd[h], (k - 1) % 32);
                const float a = sqrtf(dkt + dl) + rr;
                U = a * a * 1.00001f;
            }
            const float lim = U * keep_f;
#pragma unroll
            for (int h = 0; h < CPL; ++h) {
                bool keep = false;
                if (lane + 32 * h < nc) {
                    const int q = ci[h];
                    const float nqf = norms[q];
                    const float rq = (Q ? 5.9604645e-08f * 1.000001f * sqrtf(nqf) : rho[q] * 1.000001f);
                    const float snq = snp + sqrtf(nqf) * 1.000001f;
                    const float lo = cd[h] - coef_f * snq * snq;
                    const float r = lo > 0.f ? sqrtf(lo) * 0.99999f - (rp + rq) : 0.f;
                    const float lb = r > 0.f ? r * r * 0.99999f : 0.f;
                    keep = !(lb > lim);
                }
                need[h] = __ballot_sync(0xffffffffu, keep);
            }
        }
        // exact float32 distances of the remaining candidates
        const float* xp = X + p * D;
        float myd[CPL];
#pragma unroll
        for (int h = 0; h < CPL; ++h) myd[h] = kInf;
#pragma unroll
        for (int h = 0; h < CPL; ++h) {
            for (unsigned msk = need[h]; msk != 0u; msk &= msk - 1u) {   // warp-uniform
                const int b = __ffs(msk) - 1;
                const int q = __shfl_sync(0xffffffffu, ci[h], b);
                const float d = exact_d2(xp, X + (int64_t)q * D, D, lane);
                if (lane == b) myd[h] = d;
            }
        }
        // rank of each candidate by (exact distance, index) among the
        // computed ones; a skipped one (+inf) ranks after at least k of them
        int rank[CPL];
#pragma unroll
        for (int h = 0; h < CPL; ++h) rank[h] = 0;
#pragma unroll
        for (int hs = 0; hs < CPL; ++hs) {
            for (unsigned msk = need[hs]; msk != 0u; msk &= msk - 1u) {
                const int b = __ffs(msk) - 1;
                const float od = __shfl_sync(0xffffffffu, myd[hs], b);
                const int oi = __shfl_sync(0xffffffffu, ci[hs], b);
#pragma unroll
                for (int h = 0; h < CPL; ++h)
                    if (lex_less(od, oi, myd[h], ci[h])) ++rank[h];
            }
        }
        float dk = kInf;
#pragma unroll
        for (int h = 0; h < CPL; ++h) {
            const bool mine = lane + 32 * h < nc;
            if (mine && rank[h] < k) {
                col_idx[p * k + rank[h]] = ci[h];
                dist2[p * k + rank[h]] = myd[h];
            }
            const unsigned kth = __ballot_sync(0xffffffffu, mine && rank[h] == k - 1);
            if (kth) dk = __shfl_sync(0xffffffffu, myd[h], __ffs(kth) - 1);
        }
        if (lane == 0 && T < kInf) {
            bool ok = false;
            const double np_ = (double)norms[p];
            const double rp = Q ? u * sqrt(np_) * (1.0 + 1e-6) : (double)rho[p];
            const double sn = sqrt(np_) + sqrt(nmax);
            // tile arithmetic (gam), the norms' float32 lane sums and roundings
            const double delta = (gam + (double)(Dp / 32 + 5) * u) * sn * sn;
            const double tt = (double)T - delta;
            if (tt > 0.0) {
                const double root = sqrt(tt) - rp - rmax;
                if (root > 0.0) {
                    const double lb = root * root * (1.0 - 1e-12);
                    ok = (double)dk * (1.0 + 2.02 * err_exact) < lb;
                }
            }
            if (!ok) {
                long long* cnt = Q ? count_out : &st->fallback_count;
                const unsigned long long slot = atomicAdd((unsigned long long*)cnt, 1ull);
                fb_list[slot] = (int32_t)p;
            }
        }
    }
}

// ------------------------------------------------------------ exact fallback

// One block per listed row: 8 warps scan disjoint column subsets keeping a
// register top-k (lane i holds entry i), then warp 0 merges the 8 lists.
__global__ void __launch_bounds__(256)
knn_fallback_kernel(const float* __restrict__ X, int64_t N, int D, int k,
                    const int32_t* __restrict__ fb_list, const long long* count_ptr,
                    int32_t* __restrict__ col_idx, float* __restrict__ dist2) {
    __shared__ float md[8][32];
    __shared__ int mi[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long count = *(const volatile long long*)count_ptr;
    for (long long f = blockIdx.x; f < count; f += gridDim.x) {
        const int64_t p = fb_list[f];
        const float* xp = X + p * D;
        float ld = kInf;
        int li = kNoIdx;
        for (int64_t q = warp; q < N; q += 8) {
            if (q == p) continue;
            const float d = exact_d2(xp, X + q * D, D, lane);
            const float lastd = __shfl_sync(0xffffffffu, ld, k - 1);
            const int lasti = __shfl_sync(0xffffffffu, li, k - 1);
            if (!lex_less(d, (int)q, lastd, lasti)) continue;
            const bool less = lane < k && lex_less(d, (int)q, ld, li);
            const unsigned lm = __ballot_sync(0xffffffffu, less);
            const int pos = __ffs(lm) - 1;
            const float upd = __shfl_up_sync(0xffffffffu, ld, 1);
            const int upi = __shfl_up_sync(0xffffffffu, li, 1);
            if (lane < k) {
                if (lane == pos) { ld = d; li = (int)q; }
                else if (lane > pos) { ld = upd; li = upi; }
            }
        }
        md[warp][lane] = ld;
        mi[warp][lane] = li;
        __syncthreads();
        if (warp == 0) {
            float ed[8];
            int ei[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                ed[m] = lane < k ? md[m][lane] : kInf;
                ei[m] = lane < k ? mi[m][lane] : kNoIdx;
            }
            for (int c = 0; c < k; ++c) {
                float bd = kInf;
                int bi = kNoIdx;
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    if (lex_less(ed[m], ei[m], bd, bi)) { bd = ed[m]; bi = ei[m]; }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float od = __shfl_xor_sync(0xffffffffu, bd, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (lex_less(od, oi, bd, bi)) { bd = od; bi = oi; }
                }
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    if (ei[m] == bi) { ed[m] = kInf; ei[m] = kNoIdx; }
                if (lane == 0) { col_idx[p * k + c] = bi; dist2[p * k + c] = bd; }
            }
        }
        __syncthreads();
    }
}

// Batched exact rescan of the rows that failed the certificate.  A block
// takes R failed rows (their features cached in registers, lane-strided like
// exact_d2) and one column range; each of its 8 warps streams a share of the
// columns once for all R rows, computing every distance with exact_d2's
// arithmetic (same per-lane fmaf order, same butterfly), and keeps a
// register top-k per row (lane i holds entry i).  The 8 warp lists are
// merged in shared memory into one list per (row, column range), written to
// part_d / part_i at slot cs * k of the row's scratch.
template <int R, int DPL>
__global__ void __launch_bounds__(256)
knn_fallback_batch_kernel(const float* __restrict__ X, int64_t N, int D, int k,
                          const int32_t* __restrict__ fb_list, const long long* count_ptr,
                          int col_splits, int64_t slot_stride, float* __restrict__ part_d,
                          int32_t* __restrict__ part_i) {
    __shared__ float md[8][R][32];
    __shared__ int mi[8][R][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long count = *(const volatile long long*)count_ptr;
    const long long nbatch = (count + R - 1) / R;
    const int cs = blockIdx.y;
    const int64_t q0 = (int64_t)cs * N / col_splits, q1 = (int64_t)(cs + 1) * N / col_splits;
    for (long long b = blockIdx.x; b < nbatch; b += gridDim.x) {
        int64_t prow[R];
        float xr[R][DPL];
        float ld[R], lastd[R];
        int li[R], lasti[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long f = b * R + r;
            prow[r] = (f < count) ? (int64_t)fb_list[f] : -1;
#pragma unroll
            for (int t = 0; t < DPL; ++t) {
                const int j = lane + 32 * t;
                xr[r][t] = (prow[r] >= 0 && j < D) ? X[prow[r] * D + j] : 0.f;
            }
            ld[r] = kInf; li[r] = kNoIdx; lastd[r] = kInf; lasti[r] = kNoIdx;
        }
        for (int64_t q = q0 + warp; q < q1; q += 8) {
            float xq[DPL];
#pragma unroll
            for (int t = 0; t < DPL; ++t) {
                const int j = lane + 32 * t;
                xq[t] = (j < D) ? X[q * D + j] : 0.f;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (prow[r] < 0 || q == prow[r]) continue;
                float part = 0.f;
#pragma unroll
                for (int t = 0; t < DPL; ++t) {
                    if (lane + 32 * t < D) {
                        const float df = xr[r][t] - xq[t];
                        part = fmaf(df, df, part);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if (!lex_less(part, (int)q, lastd[r], lasti[r])) continue;
                const bool less = lane < k && lex_less(part, (int)q, ld[r], li[r]);
                const int pos = __ffs(__ballot_sync(0xffffffffu, less)) - 1;
                const float upd = __shfl_up_sync(0xffffffffu, ld[r], 1);
                const int upi = __shfl_up_sync(0xffffffffu, li[r], 1);
                if (lane < k) {
                    if (lane == pos) { ld[r] = part; li[r] = (int)q; }
                    else if (lane > pos) { ld[r] = upd; li[r] = upi; }
                }
                lastd[r] = __shfl_sync(0xffffffffu, ld[r], k - 1);
                lasti[r] = __shfl_sync(0xffffffffu, li[r], k - 1);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            md[warp][r][lane] = lane < k ? ld[r] : kInf;
            mi[warp][r][lane] = lane < k ? li[r] : kNoIdx;
        }
        __syncthreads();
        for (int r = warp; r < R; r += 8) {
            const long long f = b * R + r;
            if (f >= count) continue;
            const int64_t p = fb_list[f];
            float ed[8];
            int ei[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) { ed[m] = md[m][r][lane]; ei[m] = mi[m][r][lane]; }
            for (int c = 0; c < k; ++c) {
                float bd = kInf;
                int bi = kNoIdx;
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    if (lex_less(ed[m], ei[m], bd, bi)) { bd = ed[m]; bi = ei[m]; }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float od = __shfl_xor_sync(0xffffffffu, bd, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (lex_less(od, oi, bd, bi)) { bd = od; bi = oi; }
                }
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    if (ei[m] == bi) { ed[m] = kInf; ei[m] = kNoIdx; }
                if (lane == 0) {
                    part_d[p * slot_stride + (int64_t)cs * k + c] = bd;
                    part_i[p * slot_stride + (int64_t)cs * k + c] = bi;
                }
            }
        }
        __syncthreads();
    }
}

// Merge the col_splits partial lists of every failed row into its k nearest.
__global__ void __launch_bounds__(256)
knn_fallback_merge_kernel(int k, const int32_t* __restrict__ fb_list, const long long* count_ptr,
                          int col_splits, int64_t slot_stride, const float* __restrict__ part_d,
                          const int32_t* __restrict__ part_i, int32_t* __restrict__ col_idx,
                          float* __restrict__ dist2) {
    const int lane = threadIdx.x & 31;
    const long long count = *(const volatile long long*)count_ptr;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t f = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < count;
         f += nw) {
        const int64_t p = fb_list[f];
        float ed[8];
        int ei[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int e = lane + 32 * m;
            ed[m] = kInf;
            ei[m] = kNoIdx;
            if (e < col_splits * k) {
                ed[m] = part_d[p * slot_stride + e];
                ei[m] = part_i[p * slot_stride + e];
            }
        }
        for (int c = 0; c < k; ++c) {
            float bd = kInf;
            int bi = kNoIdx;
#pragma unroll
            for (int m = 0; m < 8; ++m)
                if (lex_less(ed[m], ei[m], bd, bi)) { bd = ed[m]; bi = ei[m]; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float od = __shfl_xor_sync(0xffffffffu, bd, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (lex_less(od, oi, bd, bi)) { bd = od; bi = oi; }
            }
#pragma unroll
            for (int m = 0; m < 8; ++m)
                if (ei[m] == bi) { ed[m] = kInf; ei[m] = kNoIdx; }
            if (lane == 0) { col_idx[p * k + c] = bi; dist2[p * k + c] = bd; }
        }
    }
}

int choose_kc(int k) { return (k + 4 <= 16) ? 16 : 32; }

struct KnnPlan {
    int64_t Np;
    int Dp, kc, splits, row_blocks, n_tiles;
    int ew;      // epilogue warps of the tensor-core kernel (lists per split: ew / 4)
    int lists;   // candidate lists per row: splits x lists per split
    bool bf16;
};

// Column splits for the persistent tensor-core kernel.  Every split restarts
// the rows' candidate lists, so prefer few, long work items (row block x
// split) of at least 8 column tiles: the smallest split count whose last
// round is at least 95 % full, else the best-filled one.
int tc_splits(int row_blocks, int n_tiles, int num_sms, int max_splits) {
    int best = 1;
    double best_eff = -1.0;
    const int s_max = std::max(1, std::min(max_splits, n_tiles / 8));
    for (int s = 1; s <= s_max; ++s) {
        const int64_t items = (int64_t)row_blocks * s;
        const int64_t rounds = (items + num_sms - 1) / num_sms;
        const double eff = (double)items / (double)(rounds * num_sms);
        if (eff >= 0.95) return s;
        if (eff > best_eff + 1e-9) { best_eff = eff; best = s; }
    }
    return best;
}

KnnPlan make_plan(const slk_ctx* ctx, int64_t N, int D, int k, int precision) {
    KnnPlan pl{};
    pl.bf16 = (precision == SLK_KNN_BF16_RERANK);
    // bfloat16 candidates carry a larger rounding error: keep about 5k
    // candidates per row and split so that the certificate still holds for
    // most rows -- for k > 6 two lists of 32 (the column halves of every
    // tile, one per epilogue warp of a pair), whose smaller last entry
    // bounds every rejected column like the last entry of one list of 64
#ifndef SLK_TC_BF16_KC64
#define SLK_TC_BF16_KC64 0
#endif
    pl.kc = pl.bf16 ? ((k <= 6 || !SLK_TC_BF16_KC64) ? 32 : 64) : choose_kc(k);
    pl.ew = (pl.bf16 && k > 6 && pl.kc == 32) ? 8 : 4;
    // the tensor-core tiles read 256-row column tiles: keep them inside the matrix
    pl.Np = (int64_t)align_up((size_t)N, pl.bf16 ? 256 : 128);
    pl.Dp = (int)align_up((size_t)D, pl.bf16 ? 64 : BK);
    pl.row_blocks = (int)(pl.Np / BM);
    pl.n_tiles = (int)(pl.Np / BN);
    const int max_splits = (32 * MAXE) / pl.kc;
    const int cap = 2 * (ctx->num_sms > 0 ? ctx->num_sms : 148);  // resident CTAs
    // smallest split count giving >= 2 waves, then the one with the best wave fill
    int best = 1;
    double best_eff = -1.0;
    for (int s = 1; s <= max_splits && s <= pl.n_tiles; ++s) {
        const int64_t total = (int64_t)pl.row_blocks * s;
        const int64_t waves = (total + cap - 1) / cap;
        double eff = (double)total / (double)(waves * cap);
        if (total < 2 * cap && s < max_splits && s < pl.n_tiles) eff *= 0.5;  // too few CTAs
        if (eff > best_eff + 1e-9) { best_eff = eff; best = s; }
        if (total >= 8 * cap) break;
    }
    pl.splits = best;
    pl.lists = pl.splits;
    if (pl.bf16) {
        const int per = knn_tc_lists_per_split(pl.kc, pl.ew);
        const int tiles_tc = (int)((pl.Np + knn_tc_tile_cols() - 1) / knn_tc_tile_cols());
        pl.splits = tc_splits(pl.row_blocks, tiles_tc, ctx->num_sms > 0 ? ctx->num_sms : 148,
                              max_splits / per);
        pl.lists = pl.splits * per;
    }
    return pl;
}

}  // namespace

size_t knn_ws_bytes(const slk_ctx* ctx, int64_t N, int D, int k, int precision) {
    const KnnPlan pl = make_plan(ctx, N, D, k, precision);
    size_t b = 0;
    b += align_up(sizeof(double) * D, 256);
    b += align_up((pl.bf16 ? 2 : 4) * (size_t)pl.Np * pl.Dp, 256);
    b += 2 * align_up(sizeof(float) * pl.Np, 256);
    b += 2 * align_up(sizeof(float) * (size_t)pl.lists * pl.Np * pl.kc, 256);
    b += align_up(sizeof(float) * pl.Np, 256) + align_up(sizeof(float) * D, 256);   // norms32, mu
    b += align_up(sizeof(int32_t) * N, 256);                                         // second list
    b += align_up(sizeof(int32_t) * (size_t)N, 256);
    return b + 4096;
}

slk_status knn_cand_bf16_launch(slk_ctx* ctx, const __nv_bfloat16* xt, const float* norms,
                                int64_t N, int Dp, int64_t Np, int kc, int ew, int splits,
                                float* cand_d, int32_t* cand_i, unsigned int* err_flag);

namespace {

// Column sums, mu and the prepared rows on the context's stream; 16-byte
// loads where the row layout and the summation bound allow them.
slk_status launch_prep(slk_ctx* ctx, const float* X, int64_t N, int D, int Dp, int64_t Np,
                       double* colsum, float* mu, float* xt32, __nv_bfloat16* xt16,
                       float* norms, float* rho, float* norms32, DevState* st) {
    cudaStream_t s = ctx->stream;
    const bool v4 = D % 4 == 0 && Dp >= 128 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(mu) & 15) == 0;
    int gy = (int)((N + 511) / 512);   // 64 rows per thread
    if (gy > 8192) gy = 8192;
    if (gy < 1) gy = 1;
    const int groups = v4 ? D / 4 : D;
    const dim3 cgrid((unsigned)((groups + 31) / 32), (unsigned)gy);
    if (v4) col_sum_kernel<4><<<cgrid, dim3(32, 8), 0, s>>>(X, N, D, colsum);
    else col_sum_kernel<1><<<cgrid, dim3(32, 8), 0, s>>>(X, N, D, colsum);
    mu_kernel<<<(D + 255) / 256, 256, 0, s>>>(colsum, N, D, mu);
    SLK_LAUNCH_CHECK(ctx, "col_sum_kernel");
    int64_t pg = (Np + 7) / 8;
    if (pg > (int64_t)ctx->num_sms * 64) pg = (int64_t)ctx->num_sms * 64;
    const int to_bf16 = xt16 != nullptr ? 1 : 0;
    if (v4)
        prep_rows_kernel<4><<<(unsigned)pg, 256, 0, s>>>(X, N, D, Dp, Np, mu, to_bf16, xt32, xt16,
                                                         norms, rho, norms32, st);
    else
        prep_rows_kernel<1><<<(unsigned)pg, 256, 0, s>>>(X, N, D, Dp, Np, mu, to_bf16, xt32, xt16,
                                                         norms, rho, norms32, st);
    SLK_LAUNCH_CHECK(ctx, "prep_rows_kernel");
    return SLK_OK;
}

}  // namespace

slk_status knn_prep_fp32_launch(slk_ctx* ctx, const float* X, int64_t N, int D, int Dp, int64_t Np,
                                double* colsum, float* mu, float* xt, float* norms, float* rho,
                                DevState* st) {
    cudaStream_t s = ctx->stream;
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(colsum, 0, sizeof(double) * D, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->knn_max_norm_bits, 0, 2 * sizeof(unsigned int), s));
    SLK_COUNT_LAUNCH(ctx, 2);
    return launch_prep(ctx, X, N, D, Dp, Np, colsum, mu, xt, nullptr, norms, rho, nullptr, st);
}

slk_status knn_graph_launch(slk_ctx* ctx, const float* X, int64_t N, int D, int k,
                            int precision, int64_t* row_ptr, int32_t* col_idx, float* dist2,
                            void* ws, DevState* st) {
    const KnnPlan pl = make_plan(ctx, N, D, k, precision);
    WsCarver wc(ws);
    double* colsum = wc.take<double>(D);
    void* xt = wc.take<unsigned char>((pl.bf16 ? 2 : 4) * (size_t)pl.Np * pl.Dp);
    float* norms = wc.take<float>(pl.Np);
    float* rho = wc.take<float>(pl.Np);
    float* cand_d = wc.take<float>((size_t)pl.lists * pl.Np * pl.kc);
    int32_t* cand_i = wc.take<int32_t>((size_t)pl.lists * pl.Np * pl.kc);
    int32_t* fb = wc.take<int32_t>(N);
    float* norms32 = wc.take<float>(pl.Np);
    float* mu = wc.take<float>(D);
    int32_t* fb2 = wc.take<int32_t>(N);
    cudaStream_t s = ctx->stream;

    SLK_CUDA_TRY(ctx, cudaMemsetAsync(colsum, 0, sizeof(double) * D, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->fallback_count, 0, sizeof(long long), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->knn_max_norm_bits, 0, 3 * sizeof(unsigned int), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->knn_max_norm32_bits, 0, sizeof(unsigned int), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->fallback2_count, 0, sizeof(long long), s));
    {
        PhaseScope ps(ctx, SLK_PHASE_KNN_PREP);
        SLK_COUNT_LAUNCH(ctx, 3);
        const slk_status r = launch_prep(ctx, X, N, D, pl.Dp, pl.Np, colsum, mu,
                                         pl.bf16 ? nullptr : (float*)xt,
                                         pl.bf16 ? (__nv_bfloat16*)xt : nullptr, norms, rho,
                                         pl.bf16 ? norms32 : nullptr, st);
        if (r != SLK_OK) return r;
    }
    float u_acc;
    {
    PhaseScope ps(ctx, SLK_PHASE_KNN_CAND);
    SLK_COUNT_LAUNCH(ctx, 1);
    if (pl.bf16) {
        slk_status r = knn_cand_bf16_launch(ctx, (const __nv_bfloat16*)xt, norms, N, pl.Dp, pl.Np,
                                            pl.kc, pl.ew, pl.splits, cand_d, cand_i, &st->knn_error);
        if (r != SLK_OK) return r;
        // 2^-23: products exact, each accumulator add off by at most one ulp
        // (truncating adds); an assumption about the tensor-core accumulator
        u_acc = 1.1920928955078125e-07f;
    } else {
        u_acc = 5.9604644775390625e-08f;  // 2^-24
#define SLK_CAND(KC_)                                                                         \
    {                                                                                         \
        auto kern = knn_cand_fp32_kernel<KC_>;                                                \
        const int smem = (int)sizeof(CandSmem<KC_>);                                          \
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)); \
        kern<<<dim3((unsigned)pl.row_blocks, (unsigned)pl.splits), KT, smem, s>>>(            \
            (const float*)xt, norms, N, pl.Dp, pl.n_tiles, pl.Np, cand_d, cand_i);            \
    }
        if (pl.kc == 16) SLK_CAND(16) else SLK_CAND(32)
#undef SLK_CAND
        SLK_LAUNCH_CHECK(ctx, "knn_cand_fp32_kernel");
    }
    }
    {
        PhaseScope ps(ctx, SLK_PHASE_KNN_RERANK);
        SLK_COUNT_LAUNCH(ctx, 1);
        int64_t grid = (N + 7) / 8;
        if (grid > (int64_t)ctx->num_sms * 16) grid = (int64_t)ctx->num_sms * 16;
        // entries per lane: the splits' lists, KC each, over 32 lanes
        const int per_lane = (pl.lists * pl.kc + 31) / 32;
#define SLK_RERANK(KC_, E_)                                                                   \
    do {                                                                                      \
        if (pl.kc == 32 && pl.ew == 8)                                                        \
            knn_rerank_kernel<32, false, E_, 64><<<(unsigned)grid, 256, 0, s>>>(              \
                X, N, D, pl.Dp, k, pl.lists, pl.Np, cand_d, cand_i, norms, rho, u_acc, row_ptr, \
                col_idx, dist2, fb, st);                                                      \
        else                                                                                  \
            knn_rerank_kernel<KC_, false, E_><<<(unsigned)grid, 256, 0, s>>>(                 \
                X, N, D, pl.Dp, k, pl.lists, pl.Np, cand_d, cand_i, norms, rho, u_acc, row_ptr, \
                col_idx, dist2, fb, st);                                                      \
    } while (0)
#define SLK_RERANK_E(KC_)                                                                     \
    if (per_lane <= 4) SLK_RERANK(KC_, 4);                                                    \
    else if (per_lane <= 8) SLK_RERANK(KC_, 8);                                               \
    else SLK_RERANK(KC_, 16);
        if (pl.kc == 16) { SLK_RERANK_E(16) }
        else if (pl.kc == 32) { SLK_RERANK_E(32) }
        else { SLK_RERANK_E(64) }
#undef SLK_RERANK_E
#undef SLK_RERANK
        SLK_LAUNCH_CHECK(ctx, "knn_rerank_kernel");
    }
    {
        PhaseScope ps(ctx, SLK_PHASE_KNN_FALLBACK);
        // rows still open after this stage: the exact scan reads them from
        // (list, count); with bfloat16 candidates a float32 stage comes first
        const int32_t* exact_list = fb;
        const long long* exact_count = &st->fallback_count;
        if (pl.bf16) {
            // float32 distance tiles of the open rows against every point, then
            // the rerank under the float32 certificate; its failures go on
            // float32 lists of at least 2k candidates (the gap between the k-th and the
            // last decides the certificate)
            const int kcq = (2 * k <= 16) ? 16 : 32;
            int qsplits = (int)std::min<int64_t>(8, (int64_t)pl.lists * pl.kc / kcq);
            if (qsplits < 1) qsplits = 1;
            const int n_tiles = (int)((N + BN - 1) / BN);
            SLK_COUNT_LAUNCH(ctx, 2);
            const unsigned qgrid = (unsigned)(ctx->num_sms * 2);
#define SLK_QCAND(KC_)                                                                        \
    {                                                                                         \
        auto kern = knn_cand_query_kernel<KC_>;                                               \
        const int smem = (int)sizeof(CandSmem<KC_>);                                          \
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)); \
        kern<<<qgrid, KT, smem, s>>>(X, N, D, pl.Dp, mu, norms32, fb, &st->fallback_count,    \
                                     qsplits, n_tiles, cand_d, cand_i);                       \
    }
            if (kcq == 16) SLK_QCAND(16) else SLK_QCAND(32)
#undef SLK_QCAND
            SLK_LAUNCH_CHECK(ctx, "knn_cand_query_kernel");
            const unsigned rgrid = (unsigned)(ctx->num_sms * 4);   // grid-stride over the open rows
            const float u32 = 5.9604644775390625e-08f;
            if (kcq == 16)
                knn_rerank_kernel<16, true><<<rgrid, 256, 0, s>>>(
                    X, N, D, pl.Dp, k, qsplits, N, cand_d, cand_i, norms32, nullptr, u32, row_ptr,
                    col_idx, dist2, fb2, st, fb, &st->fallback_count, &st->fallback2_count);
            else
                knn_rerank_kernel<32, true><<<rgrid, 256, 0, s>>>(
                    X, N, D, pl.Dp, k, qsplits, N, cand_d, cand_i, norms32, nullptr, u32, row_ptr,
                    col_idx, dist2, fb2, st, fb, &st->fallback_count, &st->fallback2_count);
            SLK_LAUNCH_CHECK(ctx, "knn_rerank_kernel (float32 stage)");
            exact_list = fb2;
            exact_count = &st->fallback2_count;
        }
        // partial lists of the batched rescan reuse the row's candidate
        // scratch: lists * KC slots per row, of which col_splits * k are used
        const int64_t slot_stride = (int64_t)pl.lists * pl.kc;
        int cs = (int)(slot_stride / k);
        if (cs > 8) cs = 8;
        const int dpl = (D + 31) / 32;
        if (cs >= 1 && dpl <= 32) {
            SLK_COUNT_LAUNCH(ctx, 2);
            // the rescan scratch is laid out per row (slot_stride entries), so
            // it may reuse cand_d / cand_i once the rerank is done with them
            dim3 grid((unsigned)((ctx->num_sms * 2 + cs - 1) / cs), (unsigned)cs);
#define SLK_FB(R_, DPL_)                                                                     \
    knn_fallback_batch_kernel<R_, DPL_><<<grid, 256, 0, s>>>(X, N, D, k, exact_list, exact_count, \
                                                             cs, slot_stride, cand_d, cand_i)
            if (dpl <= 4) SLK_FB(16, 4);
            else if (dpl <= 8) SLK_FB(8, 8);
            else if (dpl <= 16) SLK_FB(4, 16);
            else SLK_FB(2, 32);
#undef SLK_FB
            SLK_LAUNCH_CHECK(ctx, "knn_fallback_batch_kernel");
            knn_fallback_merge_kernel<<<(unsigned)(ctx->num_sms * 2), 256, 0, s>>>(
                k, exact_list, exact_count, cs, slot_stride, cand_d, cand_i, col_idx, dist2);
            SLK_LAUNCH_CHECK(ctx, "knn_fallback_merge_kernel");
        } else {
        SLK_COUNT_LAUNCH(ctx, 1);
        knn_fallback_kernel<<<(unsigned)(ctx->num_sms * 2), 256, 0, s>>>(X, N, D, k, exact_list,
                                                                         exact_count, col_idx, dist2);
        SLK_LAUNCH_CHECK(ctx, "knn_fallback_kernel");
        }
    }
    return SLK_OK;
}
