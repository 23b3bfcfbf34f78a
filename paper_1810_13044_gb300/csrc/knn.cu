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
slk_status knn_cand_split_launch(slk_ctx* ctx, const __nv_bfloat16* qh, const __nv_bfloat16* ql,
                                 const float* qnorm, int64_t Fcap, const long long* rows_dev,
                                 const __nv_bfloat16* xh, const __nv_bfloat16* xl,
                                 const float* norms, int64_t N, int Dp, int64_t Np, int ew,
                                 int splits, float* cand_d, int32_t* cand_i,
                                 unsigned int* err_flag);

namespace {

constexpr int BM = 128, BN = 128, BK = 16, KT = 256;
constexpr int QC = 32;      // per-row insertion queue of the candidate kernel
constexpr int MAXE = 16;    // merge entries per lane (splits * KC <= 512)
#define kInf __int_as_float(0x7f800000)
constexpr int kNoIdx = 0x7fffffff;

__device__ __forceinline__ bool lex_less(float d, int i, float d2, int i2) {
    return d < d2 || (d == d2 && i < i2);
}

// Open rows at or below this count skip the float32 tiles (whose 128-row
// blocks they would leave mostly empty) and go to the exact scan.
constexpr long long kExactDirectRows = 256;

// Longest row the wide exact rescan stages in shared memory (bytes).
constexpr size_t kWideSmemMax = 200 * 1024;

// Column splits of the float32 stage for F open rows: as many as a buffer of
// cap floats holds at F rows per list of KC, at most 16 (the rerank stages
// 16 lists of 32 per row).  Host and device compute it from the same count.
__host__ __device__ __forceinline__ int query_splits(long long F, long long cap, int kc) {
    if (F <= 0) return 1;
    long long sp = cap / (F * (long long)kc);
    if (sp > 16) sp = 16;
    if (sp < 1) sp = 1;
    return (int)sp;
}

// Column splits of the exact scan for F rows: partial lists of k entries per
// (row, split), at most 1024 splits (a few open rows still fill the GPU), as
// many as cap entries hold.
__host__ __device__ __forceinline__ int exact_splits(long long F, long long cap, int k) {
    if (F <= 0) return 1;
    long long sp = cap / (F * (long long)k);
    if (sp > 1024) sp = 1024;
    if (sp < 1) sp = 1;
    return (int)sp;
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

// rho >= sqrt(e2 bound) + u sqrt(v2 bound) and kappa >= rho / ||v|| with
// ||v|| >= sqrt(v2 / bound), from the float pairs (eh, el) = e2 and (vh, vl)
// = v2 (lane sums of e^2 and v^2); every step rounded toward the bound.
// kappa = 0 when v2 = 0 (then e = 0 and rho = 0), +inf when ||v|| underflows.
__device__ __forceinline__ void rho_kappa(float eh, float el, float vh, float vl, float bound_u,
                                          float& rho, float& kappa) {
    const float e2 = __fadd_ru(eh, el), v2 = __fadd_ru(vh, vl);
    const float t1 = __fsqrt_ru(__fmul_ru(e2, bound_u));
    const float t2 = __fmul_ru(5.9604644775390625e-08f, __fsqrt_ru(__fmul_ru(v2, bound_u)));
    rho = __fadd_ru(t1, t2);
    const float vlo = __fsqrt_rd(__fdiv_rd(__fadd_rd(vh, vl), bound_u));
    kappa = (v2 > 0.f) ? (vlo > 0.f ? __fdiv_ru(rho, vlo) : __int_as_float(0x7f800000)) : 0.f;
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
// The row maxima go to st with one atomic per block, with that of
// kappa_p = rho_p / ||v_p|| (||v_p|| from below), so that rho_q <= kappa ||v_q||
// for every row.
// aug (nullable, Np x 32 bfloat16): the folded-norm columns of the
// tensor-core tiles, [1, 1, 1, a_p, 0...] in columns 0..15 and [a_p, 1, 1, 1,
// 0...] in 16..31, a_p = (t1, t2, t3) the bfloat16 terms of -norms[p] / 2
// (t1 = bf16(x), t2 = bf16(x - t1), t3 = bf16(x - t1 - t2), each difference
// exact in float32, so t1 + t2 + t3 is within 2^-24 (1.02) |x| of x); a
// padding row has a_p = (-inf, 0, 0).
template <int V>
__global__ void __launch_bounds__(256)
prep_rows_kernel(const float* __restrict__ X, int64_t N, int D, int Dp,
                 int64_t Np, const float* __restrict__ mu, int to_bf16,
                 float* __restrict__ xt32, __nv_bfloat16* __restrict__ xt16,
                 float* __restrict__ norms, float* __restrict__ rho,
                 float* __restrict__ norms32, __nv_bfloat16* __restrict__ aug, DevState* st) {
    __shared__ unsigned bmax_n, bmax_r, bmax_n32, bmax_k;
    if (threadIdx.x == 0) { bmax_n = 0u; bmax_r = 0u; bmax_n32 = 0u; bmax_k = 0u; }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    // 1 + (Dp/32 + 2) u, rounded up: the lane sums' relative error bound
    const float bound_u = __double2float_ru(1.0 + (double)(Dp / 32 + 2) * 5.9604644775390625e-08);
    unsigned my_n = 0u, my_r = 0u, my_n32 = 0u, my_k = 0u;
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
            // the pair sums rounded to nearest (norms), up and down (bounds);
            // float32 with directed rounding keeps the bounds off the slow
            // float64 pipe
            const float nf = __fadd_rn(nh, nl);
            float rf, kf;
            rho_kappa(eh, el, vh, vl, bound_u, rf, kf);
            // padding rows get an infinite norm: no distance to them can pass a filter
            norms[p] = (p < N) ? nf : __int_as_float(0x7f800000);
            rho[p] = rf;
            const float n32 = __fadd_rn(vh, vl);   // ||v||^2 of the float32 operand v
            if (norms32) norms32[p] = (p < N) ? n32 : __int_as_float(0x7f800000);
            if (p < N) {
                my_n = max(my_n, __float_as_uint(nf));
                my_r = max(my_r, __float_as_uint(rf));
                my_n32 = max(my_n32, __float_as_uint(n32));
                my_k = max(my_k, __float_as_uint(kf));
            }
        }
        if (aug) {
            // lanes 0..3 write 8 columns each (16-byte stores)
            const float nfa = __shfl_sync(0xffffffffu, __fadd_rn(nh, nl), 0);
            if (lane < 4) {
                const float x = -0.5f * nfa;
                const __nv_bfloat16 t1 = __float2bfloat16_rn(x);
                const float r1 = x - __bfloat162float(t1);
                const __nv_bfloat16 t2 = __float2bfloat16_rn(r1);
                const __nv_bfloat16 t3 = __float2bfloat16_rn(r1 - __bfloat162float(t2));
                const __nv_bfloat16 one = __float2bfloat16_rn(1.f), zero = __float2bfloat16_rn(0.f);
                const __nv_bfloat16 a1 = (p < N) ? t1 : __float2bfloat16_rn(-__int_as_float(0x7f800000));
                const __nv_bfloat16 a2 = (p < N) ? t2 : zero, a3 = (p < N) ? t3 : zero;
                __nv_bfloat16 w[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) w[q] = zero;
                if (lane == 0) {          // columns 0..7: 1, 1, 1, a1, a2, a3
                    w[0] = one; w[1] = one; w[2] = one; w[3] = a1; w[4] = a2; w[5] = a3;
                } else if (lane == 2) {   // columns 16..23: a1, a2, a3, 1, 1, 1
                    w[0] = a1; w[1] = a2; w[2] = a3; w[3] = one; w[4] = one; w[5] = one;
                }
                *reinterpret_cast<uint4*>(aug + p * 32 + 8 * lane) = *reinterpret_cast<const uint4*>(w);
            }
        }
    }
    if (lane == 0) {
        atomicMax(&bmax_n, my_n);
        atomicMax(&bmax_r, my_r);
        atomicMax(&bmax_n32, my_n32);
        atomicMax(&bmax_k, my_k);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&st->knn_max_norm_bits, bmax_n);
        atomicMax(&st->knn_max_rho_bits, bmax_r);
        atomicMax(&st->knn_max_norm32_bits, bmax_n32);
        atomicMax(&st->knn_max_kappa_bits, bmax_k);
    }
}

// ------------------------------------------------- two-term bfloat16 operand

// One warp per padded row p < Np, for the rows the bfloat16 certificate
// leaves open (nothing runs when *open_count is 0): with v = fl(x - mu) and
// h = bf16(v) (the candidate operand xt), the second term l = bf16(v - h)
// (v - h is exact), so that s = h + l carries 16 significant bits of v:
//   xl[p]      = l,
//   norms_s[p] = ||s||^2 (s = h + l is exact in float32: l either equals
//                v - h, then s = v, or has its last bit above v's),
//   rho_s[p]  >= ||s - (x_p - mu)||, from e = s - v (exact) and
//                |v - (x - mu)| <= u |v|, as for the other operands.
// Sums as in prep_rows_kernel (the same lane split and float-pair butterfly,
// so the same summation bound); row maxima to st.
template <int V>
__global__ void __launch_bounds__(256)
prep_split_kernel(const float* __restrict__ X, int64_t N, int D, int Dp, int64_t Np,
                  const float* __restrict__ mu, const long long* __restrict__ open_count,
                  __nv_bfloat16* __restrict__ xl, float* __restrict__ norms_s,
                  float* __restrict__ rho_s, DevState* st) {
    if (*open_count == 0) return;
    __shared__ unsigned bmax_n, bmax_r, bmax_k;
    if (threadIdx.x == 0) { bmax_n = 0u; bmax_r = 0u; bmax_k = 0u; }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    // 1 + (Dp/32 + 2) u, rounded up: the lane sums' relative error bound
    const float bound_u = __double2float_ru(1.0 + (double)(Dp / 32 + 2) * 5.9604644775390625e-08);
    unsigned my_n = 0u, my_r = 0u, my_k = 0u;
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < Np;
         p += nw) {
        float n2v[V], e2v[V], v2v[V];
#pragma unroll
        for (int q = 0; q < V; ++q) { n2v[q] = 0.f; e2v[q] = 0.f; v2v[q] = 0.f; }
#pragma unroll 4
        for (int j = lane * V; j < Dp; j += 32 * V) {
            float v[V];
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
            __nv_bfloat16 lb[V];
            float sv[V];
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const float h = __bfloat162float(__float2bfloat16_rn(v[q]));
                lb[q] = __float2bfloat16_rn(v[q] - h);
                sv[q] = h + __bfloat162float(lb[q]);
            }
            if constexpr (V == 4) {
                __nv_bfloat162 b01, b23;
                b01.x = lb[0]; b01.y = lb[1]; b23.x = lb[2]; b23.y = lb[3];
                uint2 w;
                w.x = *reinterpret_cast<const unsigned*>(&b01);
                w.y = *reinterpret_cast<const unsigned*>(&b23);
                *reinterpret_cast<uint2*>(xl + p * Dp + j) = w;
            } else {
                xl[p * Dp + j] = lb[0];
            }
#pragma unroll
            for (int q = 0; q < V; ++q) {
                n2v[q] = fmaf(sv[q], sv[q], n2v[q]);
                const float e = sv[q] - v[q];
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
        float nh = n2, nl = 0.f, eh = e2, el = 0.f, vh = v2, vl = 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fpair_add(nh, nl, __shfl_xor_sync(0xffffffffu, nh, o), __shfl_xor_sync(0xffffffffu, nl, o));
            fpair_add(eh, el, __shfl_xor_sync(0xffffffffu, eh, o), __shfl_xor_sync(0xffffffffu, el, o));
            fpair_add(vh, vl, __shfl_xor_sync(0xffffffffu, vh, o), __shfl_xor_sync(0xffffffffu, vl, o));
        }
        if (lane == 0) {
            const float nf = __fadd_rn(nh, nl);
            float rf, kf;
            rho_kappa(eh, el, vh, vl, bound_u, rf, kf);
            norms_s[p] = (p < N) ? nf : __int_as_float(0x7f800000);
            rho_s[p] = rf;
            if (p < N) {
                my_n = max(my_n, __float_as_uint(nf));
                my_r = max(my_r, __float_as_uint(rf));
                my_k = max(my_k, __float_as_uint(kf));
            }
        }
    }
    if (lane == 0) {
        atomicMax(&bmax_n, my_n);
        atomicMax(&bmax_r, my_r);
        atomicMax(&bmax_k, my_k);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&st->knn_max_norm_s_bits, bmax_n);
        atomicMax(&st->knn_max_rho_s_bits, bmax_r);
        atomicMax(&st->knn_max_kappa_s_bits, bmax_k);
    }
}

// Query rows of the two-term stage: row f < min(*count, Fcap) of qh / ql /
// qnorm is row fb[f] of xh / xl / norms_s; the rest of its 128-row block is
// zero with an infinite norm.  One warp per row, 16-byte copies (Dp is a
// multiple of 64).
__global__ void __launch_bounds__(256)
gather_split_kernel(const __nv_bfloat16* __restrict__ xh, const __nv_bfloat16* __restrict__ xl,
                    const float* __restrict__ norms_s, int Dp, const int32_t* __restrict__ fb,
                    const long long* __restrict__ count, int64_t Fcap,
                    __nv_bfloat16* __restrict__ qh, __nv_bfloat16* __restrict__ ql,
                    float* __restrict__ qnorm) {
    long long c = *count;
    if (c > Fcap) c = Fcap;
    const int64_t rows = (c + 127) / 128 * 128;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int n16 = Dp / 8;   // 16-byte words per row
    for (int64_t f = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < rows;
         f += nw) {
        const bool live = f < c;
        const int64_t p = live ? (int64_t)fb[f] : 0;
        const uint4* sh = reinterpret_cast<const uint4*>(xh + p * Dp);
        const uint4* sl = reinterpret_cast<const uint4*>(xl + p * Dp);
        uint4* dh = reinterpret_cast<uint4*>(qh + f * Dp);
        uint4* dl = reinterpret_cast<uint4*>(ql + f * Dp);
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (int j = lane; j < n16; j += 32) {
            dh[j] = live ? __ldg(sh + j) : z;
            dl[j] = live ? __ldg(sl + j) : z;
        }
        if (lane == 0) qnorm[f] = live ? norms_s[p] : __int_as_float(0x7f800000);
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

// Float32 distance tiles for listed query rows (the rows the earlier
// certificates left open): rows fb_list[f], f < F = *count, against every
// point.  Both operands are centred on the fly, v = fl(x - mu) -- the float32
// operand the float32 path would hold -- and the norms are its norms.  Work
// items (query row block, column split) are taken persistently, so the grid
// does not depend on the count; the split count is query_splits(F, cap, KC)
// and lists go to ((split F + f) KC).  Nothing runs for F <=
// kExactDirectRows (those rows go to the exact scan).
template <int KC>
__global__ void __launch_bounds__(KT, 2)
knn_cand_query_kernel(const float* __restrict__ X, int64_t N, int D, int Dp,
                      const float* __restrict__ mu, const float* __restrict__ norms32,
                      const int32_t* __restrict__ fb_list, const long long* count_ptr,
                      long long cap, int n_tiles, float* __restrict__ cand_d,
                      int32_t* __restrict__ cand_i) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CandSmem<KC>& s = *reinterpret_cast<CandSmem<KC>*>(smem_raw);
    __shared__ int64_t prow[BM];
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const long long F = *(const volatile long long*)count_ptr;
    if (F <= kExactDirectRows) return;
    const int splits = query_splits(F, cap, KC);
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
                const int64_t o = ((int64_t)sp * F + f) * KC;
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

// Feature-loop unrolling of the rerank's exact distances (gathers in flight;
// measured at 1e6 x 128: 4 gives 10.0 ms against 9.0 for 1)
#ifndef SLK_RERANK_UNROLL
#define SLK_RERANK_UNROLL 1
#endif
constexpr int kRerankUnroll = SLK_RERANK_UNROLL;

// Rerank + certificate, one warp per row.  Lists hold KC entries each; the
// SEL best of their union (SEL >= KC: several lists of a split together, as
// the two column halves of the 8-warp tensor-core kernel) are the candidates
// whose last one bounds the rest.  gam bounds the error of a tile's dot
// product relative to |xt_p| |xt_q| (with the norms' roundings added here).
//   MODE 0: every row p < N, the lists of the candidate kernels at
//           ((list Np + p) KC), failures appended to fb_list.
//   MODE 1: the rows fb_in[f], f < F = *count_in, their float32 query lists
//           at ((split F + f) KC), query_splits(F, Np, KC) of them (Np: the
//           list buffer's capacity in floats), norms of the float32 operand
//           (rho <= u ||v||), failures appended to fb_list / *count_out; for
//           F <= kExactDirectRows every row is appended (no lists were made).
//   MODE 2: the rows fb_in[f], f < *count_in, their two-term bfloat16 query
//           lists at ((list Np + f) KC) for f < Np (Np: the query stage's
//           row capacity), norms and rho of the two-term operand; the rows
//           from Np on, and the failures, appended to fb_list / *count_out.
template <int KC, int MODE, int E = MAXE, int SEL = KC>
__global__ void __launch_bounds__(256, 4)
knn_rerank_kernel(const float* __restrict__ X, int64_t N, int D, int Dp, int k, int splits_in,
                  int64_t Np, const float* __restrict__ cand_d, const int32_t* __restrict__ cand_i,
                  const float* __restrict__ norms, const float* __restrict__ rho, double gam,
                  int64_t* __restrict__ row_ptr, int32_t* __restrict__ col_idx,
                  float* __restrict__ dist2, int32_t* __restrict__ fb_list, DevState* st,
                  const int32_t* __restrict__ fb_in = nullptr, const long long* count_in = nullptr,
                  long long* count_out = nullptr) {
    constexpr bool Q = MODE != 0;
    __shared__ float s_d[8][32 * E];   // each warp's staged lists (256 threads)
    __shared__ int s_i[8][32 * E];
    __shared__ float s_od[8][SEL];     // and its SEL selected candidates
    __shared__ int s_oi[8][SEL];
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const double u = 5.9604644775390625e-08;  // 2^-24
    const double nmax = (double)__uint_as_float(
        MODE == 0 ? st->knn_max_norm_bits : MODE == 1 ? st->knn_max_norm32_bits : st->knn_max_norm_s_bits);
    const double rmax = MODE == 1 ? u * sqrt(nmax) * (1.0 + 1e-6)
                                  : (double)__uint_as_float(MODE == 0 ? st->knn_max_rho_bits
                                                                      : st->knn_max_rho_s_bits);
    // rho_q <= kappa ||v_q|| for every row q
    const double kappa = MODE == 1 ? u * (1.0 + 1e-5)
                                   : (double)__uint_as_float(MODE == 0 ? st->knn_max_kappa_bits
                                                                       : st->knn_max_kappa_s_bits);
    const double err_exact = 1.01 * (double)(D + 8) * u;
    // float32 copies of the bound's constants for the candidate pruning
    // (margins of 1e-6 .. 1e-5 cover the float rounding of the bounds)
    const float coef_f = (float)((gam + (double)(Dp / 32 + 5) * u) * (1.0 + 1e-6));
    const float rmax_f = (float)(rmax * (1.0 + 1e-6));
    const float snmax_f = (float)(sqrt(nmax) * (1.0 + 1e-6));
    const float keep_f = (float)((1.0 + 2.02 * err_exact) / (1.0 - 2.02 * err_exact) * (1.0 + 1e-5));
    const int64_t rows = Q ? (int64_t)(*(const volatile long long*)count_in) : N;
    const int splits = MODE == 1 ? query_splits(rows, Np, KC) : splits_in;
    const int64_t stride = MODE == 1 ? rows : Np;
    if (MODE == 1 && rows <= kExactDirectRows) {
        // too few rows for the float32 tiles: all of them to the exact scan
        for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < rows;
             f += (int64_t)gridDim.x * blockDim.x) {
            const unsigned long long slot = atomicAdd((unsigned long long*)count_out, 1ull);
            fb_list[slot] = fb_in[f];
        }
        return;
    }
    if (!Q && blockIdx.x == 0 && threadIdx.x == 0) row_ptr[N] = N * (int64_t)k;
    for (int64_t f = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < rows;
         f += nw) {
        const int64_t p = Q ? (int64_t)fb_in[f] : f;
        if (MODE == 2 && f >= Np) {
            // beyond the query stage's capacity: on to the next stage
            if (lane == 0) {
                const unsigned long long slot = atomicAdd((unsigned long long*)count_out, 1ull);
                fb_list[slot] = (int32_t)p;
            }
            continue;
        }
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
            const float rp = MODE == 1 ? 5.9604645e-08f * 1.000001f * sqrtf(npf) : rho[p] * 1.000001f;
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
                    const float rq = (MODE == 1 ? 5.9604645e-08f * 1.000001f * sqrtf(nqf) : rho[q] * 1.000001f);
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
            if (D > 256) {
                // long rows: a candidate's own loads already overlap
                for (unsigned msk = need[h]; msk != 0u; msk &= msk - 1u) {   // warp-uniform
                    const int b = __ffs(msk) - 1;
                    const int q = __shfl_sync(0xffffffffu, ci[h], b);
                    const float d = exact_d2(xp, X + (int64_t)q * D, D, lane);
                    if (lane == b) myd[h] = d;
                }
                continue;
            }
            // short rows: four candidates at a time, their row gathers overlap;
            // each one's sum has exact_d2's per-lane order and butterfly (the
            // same bits)
            unsigned msk = need[h];   // warp-uniform
            while (msk != 0u) {
                int b[4], q[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    b[c] = msk != 0u ? __ffs(msk) - 1 : -1;
                    if (msk != 0u) msk &= msk - 1u;
                    q[c] = __shfl_sync(0xffffffffu, ci[h], b[c] < 0 ? 0 : b[c]);
                }
                float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll kRerankUnroll
                for (int j = lane; j < D; j += 32) {
                    const float a = xp[j];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (b[c] >= 0) {
                            const float df = a - X[(int64_t)q[c] * D + j];
                            part[c] = fmaf(df, df, part[c]);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part[c] += __shfl_xor_sync(0xffffffffu, part[c], o);
                    if (b[c] >= 0 && lane == b[c]) myd[h] = part[c];
                }
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
            const double rp = MODE == 1 ? u * sqrt(np_) * (1.0 + 1e-6) : (double)rho[p];
            // every point q outside the candidates must be farther than
            // K = dk (1 + 2.02 err_exact), the k-th candidate's exact distance
            // inflated by its rounding.  With y = x - mu, a q with |y_q| >=
            // |y_p| + sqrt(K) is (|y_q| - |y_p| >= sqrt(K)); any other has
            // |y_q| < R = |xt_p| + rho_p + sqrt(K), hence rho_q <= kappa
            // ||v_q|| <= kappa (1 + u) R and |xt_q| < R + rho_q.  Its
            // distance is at least (sqrt(T - delta_q) - rho_p - rho_q)^2 with
            // delta_q = coef (|xt_p| + |xt_q|)^2 (tile arithmetic gam, the
            // norms' float32 lane sums and roundings), |xt_q| and rho_q taken
            // at the smaller of these bounds and the largest norm and rho of
            // all rows.
            const double K = (double)dk * (1.0 + 2.02 * err_exact);
            const double sp = sqrt(np_) * (1.0 + (double)(Dp / 32 + 4) * u);
            const double R = (sp + rp + sqrt(K)) * (1.0 + 1e-9);
            const double rq = fmin(rmax, kappa * (1.0 + u) * R * (1.0 + 1e-9));
            const double sn = fmin(sqrt(np_) + sqrt(nmax), sp + R + rq);
            const double delta = (gam + (double)(Dp / 32 + 5) * u) * sn * sn;
            const double tt = (double)T - delta;
            if (tt > 0.0) {
                const double root = sqrt(tt) - rp - rq;
                if (root > 0.0) {
                    const double lb = root * root * (1.0 - 1e-12);
                    ok = K < lb;
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

// Exact rescan for long rows (D above the 32 x 32 features the batched form
// keeps in registers): work items (one failed row, one of cs =
// exact_splits(F, cap, k) column ranges) taken persistently, so that a few
// rows still spread over every SM.  The row's features are staged in shared
// memory; each of the 8 warps streams a share of the range, computing every
// distance with exact_d2 (the same per-lane order and butterfly) and keeping
// a register top-k (lane i holds entry i); the 8 lists are merged into the
// (row, range) partial list at ((f cs + range) k), as the batched form does.
__global__ void __launch_bounds__(256)
knn_fallback_wide_kernel(const float* __restrict__ X, int64_t N, int D, int k,
                         const int32_t* __restrict__ fb_list, const long long* count_ptr,
                         long long cap, float* __restrict__ part_d, int32_t* __restrict__ part_i) {
    extern __shared__ float xs[];   // D floats: the row's features
    __shared__ float md[8][32];
    __shared__ int mi[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long count = *(const volatile long long*)count_ptr;
    const int col_splits = exact_splits(count, cap, k);
    for (long long item = blockIdx.x; item < count * col_splits; item += gridDim.x) {
        const long long f = item / col_splits;
        const int cs = (int)(item % col_splits);
        const int64_t p = fb_list[f];
        const int64_t q0 = (int64_t)cs * N / col_splits, q1 = (int64_t)(cs + 1) * N / col_splits;
        __syncthreads();   // the previous item is done with xs and md / mi
        for (int j = threadIdx.x; j < D; j += blockDim.x) xs[j] = X[p * D + j];
        __syncthreads();
        float ld = kInf;
        int li = kNoIdx;
        for (int64_t q = q0 + warp; q < q1; q += 8) {
            if (q == p) continue;
            const float d = exact_d2(xs, X + q * D, D, lane);
            const float lastd = __shfl_sync(0xffffffffu, ld, k - 1);
            const int lasti = __shfl_sync(0xffffffffu, li, k - 1);
            if (!lex_less(d, (int)q, lastd, lasti)) continue;
            const bool less = lane < k && lex_less(d, (int)q, ld, li);
            const int pos = __ffs(__ballot_sync(0xffffffffu, less)) - 1;
            const float upd = __shfl_up_sync(0xffffffffu, ld, 1);
            const int upi = __shfl_up_sync(0xffffffffu, li, 1);
            if (lane < k) {
                if (lane == pos) { ld = d; li = (int)q; }
                else if (lane > pos) { ld = upd; li = upi; }
            }
        }
        md[warp][lane] = lane < k ? ld : kInf;
        mi[warp][lane] = lane < k ? li : kNoIdx;
        __syncthreads();
        if (warp == 0) {
            float ed[8];
            int ei[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) { ed[m] = md[m][lane]; ei[m] = mi[m][lane]; }
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
                    part_d[(f * col_splits + cs) * k + c] = bd;
                    part_i[(f * col_splits + cs) * k + c] = bi;
                }
            }
        }
    }
}

// Batched exact rescan of the rows that failed the certificate.  Work items
// (R failed rows, one of cs = exact_splits(F, cap, k) column ranges) are
// taken persistently, so the grid does not depend on the count F.  The R
// rows' features are cached in registers, lane-strided like exact_d2; each
// of the block's 8 warps streams a share of the column range once for all R
// rows, computing every distance with exact_d2's arithmetic (same per-lane
// fmaf order, same butterfly), and keeps a register top-k per row (lane i
// holds entry i).  The 8 warp lists are merged in shared memory into one
// list per (row, column range), written to part_d / part_i at
// ((f cs + range) k).
template <int R, int DPL>
__global__ void __launch_bounds__(256)
knn_fallback_batch_kernel(const float* __restrict__ X, int64_t N, int D, int k,
                          const int32_t* __restrict__ fb_list, const long long* count_ptr,
                          long long cap, float* __restrict__ part_d,
                          int32_t* __restrict__ part_i) {
    __shared__ float md[8][R][32];
    __shared__ int mi[8][R][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long count = *(const volatile long long*)count_ptr;
    const long long nbatch = (count + R - 1) / R;
    const int col_splits = exact_splits(count, cap, k);
    for (long long item = blockIdx.x; item < nbatch * col_splits; item += gridDim.x) {
        const long long b = item / col_splits;
        const int cs = (int)(item % col_splits);
        const int64_t q0 = (int64_t)cs * N / col_splits, q1 = (int64_t)(cs + 1) * N / col_splits;
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
        // the next column's features are loaded while this one is summed
        float xq[DPL];
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            const int j = lane + 32 * t;
            xq[t] = (q0 + warp < q1 && j < D) ? X[(q0 + warp) * D + j] : 0.f;
        }
        for (int64_t q = q0 + warp; q < q1; q += 8) {
            float xn[DPL];
#pragma unroll
            for (int t = 0; t < DPL; ++t) {
                const int j = lane + 32 * t;
                xn[t] = (q + 8 < q1 && j < D) ? X[(q + 8) * D + j] : 0.f;
            }
            // every row's lane sums, then their butterflies side by side (the
            // R chains overlap), then the insertions; each sum in exact_d2's order
            float part[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                part[r] = 0.f;
#pragma unroll
                for (int t = 0; t < DPL; ++t) {
                    if (lane + 32 * t < D) {
                        const float df = xr[r][t] - xq[t];
                        part[r] = fmaf(df, df, part[r]);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int r = 0; r < R; ++r) part[r] += __shfl_xor_sync(0xffffffffu, part[r], o);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (prow[r] < 0 || q == prow[r]) continue;
                if (!lex_less(part[r], (int)q, lastd[r], lasti[r])) continue;
                const bool less = lane < k && lex_less(part[r], (int)q, ld[r], li[r]);
                const int pos = __ffs(__ballot_sync(0xffffffffu, less)) - 1;
                const float upd = __shfl_up_sync(0xffffffffu, ld[r], 1);
                const int upi = __shfl_up_sync(0xffffffffu, li[r], 1);
                if (lane < k) {
                    if (lane == pos) { ld[r] = part[r]; li[r] = (int)q; }
                    else if (lane > pos) { ld[r] = upd; li[r] = upi; }
                }
                lastd[r] = __shfl_sync(0xffffffffu, ld[r], k - 1);
                lasti[r] = __shfl_sync(0xffffffffu, li[r], k - 1);
            }
#pragma unroll
            for (int t = 0; t < DPL; ++t) xq[t] = xn[t];
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
                    part_d[(f * col_splits + cs) * k + c] = bd;
                    part_i[(f * col_splits + cs) * k + c] = bi;
                }
            }
        }
        __syncthreads();
    }
}

// Merge the partial lists of every failed row (cs = exact_splits(F, cap, k)
// of k entries at ((f cs) k)) into its k nearest: chunks of 7 entries per
// lane beside the running k best (lane i holds entry i), k rounds of a warp
// minimum per chunk.
__global__ void __launch_bounds__(256)
knn_fallback_merge_kernel(int k, const int32_t* __restrict__ fb_list, const long long* count_ptr,
                          long long cap, const float* __restrict__ part_d,
                          const int32_t* __restrict__ part_i, int32_t* __restrict__ col_idx,
                          float* __restrict__ dist2) {
    const int lane = threadIdx.x & 31;
    const long long count = *(const volatile long long*)count_ptr;
    const int col_splits = exact_splits(count, cap, k);
    const int total = col_splits * k;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t f = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < count;
         f += nw) {
        const int64_t p = fb_list[f];
        const float* pd = part_d + f * total;
        const int32_t* pi = part_i + f * total;
        float bestd = kInf;   // lane i < k: the i-th best so far
        int besti = kNoIdx;
        for (int e0 = 0; e0 < total; e0 += 7 * 32) {
            float ed[8];
            int ei[8];
            ed[7] = bestd;
            ei[7] = besti;
#pragma unroll
            for (int m = 0; m < 7; ++m) {
                const int e = e0 + lane + 32 * m;
                ed[m] = e < total ? pd[e] : kInf;
                ei[m] = e < total ? pi[e] : kNoIdx;
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
                // the winner is unique (distinct indices): remove it where it sits
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    if (ei[m] == bi && ed[m] == bd) { ed[m] = kInf; ei[m] = kNoIdx; }
                if (lane == c) { bestd = bd; besti = bi; }
            }
        }
        if (lane < k) { col_idx[p * k + lane] = besti; dist2[p * k + lane] = bestd; }
    }
}

int choose_kc(int k) { return (k + 4 <= 16) ? 16 : 32; }

struct KnnPlan {
    int64_t Np;
    int Dp, kc, splits, row_blocks, n_tiles;
    int ew;      // epilogue warps of the tensor-core kernel (lists per split: ew / 4)
    int lists;   // candidate lists per row: splits x lists per split
    bool bf16;
    bool aug;    // tensor-core tiles with the norms folded into one more K slice
    // two-term stage (bfloat16 and N >= kTwoTermMinRows): row capacity (a
    // multiple of 128), column splits and lists (of 32) per row
    bool two_term;
    int64_t fcap;
    int ssplits, slists;
};

// Rows the two-term tensor-core stage takes at most (fewer at large D, see
// make_plan); the open rows beyond it go to the float32 stage.
constexpr int64_t kSplitRowCap = 65536;
// Below this many points the open rows go straight to the float32 stage (its
// tiles over N points are cheap there, and the two-term stage's four launches
// would cost more than they save: the batched form runs many such graphs).
constexpr int64_t kTwoTermMinRows = 100000;

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
    // where the tiles' epilogue outweighs their MMAs (small D), fold the
    // norms into the MMAs: the epilogue then reads no norms and takes no
    // barrier per tile
#ifndef SLK_TC_AUG_MAX_DP
#define SLK_TC_AUG_MAX_DP 256
#endif
    // the tensor-core tiles read 256-row column tiles: keep them inside the matrix
    pl.Np = (int64_t)align_up((size_t)N, pl.bf16 ? 256 : 128);
    pl.Dp = (int)align_up((size_t)D, pl.bf16 ? 64 : BK);
    pl.aug = pl.bf16 && pl.kc == 32 && pl.Dp <= SLK_TC_AUG_MAX_DP;
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
        // the open rows are few: split the columns as far as the rerank's
        // staging (32 MAXE entries per row) and 8 tiles per item allow
        // at most 65536 rows, and query operands (h and l) of at most 64 MiB
        const int64_t by_mem = std::max<int64_t>(128, ((int64_t)1 << 24) / pl.Dp / 128 * 128);
        pl.fcap = std::min<int64_t>(std::min<int64_t>((int64_t)align_up((size_t)N, 128), kSplitRowCap),
                                    by_mem);
        pl.ssplits = std::max(1, std::min((32 * MAXE) / (32 * per), tiles_tc / 8));
        pl.slists = pl.ssplits * per;
        pl.two_term = N >= kTwoTermMinRows;
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
    if (pl.aug) b += align_up(2 * 32 * (size_t)pl.Np, 256);   // folded-norm columns
    if (pl.bf16 && pl.two_term) {
        // two-term stage: xl, norms_s, rho_s, query rows (h, l, norms), lists
        b += align_up(2 * (size_t)pl.Np * pl.Dp, 256) + 2 * align_up(sizeof(float) * pl.Np, 256);
        b += 2 * align_up(2 * (size_t)pl.fcap * pl.Dp, 256) + align_up(sizeof(float) * pl.fcap, 256);
        b += 2 * align_up(sizeof(float) * (size_t)pl.slists * pl.fcap * 32, 256);
    }
    if (pl.bf16) b += align_up(sizeof(int32_t) * (size_t)N, 256);   // third list
    return b + 4096;
}

slk_status knn_cand_bf16_launch(slk_ctx* ctx, const __nv_bfloat16* xt, const float* norms,
                                const __nv_bfloat16* aug, int64_t N, int Dp, int64_t Np, int kc,
                                int ew, int splits, float* cand_d, int32_t* cand_i,
                                unsigned int* err_flag, unsigned long long* sweep);

namespace {

// Column sums, mu and the prepared rows on the context's stream; 16-byte
// loads where the row layout and the summation bound allow them.
slk_status launch_prep(slk_ctx* ctx, const float* X, int64_t N, int D, int Dp, int64_t Np,
                       double* colsum, float* mu, float* xt32, __nv_bfloat16* xt16,
                       float* norms, float* rho, float* norms32, __nv_bfloat16* aug, DevState* st) {
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
                                                         norms, rho, norms32, aug, st);
    else
        prep_rows_kernel<1><<<(unsigned)pg, 256, 0, s>>>(X, N, D, Dp, Np, mu, to_bf16, xt32, xt16,
                                                         norms, rho, norms32, aug, st);
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
    return launch_prep(ctx, X, N, D, Dp, Np, colsum, mu, xt, nullptr, norms, rho, nullptr, nullptr, st);
}

slk_status knn_graph_launch(slk_ctx* ctx, const float* X, int64_t N, int D, int k,
                            int precision, int64_t* row_ptr, int32_t* col_idx, float* dist2,
                            void* ws, DevState* st) {
    const KnnPlan pl = make_plan(ctx, N, D, k, precision);
    ctx->knn_last_bf16 = pl.bf16;
    ctx->knn_last_two_term = pl.bf16 && pl.two_term;
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
    // two-term stage
    const bool tt = pl.bf16 && pl.two_term;
    const size_t nd_s = tt ? (size_t)pl.Np * pl.Dp : 0, np_s = tt ? (size_t)pl.Np : 0;
    const size_t fd_s = tt ? (size_t)pl.fcap * pl.Dp : 0, f_s = tt ? (size_t)pl.fcap : 0;
    __nv_bfloat16* xl16 = wc.take<__nv_bfloat16>(nd_s);
    float* norms_s = wc.take<float>(np_s);
    float* rho_s = wc.take<float>(np_s);
    __nv_bfloat16* qh = wc.take<__nv_bfloat16>(fd_s);
    __nv_bfloat16* ql = wc.take<__nv_bfloat16>(fd_s);
    float* qnorm = wc.take<float>(f_s);
    float* scand_d = wc.take<float>(tt ? (size_t)pl.slists * pl.fcap * 32 : 0);
    int32_t* scand_i = wc.take<int32_t>(tt ? (size_t)pl.slists * pl.fcap * 32 : 0);
    int32_t* fb3 = wc.take<int32_t>(pl.bf16 ? (size_t)N : 0);
    __nv_bfloat16* aug = wc.take<__nv_bfloat16>(pl.aug ? 32 * (size_t)pl.Np : 0);
    cudaStream_t s = ctx->stream;

    SLK_CUDA_TRY(ctx, cudaMemsetAsync(colsum, 0, sizeof(double) * D, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->fallback_count, 0, sizeof(long long), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->knn_max_norm_bits, 0, 3 * sizeof(unsigned int), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->knn_max_norm32_bits, 0, sizeof(unsigned int), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->fallback2_count, 0, sizeof(long long), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->knn_max_norm_s_bits, 0, 4 * sizeof(unsigned int), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->fallback3_count, 0, sizeof(long long), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->knn_sweep, 0, sizeof(unsigned long long), s));
    {
        PhaseScope ps(ctx, SLK_PHASE_KNN_PREP);
        SLK_COUNT_LAUNCH(ctx, 3);
        const slk_status r = launch_prep(ctx, X, N, D, pl.Dp, pl.Np, colsum, mu,
                                         pl.bf16 ? nullptr : (float*)xt,
                                         pl.bf16 ? (__nv_bfloat16*)xt : nullptr, norms, rho,
                                         pl.bf16 ? norms32 : nullptr, pl.aug ? aug : nullptr, st);
        if (r != SLK_OK) return r;
    }
    float u_acc;   // rounding unit of a tile's dot-product accumulation
    {
    PhaseScope ps(ctx, SLK_PHASE_KNN_CAND);
    SLK_COUNT_LAUNCH(ctx, 1);
    if (pl.bf16) {
        slk_status r = knn_cand_bf16_launch(ctx, (const __nv_bfloat16*)xt, norms,
                                            pl.aug ? aug : nullptr, N, pl.Dp, pl.Np, pl.kc, pl.ew,
                                            pl.splits, cand_d, cand_i, &st->knn_error,
                                            &st->knn_sweep);
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
        // folded norms: 6 more products a dot, and the aug terms' magnitudes
        // (about (n_p + n_q) / 2) join the products' sum: 2 |p| |q| + n_p +
        // n_q = (|p| + |q|)^2, so the bound keeps its form with a 1.01 factor
        const double g = (double)(pl.Dp + (pl.aug ? 6 : 0)) * (double)u_acc;
        const double gam = (pl.aug ? 1.01 : 1.0) * g / (1.0 - g);
#define SLK_RERANK(KC_, E_)                                                                   \
    do {                                                                                      \
        if (pl.kc == 32 && pl.ew == 8)                                                        \
            knn_rerank_kernel<32, 0, E_, 64><<<(unsigned)grid, 256, 0, s>>>(                  \
                X, N, D, pl.Dp, k, pl.lists, pl.Np, cand_d, cand_i, norms, rho, gam, row_ptr,   \
                col_idx, dist2, fb, st);                                                      \
        else                                                                                  \
            knn_rerank_kernel<KC_, 0, E_><<<(unsigned)grid, 256, 0, s>>>(                     \
                X, N, D, pl.Dp, k, pl.lists, pl.Np, cand_d, cand_i, norms, rho, gam, row_ptr,   \
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
            // the float32 stage's input and its failures (for the exact scan)
            const int32_t* f32_in = fb;
            const long long* f32_cnt = &st->fallback_count;
            if (pl.two_term) {
            f32_in = fb2;
            f32_cnt = &st->fallback2_count;
            // (a) two-term bfloat16 tiles of the open rows on the tensor cores
            // (h . h + h . l + l . h of s = h + l, about 16 significant bits
            // of v), the rerank under their certificate; its failures, and
            // open rows beyond the stage's capacity, go on to (b)
            const bool v4 = D % 4 == 0 && pl.Dp >= 128 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                            (reinterpret_cast<uintptr_t>(mu) & 15) == 0;
            int64_t pg = (pl.Np + 7) / 8;
            if (pg > (int64_t)ctx->num_sms * 64) pg = (int64_t)ctx->num_sms * 64;
            SLK_COUNT_LAUNCH(ctx, 4);
            if (v4)
                prep_split_kernel<4><<<(unsigned)pg, 256, 0, s>>>(X, N, D, pl.Dp, pl.Np, mu,
                                                                  &st->fallback_count, xl16, norms_s,
                                                                  rho_s, st);
            else
                prep_split_kernel<1><<<(unsigned)pg, 256, 0, s>>>(X, N, D, pl.Dp, pl.Np, mu,
                                                                  &st->fallback_count, xl16, norms_s,
                                                                  rho_s, st);
            SLK_LAUNCH_CHECK(ctx, "prep_split_kernel");
            int64_t gg = (pl.fcap + 7) / 8;
            if (gg > (int64_t)ctx->num_sms * 16) gg = (int64_t)ctx->num_sms * 16;
            gather_split_kernel<<<(unsigned)gg, 256, 0, s>>>((const __nv_bfloat16*)xt, xl16, norms_s,
                                                            pl.Dp, fb, &st->fallback_count, pl.fcap,
                                                            qh, ql, qnorm);
            SLK_LAUNCH_CHECK(ctx, "gather_split_kernel");
            slk_status r = knn_cand_split_launch(ctx, qh, ql, qnorm, pl.fcap, &st->fallback_count,
                                                 (const __nv_bfloat16*)xt, xl16, norms_s, N, pl.Dp,
                                                 pl.Np, pl.ew, pl.ssplits, scand_d, scand_i,
                                                 &st->knn_error);
            if (r != SLK_OK) return r;
            {
                // dot products of 3 Dp bfloat16 products (2^-23 accumulator
                // unit, as above), |h|, |l| within 1.004 |s| and 0.0040 |s|,
                // plus the dropped l . l term (at most 1.016 2^-16 |s_p| |s_q|)
                const double g3 = 3.0 * (double)pl.Dp * 1.1920928955078125e-07;
                const double gam_s = 1.02 * g3 / (1.0 - g3) + 1.02 * 1.52587890625e-05;
                const unsigned rgrid = (unsigned)(ctx->num_sms * 4);
                const int per_lane = (pl.slists * 32 + 31) / 32;
#define SLK_RERANK_S(E_, SEL_)                                                                \
    knn_rerank_kernel<32, 2, E_, SEL_><<<rgrid, 256, 0, s>>>(                                 \
        X, N, D, pl.Dp, k, pl.slists, pl.fcap, scand_d, scand_i, norms_s, rho_s, gam_s, row_ptr, \
        col_idx, dist2, fb2, st, fb, &st->fallback_count, &st->fallback2_count)
                if (pl.ew == 8) {
                    if (per_lane <= 8) SLK_RERANK_S(8, 64);
                    else SLK_RERANK_S(16, 64);
                } else {
                    if (per_lane <= 8) SLK_RERANK_S(8, 32);
                    else SLK_RERANK_S(16, 32);
                }
#undef SLK_RERANK_S
                SLK_LAUNCH_CHECK(ctx, "knn_rerank_kernel (two-term stage)");
            }
            }
            // (b) float32 distance tiles of the rows still open against every
            // point, then the rerank under the float32 certificate; its
            // failures go on float32 lists of at least 2k candidates (the gap
            // between the k-th and the last decides the certificate)
            const int kcq = (2 * k <= 16) ? 16 : 32;
            // column splits chosen on the device from the count (query_splits)
            const long long qcap = (long long)pl.lists * pl.Np * pl.kc;
            const int n_tiles = (int)((N + BN - 1) / BN);
            SLK_COUNT_LAUNCH(ctx, 2);
            const unsigned qgrid = (unsigned)(ctx->num_sms * 2);
#define SLK_QCAND(KC_)                                                                        \
    {                                                                                         \
        auto kern = knn_cand_query_kernel<KC_>;                                               \
        const int smem = (int)sizeof(CandSmem<KC_>);                                          \
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)); \
        kern<<<qgrid, KT, smem, s>>>(X, N, D, pl.Dp, mu, norms32, f32_in, f32_cnt, qcap,      \
                                     n_tiles, cand_d, cand_i);                                \
    }
            if (kcq == 16) SLK_QCAND(16) else SLK_QCAND(32)
#undef SLK_QCAND
            SLK_LAUNCH_CHECK(ctx, "knn_cand_query_kernel");
            const unsigned rgrid = (unsigned)(ctx->num_sms * 4);   // grid-stride over the open rows
            const double g32 = (double)pl.Dp * 5.9604644775390625e-08;
            const double gam32 = g32 / (1.0 - g32);
            if (kcq == 16)
                knn_rerank_kernel<16, 1><<<rgrid, 256, 0, s>>>(
                    X, N, D, pl.Dp, k, 0, qcap, cand_d, cand_i, norms32, nullptr, gam32, row_ptr,
                    col_idx, dist2, fb3, st, f32_in, f32_cnt, &st->fallback3_count);
            else
                knn_rerank_kernel<32, 1><<<rgrid, 256, 0, s>>>(
                    X, N, D, pl.Dp, k, 0, qcap, cand_d, cand_i, norms32, nullptr, gam32, row_ptr,
                    col_idx, dist2, fb3, st, f32_in, f32_cnt, &st->fallback3_count);
            SLK_LAUNCH_CHECK(ctx, "knn_rerank_kernel (float32 stage)");
            exact_list = fb3;
            exact_count = &st->fallback3_count;
        }
        // the batched rescan's partial lists reuse the candidate buffer
        // (its lists are read by now): cs column ranges of k entries for each
        // of the F open rows, cs chosen on the device from F
        const long long cap = (long long)pl.lists * pl.Np * pl.kc;
        const int dpl = (D + 31) / 32;
        if (dpl <= 32) {
            SLK_COUNT_LAUNCH(ctx, 2);
            const unsigned grid = (unsigned)(ctx->num_sms * 2);
#define SLK_FB(R_, DPL_)                                                                     \
    knn_fallback_batch_kernel<R_, DPL_><<<grid, 256, 0, s>>>(X, N, D, k, exact_list, exact_count, \
                                                             cap, cand_d, cand_i)
            if (dpl <= 4) SLK_FB(16, 4);
            else if (dpl <= 8) SLK_FB(8, 8);
            else if (dpl <= 16) SLK_FB(4, 16);
            else SLK_FB(2, 32);
#undef SLK_FB
            SLK_LAUNCH_CHECK(ctx, "knn_fallback_batch_kernel");
            knn_fallback_merge_kernel<<<(unsigned)(ctx->num_sms * 2), 256, 0, s>>>(
                k, exact_list, exact_count, cap, cand_d, cand_i, col_idx, dist2);
            SLK_LAUNCH_CHECK(ctx, "knn_fallback_merge_kernel");
        } else if ((size_t)D * sizeof(float) <= kWideSmemMax) {
            // long rows: staged in shared memory, (row, column range) items
            SLK_COUNT_LAUNCH(ctx, 2);
            const int smem = (int)((size_t)D * sizeof(float));
            SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(knn_fallback_wide_kernel,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            knn_fallback_wide_kernel<<<(unsigned)(ctx->num_sms * 4), 256, smem, s>>>(
                X, N, D, k, exact_list, exact_count, cap, cand_d, cand_i);
            SLK_LAUNCH_CHECK(ctx, "knn_fallback_wide_kernel");
            knn_fallback_merge_kernel<<<(unsigned)(ctx->num_sms * 2), 256, 0, s>>>(
                k, exact_list, exact_count, cap, cand_d, cand_i, col_idx, dist2);
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
