// Starting modes (Section 4.2): the initial assignment of every point to its
// nearest seed, then for each cluster the mode definition of Eq. (1) with
// that one-hot z:
//   m_l = argmax_{y in X} f_l(y),  f_l(y) = sum_{p: c(p) = l} k(x_p, y),
// k the Gaussian kernel, ties to the smaller index; an empty cluster keeps
// its seed.  f_l at every point is a dense N x |cluster| sum:
//   seed_assign_kernel   c(p) by float32 chunk sums of (x - s)^2 in float64
//   label_count / label_scan / label_scatter
//                        stable counting sort of the points by cluster
//                        (perm, offsets), deterministic
//   density_tile_kernel  128 x 128 float32 distance tiles of the centred
//                        data by the norm expansion, one cluster's columns
//                        per work item, exp in the epilogue, per-row sums of
//                        8 kernel values in float32 added in float64
//   density_bound_kernel / density_cand_kernel
//                        f^_l(y) = the float64 sum of the items of cluster l;
//                        the tiles' rounding bounds give |d^2 - d2| <= delta_y,
//                        so f_l(y) lies in f^_l(y) exp(+-eta_y); every y whose
//                        upper bound reaches the largest lower bound is a
//                        candidate (the exact maximiser always is one)
//   density_exact_kernel f_l of each candidate from float32 differences
//                        (squares in float32 chunks of 8, float64 sums); the
//                        largest, ties to the smaller index, is the mode
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "slk_internal.cuh"

namespace {

constexpr int DBM = 128, DBN = 128, DBK = 16, DT = 256;
constexpr int kSortChunk = 1024;  // points per block of the counting sort

// ------------------------------------------------------------- assignment

// Block: 32 points x all L seeds, features staged 32 at a time (as the
// unary kernel).  Thread t owns point t % 32 and seeds t / 32 + 8 j.
template <int LPT>
__global__ void __launch_bounds__(256)
seed_assign_kernel(const float* __restrict__ X, int64_t N, int D, const int32_t* __restrict__ seeds,
                   int L, int32_t* __restrict__ assign) {
    extern __shared__ float sm[];
    float* xs = sm;                   // [32][33]
    float* ss = xs + 32 * 33;         // [L][33]
    double* dd = reinterpret_cast<double*>(ss + L * 33 + (L & 1));  // [32][L]
    __shared__ int srow[SLK_MAX_L];
    const int t = threadIdx.x, pl = t % 32, lb = t / 32;
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    for (int l = t; l < L; l += 256) srow[l] = seeds[l];
    double acc[LPT];
#pragma unroll
    for (int j = 0; j < LPT; ++j) acc[j] = 0.0;
    __syncthreads();
    for (int d0 = 0; d0 < D; d0 += 32) {
        const int dc = min(32, D - d0);
        for (int i = t; i < 32 * 32; i += 256) {
            const int r = i / 32, c = i % 32;
            xs[r * 33 + c] = (p0 + r < N && c < dc) ? X[(p0 + r) * D + d0 + c] : 0.f;
        }
        for (int i = t; i < L * 32; i += 256) {
            const int r = i / 32, c = i % 32;
            ss[r * 33 + c] = (c < dc) ? X[(int64_t)srow[r] * D + d0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int l = lb + 8 * j;
            if (l < L) {
                float part = 0.f;
                for (int c = 0; c < dc; ++c) {
                    const float df = xs[pl * 33 + c] - ss[l * 33 + c];
                    part = fmaf(df, df, part);
                }
                acc[j] += (double)part;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        const int l = lb + 8 * j;
        if (l < L) dd[pl * L + l] = acc[j];
    }
    __syncthreads();
    if (t < 32 && p0 + t < N) {
        int best = 0;
        double bd = dd[t * L];
        for (int l = 1; l < L; ++l)
            if (dd[t * L + l] < bd) { bd = dd[t * L + l]; best = l; }
        assign[p0 + t] = best;
    }
}

// ------------------------------------------------------ stable counting sort

__global__ void label_count_kernel(const int32_t* __restrict__ lab, int64_t N, int L,
                                   int32_t* __restrict__ counts) {
    extern __shared__ int cnt[];
    for (int l = threadIdx.x; l < L; l += blockDim.x) cnt[l] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kSortChunk;
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x)
        if (b0 + i < N) atomicAdd(&cnt[lab[b0 + i]], 1);
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) counts[(int64_t)blockIdx.x * L + l] = cnt[l];
}

// One block: base[b][l] = off[l] + sum_{b' < b} counts[b'][l]; off[L] = N.
__global__ void label_scan_kernel(const int32_t* __restrict__ counts, int nb, int L,
                                  int64_t* __restrict__ base, int64_t* __restrict__ off) {
    __shared__ int64_t tot[SLK_MAX_L + 1];
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        int64_t s = 0;
        for (int b = 0; b < nb; ++b) s += counts[(int64_t)b * L + l];
        tot[l] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int l = 0; l < L; ++l) {
            const int64_t c = tot[l];
            tot[l] = run;
            off[l] = run;
            run += c;
        }
        off[L] = run;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        int64_t run = tot[l];
        for (int b = 0; b < nb; ++b) {
            base[(int64_t)b * L + l] = run;
            run += counts[(int64_t)b * L + l];
        }
    }
}

// Each point's rank among the points of its cluster that come before it
// (warp match masks + per-warp counts), so perm lists every cluster in
// increasing point order.  256 threads, one point per thread and round.
__global__ void __launch_bounds__(256)
label_scatter_kernel(const int32_t* __restrict__ lab, int64_t N, int L,
                     const int64_t* __restrict__ base, int32_t* __restrict__ perm) {
    extern __shared__ int sh[];
    int* run = sh;            // [L] placed so far in this block
    int* wc = sh + L;         // [8][L] per-warp counts of the round
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int l = t; l < L; l += 256) run[l] = 0;
    const int64_t b0 = (int64_t)blockIdx.x * kSortChunk;
    for (int r0 = 0; r0 < kSortChunk; r0 += 256) {
        for (int i = t; i < 8 * L; i += 256) wc[i] = 0;
        __syncthreads();
        const int64_t p = b0 + r0 + t;
        const bool ok = p < N;
        const int l = ok ? lab[p] : -1;
        const unsigned mm = __match_any_sync(0xffffffffu, l);
        const int rin = __popc(mm & ((1u << lane) - 1u));
        if (ok && rin == 0) wc[w * L + l] = __popc(mm);
        __syncthreads();
        if (ok) {
            int before = run[l];
            for (int ww = 0; ww < w; ++ww) before += wc[ww * L + l];
            perm[base[(int64_t)blockIdx.x * L + l] + before + rin] = (int32_t)p;
        }
        __syncthreads();
        for (int ll = t; ll < L; ll += 256) {
            int s = 0;
            for (int ww = 0; ww < 8; ++ww) s += wc[ww * L + ll];
            run[ll] += s;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ density tiles

struct DensItem {
    int32_t label;
    int32_t col0, col1;   // range of perm positions (within the label)
    int32_t slot;         // row of the partial-sum matrix
};

struct DensSmem {
    float As[2][DBK][DBM];
    float Bs[2][DBK][DBN];
    double rowsum[DBM];
    float nrow[DBM];
    float ncol[DBN];
    int cidx[DBN];
};

// Grid: (row blocks of 128, items).  Thread (ty, tx) = (t / 16, t % 16) owns
// rows {4ty..4ty+3, 64+4ty..+3} and the same pattern of columns.
__global__ void __launch_bounds__(DT, 2)
density_tile_kernel(const float* __restrict__ xt, const float* __restrict__ norms, int64_t N,
                    int Dp, const int32_t* __restrict__ perm, const DensItem* __restrict__ items,
                    const float* __restrict__ sigma_dev, double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DensSmem& s = *reinterpret_cast<DensSmem*>(smem_raw);
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const int64_t row0 = (int64_t)blockIdx.x * DBM;
    const DensItem it = items[blockIdx.y];
    const float sg = *sigma_dev;
    const float inv2s2 = 1.0f / (2.0f * sg * sg);
    if (t < DBM) {
        s.nrow[t] = norms[row0 + t];
        s.rowsum[t] = 0.0;
    }
    const int nk = Dp / DBK;
    const int lr0 = t & 127, lq0 = t >> 7, lq1 = lq0 + 2;
    for (int c0 = it.col0; c0 < it.col1; c0 += DBN) {
        __syncthreads();  // previous tile done with ncol / cidx / buffers
        if (t < DBN) {
            const int c = c0 + t;
            const int q = perm[c < it.col1 ? c : it.col0];
            s.cidx[t] = (c < it.col1) ? q : -1;
            s.ncol[t] = norms[q];
        }
        __syncthreads();
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        const int qb = s.cidx[lr0] >= 0 ? s.cidx[lr0] : s.cidx[0];
        const float* pa = xt + (row0 + lr0) * Dp;
        const float* pb = xt + (int64_t)qb * Dp;
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
        for (int kb = 0; kb < nk; ++kb) {
            const int cur = kb & 1;
            if (kb + 1 < nk) {
                const int ko = (kb + 1) * DBK;
                ra0 = __ldg(reinterpret_cast<const float4*>(pa + ko + 4 * lq0));
                ra1 = __ldg(reinterpret_cast<const float4*>(pa + ko + 4 * lq1));
                rb0 = __ldg(reinterpret_cast<const float4*>(pb + ko + 4 * lq0));
                rb1 = __ldg(reinterpret_cast<const float4*>(pb + ko + 4 * lq1));
            }
#pragma unroll
            for (int kk = 0; kk < DBK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4*>(&s.As[cur][kk][4 * ty]);
                const float4 a1 = *reinterpret_cast<const float4*>(&s.As[cur][kk][64 + 4 * ty]);
                const float4 b0 = *reinterpret_cast<const float4*>(&s.Bs[cur][kk][4 * tx]);
                const float4 b1 = *reinterpret_cast<const float4*>(&s.Bs[cur][kk][64 + 4 * tx]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            if (kb + 1 < nk) {
                stash(cur ^ 1);
                __syncthreads();
            }
        }
        // epilogue: k = exp(-(n_y + n_q - 2 dot) / (2 sigma^2)) over the valid
        // columns; the 8 values of a thread and then the 16 column groups of
        // the row (lanes tx of the same ty) are summed in float32, the tiles
        // in float64 by the lane tx = 0
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + (i - 4);
            const float nr = s.nrow[r];
            float sum = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = (j < 4) ? 4 * tx + j : 64 + 4 * tx + (j - 4);
                if (s.cidx[c] >= 0) {
                    const float d2 = fmaxf(nr + s.ncol[c] - 2.f * acc[i][j], 0.f);
                    sum += expf(-d2 * inv2s2);
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, 16);
            if (tx == 0) s.rowsum[r] += (double)sum;
        }
    }
    __syncthreads();
    if (t < DBM && row0 + t < N) part[(int64_t)it.slot * N + row0 + t] = s.rowsum[t];
}

// f^_l(y): the item rows of label l summed in slot order.
__device__ __forceinline__ double density_at(const double* __restrict__ part, int64_t N, int a,
                                             int b, int64_t y) {
    double f = 0.0;
    for (int sl = a; sl < b; ++sl) f += part[(int64_t)sl * N + y];
    return f;
}

// Relative error bound of f^_l(y) in the exponent: the tile distance
// d2^ = n_y + n_p - 2 x_y . x_p (float32, Dp-term dot product, norms from
// float32 lane sums, operands rounded by at most rho <= u ||v||) is within
//   delta_y = (Dp + Dp/32 + 16) u (sqrt(n_y) + sqrt(n_max))^2
// of the distance of the centred features; the float32 exp and the float32
// partial sums add less than 1e-6.
__device__ __forceinline__ double density_eta(float ny, double sqrt_nmax, double cu,
                                              double inv2s2) {
    const double r = sqrt((double)ny) + sqrt_nmax;
    return cu * r * r * inv2s2 + 1e-6;
}

// Pass 0: T_l = max_y f^_l(y) exp(-eta_y) (a lower bound of max_y f_l).
// Pass 1: append every y with f^_l(y) exp(eta_y) >= T_l to the candidates.
__global__ void __launch_bounds__(256)
density_bound_kernel(const double* __restrict__ part, int64_t N, int Dp,
                     const float* __restrict__ norms, const DevState* __restrict__ st,
                     const float* __restrict__ sigma_dev, const int32_t* __restrict__ slot0,
                     int pass, unsigned long long* __restrict__ tbits, int2* __restrict__ cand,
                     unsigned long long* __restrict__ ncand, int64_t cand_cap) {
    const int l = blockIdx.y;
    const int a = slot0[l], b = slot0[l + 1];
    if (a == b) return;
    const double sg = (double)*sigma_dev;
    const double inv2s2 = 1.0 / (2.0 * sg * sg);
    const double sqrt_nmax = sqrt((double)__uint_as_float(st->knn_max_norm_bits));
    const double cu = (double)(Dp + Dp / 32 + 16) * 5.9604644775390625e-08;
    __shared__ unsigned long long smax;
    if (threadIdx.x == 0) smax = 0ull;
    __syncthreads();
    const double T = pass ? __longlong_as_double((long long)tbits[l]) : 0.0;
    unsigned long long mx = 0ull;
    for (int64_t y = (int64_t)blockIdx.x * 256 + threadIdx.x; y < N; y += (int64_t)gridDim.x * 256) {
        const double f = density_at(part, N, a, b, y);
        const double eta = density_eta(norms[y], sqrt_nmax, cu, inv2s2);
        if (pass == 0) {
            const unsigned long long lo = (unsigned long long)__double_as_longlong(f * exp(-eta));
            mx = mx > lo ? mx : lo;
        } else if (f * exp(eta) >= T) {
            const unsigned long long slot = atomicAdd(ncand, 1ull);
            if ((int64_t)slot < cand_cap) cand[slot] = make_int2((int)y, l);
        }
    }
    if (pass == 0) {
        atomicMax(&smax, mx);
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(&tbits[l], smax);
    }
}

// f_l(y) of candidate c (or, with all_pairs, of pair c = y L + l) from the
// features: 8 warps over the points of cluster l, warp_sq_dist distances,
// float64 kernel sums in a fixed order.
__global__ void __launch_bounds__(256)
density_exact_kernel(const float* __restrict__ X, int64_t N, int D, int L,
                     const int32_t* __restrict__ perm, const int64_t* __restrict__ off,
                     const int2* __restrict__ cand, int all_pairs, int64_t c0,
                     const float* __restrict__ sigma_dev, double* __restrict__ fexact) {
    __shared__ double red[8];
    const int64_t c = c0 + blockIdx.x;
    int64_t y;
    int l;
    if (all_pairs) {
        y = c / L;
        l = (int)(c % L);
    } else {
        y = cand[c].x;
        l = cand[c].y;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double sg = (double)*sigma_dev;
    const double inv2s2 = 1.0 / (2.0 * sg * sg);
    const float* xy = X + y * D;
    double f = 0.0;
    for (int64_t i = off[l] + warp; i < off[l + 1]; i += 8) {
        const int64_t p = perm[i];
        const double d2 = warp_sq_dist(X + p * D, xy, nullptr, D, lane);
        f += exp(-d2 * inv2s2);
    }
    if (lane == 0) red[warp] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        fexact[blockIdx.x] = s;
    }
}

// Pass 0: the largest exact density per label (non-negative doubles order as
// their bit patterns); pass 1: the smallest y attaining it.
__global__ void __launch_bounds__(256)
density_pick_kernel(const double* __restrict__ fexact, const int2* __restrict__ cand, int64_t c0,
                    int64_t count, int all_pairs, int L, int pass,
                    unsigned long long* __restrict__ fmax_bits, int32_t* __restrict__ arg) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * 256) {
        const int64_t c = c0 + i;
        const int64_t y = all_pairs ? c / L : cand[c].x;
        const int l = all_pairs ? (int)(c % L) : cand[c].y;
        const unsigned long long fb = (unsigned long long)__double_as_longlong(fexact[i]);
        if (pass == 0) atomicMax(&fmax_bits[l], fb);
        else if (fb == fmax_bits[l]) atomicMin(&arg[l], (int)y);
    }
}

// Modes from the arg-maxima; an empty cluster keeps its seed.
__global__ void density_finish_kernel(int L, const int32_t* __restrict__ slot0,
                                      const unsigned long long* __restrict__ fmax_bits,
                                      const int32_t* __restrict__ arg,
                                      const int32_t* __restrict__ seeds, int32_t* __restrict__ modes,
                                      double* __restrict__ density) {
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const bool empty = slot0[l] == slot0[l + 1];
        modes[l] = empty ? seeds[l] : arg[l];
        if (density) density[l] = empty ? 0.0 : __longlong_as_double((long long)fmax_bits[l]);
    }
}

struct InitPlan {
    int64_t Np;
    int Dp, nb;       // padded sizes, sort blocks
    int chunk;        // columns per density item (multiple of 128)
    int max_items;
    int64_t cand_cap; // candidates kept in a list; more means every (y, l) is recomputed
};

InitPlan init_plan(int64_t N, int D, int L) {
    InitPlan p{};
    p.Dp = ((D + DBK - 1) / DBK) * DBK;
    p.Np = ((N + DBM - 1) / DBM) * DBM;
    p.nb = (int)((N + kSortChunk - 1) / kSortChunk);
    const int64_t tiles = (N + DBN - 1) / DBN;
    int64_t per = (tiles + 63) / 64;          // at most ~64 items beyond one per cluster
    if (per < 16) per = 16;
    p.chunk = (int)(per * DBN);
    p.max_items = (int)((N + p.chunk - 1) / p.chunk) + L;
    p.cand_cap = std::min<int64_t>((int64_t)N * L, (int64_t)1 << 22);
    return p;
}

}  // namespace

size_t init_modes_ws_bytes(const slk_ctx* ctx, int64_t N, int D, int L) {
    (void)ctx;
    const InitPlan p = init_plan(N, D, L);
    size_t b = 0;
    b += align_up(sizeof(int32_t) * N, 256) * 2;                          // assign, perm
    b += align_up(sizeof(int32_t) * (size_t)p.nb * L, 256);               // counts
    b += align_up(sizeof(int64_t) * (size_t)p.nb * L, 256);               // base
    b += align_up(sizeof(int64_t) * (L + 1), 256);                        // off
    b += align_up(sizeof(double) * D, 256) + align_up(sizeof(float) * D, 256);   // colsum, mu
    b += align_up(sizeof(float) * (size_t)p.Np * p.Dp, 256);              // xt
    b += 2 * align_up(sizeof(float) * (size_t)p.Np, 256);                 // norms, rho
    b += align_up(sizeof(DensItem) * p.max_items, 256);
    b += align_up(sizeof(int32_t) * (L + 1), 256) * 2;                    // slot0, arg
    b += align_up(sizeof(double) * (size_t)p.max_items * N, 256);         // parts
    b += align_up(sizeof(int2) * (size_t)p.cand_cap, 256);                 // candidates
    b += align_up(sizeof(double) * (size_t)p.cand_cap, 256);               // exact densities
    b += align_up(sizeof(unsigned long long) * (L + 2), 256);             // T_l, count
    return b + 4096;
}

slk_status init_modes_launch(slk_ctx* ctx, const float* X, int64_t N, int D, const int32_t* seeds,
                             int L, const float* sigma_dev, int32_t* modes, int32_t* assign_out,
                             double* density, void* ws, DevState* st) {
    const InitPlan pl = init_plan(N, D, L);
    cudaStream_t s = ctx->stream;
    WsCarver wc(ws);
    int32_t* assign = wc.take<int32_t>(N);
    int32_t* perm = wc.take<int32_t>(N);
    int32_t* counts = wc.take<int32_t>((size_t)pl.nb * L);
    int64_t* base = wc.take<int64_t>((size_t)pl.nb * L);
    int64_t* off = wc.take<int64_t>(L + 1);
    double* colsum = wc.take<double>(D);
    float* mu = wc.take<float>(D);
    float* xt = wc.take<float>((size_t)pl.Np * pl.Dp);
    float* norms = wc.take<float>(pl.Np);
    float* rho = wc.take<float>(pl.Np);
    DensItem* items = wc.take<DensItem>(pl.max_items);
    int32_t* slot0 = wc.take<int32_t>(L + 1);
    int32_t* arg = wc.take<int32_t>(L + 1);
    double* part = wc.take<double>((size_t)pl.max_items * N);
    int2* cand = wc.take<int2>((size_t)pl.cand_cap);
    double* fexact = wc.take<double>((size_t)pl.cand_cap);
    unsigned long long* tbits = wc.take<unsigned long long>(L + 2);
    unsigned long long* ncand = tbits + L;

    // 1. nearest seed
    {
        SLK_COUNT_LAUNCH(ctx, 1);
        const size_t smem = sizeof(float) * (32 * 33 + (size_t)L * 33 + 1) + sizeof(double) * 32 * L + 16;
        const int lpt = (L + 7) / 8;
        const unsigned grid = (unsigned)((N + 31) / 32);
#define SLK_ASSIGN(LPT_)                                                                        \
    {                                                                                           \
        auto kern = seed_assign_kernel<LPT_>;                                                   \
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                               (int)smem));                                     \
        kern<<<grid, 256, smem, s>>>(X, N, D, seeds, L, assign);                                \
    }
        if (lpt <= 1) { SLK_ASSIGN(1) }
        else if (lpt <= 2) { SLK_ASSIGN(2) }
        else if (lpt <= 4) { SLK_ASSIGN(4) }
        else if (lpt <= 8) { SLK_ASSIGN(8) }
        else if (lpt <= 16) { SLK_ASSIGN(16) }
        else { SLK_ASSIGN(32) }
#undef SLK_ASSIGN
        SLK_LAUNCH_CHECK(ctx, "seed_assign_kernel");
    }
    // 2. stable counting sort by cluster
    SLK_COUNT_LAUNCH(ctx, 3);
    label_count_kernel<<<pl.nb, 256, sizeof(int) * L, s>>>(assign, N, L, counts);
    label_scan_kernel<<<1, 256, 0, s>>>(counts, pl.nb, L, base, off);
    label_scatter_kernel<<<pl.nb, 256, sizeof(int) * 9 * L, s>>>(assign, N, L, base, perm);
    SLK_LAUNCH_CHECK(ctx, "counting sort");
    // 3. centred operand and norms
    slk_status r = knn_prep_fp32_launch(ctx, X, N, D, pl.Dp, pl.Np, colsum, mu, xt, norms, rho, st);
    if (r != SLK_OK) return r;
    // 4. work items: every cluster's perm range cut into chunks (host, from the offsets)
    std::vector<int64_t> hoff(L + 1);
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(hoff.data(), off, sizeof(int64_t) * (L + 1),
                                      cudaMemcpyDeviceToHost, s));
    SLK_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    std::vector<DensItem> hit;
    std::vector<int32_t> hslot(L + 1, 0);
    for (int l = 0; l < L; ++l) {
        hslot[l] = (int32_t)hit.size();
        for (int64_t c = hoff[l]; c < hoff[l + 1]; c += pl.chunk) {
            DensItem it;
            it.label = l;
            it.col0 = (int32_t)c;
            it.col1 = (int32_t)std::min<int64_t>(c + pl.chunk, hoff[l + 1]);
            it.slot = (int32_t)hit.size();
            hit.push_back(it);
        }
    }
    hslot[L] = (int32_t)hit.size();
    if ((int)hit.size() > pl.max_items) return set_err(ctx, SLK_ERR_CUDA, "density items overflow");
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(items, hit.data(), sizeof(DensItem) * hit.size(),
                                      cudaMemcpyHostToDevice, s));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(slot0, hslot.data(), sizeof(int32_t) * (L + 1),
                                      cudaMemcpyHostToDevice, s));
    // 5. density tiles
    if (!hit.empty()) {
        SLK_COUNT_LAUNCH(ctx, 1);
        const int smem = (int)sizeof(DensSmem);
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(density_tile_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        density_tile_kernel<<<dim3((unsigned)(pl.Np / DBM), (unsigned)hit.size()), DT, smem, s>>>(
            xt, norms, N, pl.Dp, perm, items, sigma_dev, part);
        SLK_LAUNCH_CHECK(ctx, "density_tile_kernel");
    }
    // 6. candidates: upper bound of f_l(y) reaches the largest lower bound
    SLK_COUNT_LAUNCH(ctx, 2);
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(tbits, 0, sizeof(unsigned long long) * (L + 1), s));
    int gx = (int)((N + 255) / 256);
    if (gx > 4 * ctx->num_sms) gx = 4 * ctx->num_sms;
    for (int pass = 0; pass < 2; ++pass)
        density_bound_kernel<<<dim3((unsigned)gx, (unsigned)L), 256, 0, s>>>(
            part, N, pl.Dp, norms, st, sigma_dev, slot0, pass, tbits, cand, ncand, pl.cand_cap);
    SLK_LAUNCH_CHECK(ctx, "density_bound_kernel");
    unsigned long long hcount = 0;
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(&hcount, ncand, sizeof(hcount), cudaMemcpyDeviceToHost, s));
    SLK_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    // 7. exact densities of the candidates; when the list overflowed, of every
    // (y, l) pair, in rounds of the list's capacity (recomputed for pass 1)
    const int all_pairs = ((int64_t)hcount > pl.cand_cap) ? 1 : 0;
    const int64_t count = all_pairs ? (int64_t)N * L : (int64_t)hcount;
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->mode_best[0], 0, sizeof(unsigned long long) * L, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(arg, 0x7f, sizeof(int32_t) * L, s));
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t c0 = 0; c0 < count; c0 += pl.cand_cap) {
            const int64_t n = std::min<int64_t>(pl.cand_cap, count - c0);
            if (pass == 0 || all_pairs) {
                SLK_COUNT_LAUNCH(ctx, 1);
                density_exact_kernel<<<(unsigned)n, 256, 0, s>>>(X, N, D, L, perm, off, cand,
                                                                 all_pairs, c0, sigma_dev, fexact);
            }
            int pg = (int)((n + 255) / 256);
            if (pg > 4 * ctx->num_sms) pg = 4 * ctx->num_sms;
            SLK_COUNT_LAUNCH(ctx, 1);
            density_pick_kernel<<<(unsigned)pg, 256, 0, s>>>(fexact, cand, c0, n, all_pairs, L, pass,
                                                             &st->mode_best[0], arg);
        }
    }
    SLK_COUNT_LAUNCH(ctx, 1);
    density_finish_kernel<<<1, 256, 0, s>>>(L, slot0, &st->mode_best[0], arg, seeds, modes, density);
    SLK_LAUNCH_CHECK(ctx, "density_exact_kernel");
    ctx->init_candidates = count;
    if (assign_out)
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(assign_out, assign, sizeof(int32_t) * N,
                                          cudaMemcpyDeviceToDevice, s));
    return SLK_OK;
}

// ---------------------------------------------------------------- row order for locality

namespace {

__global__ void row_argmax_kernel(const float* __restrict__ A, int64_t N, int L,
                                  int32_t* __restrict__ lab) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        const float* a = A + p * L;
        int best = 0;
        float bv = a[0];
        for (int l = 1; l < L; ++l)
            if (a[l] > bv) { bv = a[l]; best = l; }
        lab[p] = best;
    }
}

__global__ void inverse_perm_kernel(const int32_t* __restrict__ perm, int64_t N,
                                    int32_t* __restrict__ inv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        inv[perm[i]] = (int32_t)i;
}

// dst row i = src row perm[i] (rows of W floats), one warp per row.
__global__ void gather_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ perm,
                                   int64_t N, int W, float* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < N; i += nw) {
        const float* s = src + (int64_t)perm[i] * W;
        float* d = dst + i * W;
        for (int j = lane; j < W; j += 32) d[j] = s[j];
    }
}

// dst row perm[i] = src row i.
__global__ void scatter_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ perm,
                                    int64_t N, int W, float* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < N; i += nw) {
        const float* s = src + i * W;
        float* d = dst + (int64_t)perm[i] * W;
        for (int j = lane; j < W; j += 32) d[j] = s[j];
    }
}

// Uniform-degree CSR in the new row order: row i = old row perm[i], every
// neighbour renamed by inv, edge order kept (so each row sums alike).
__global__ void permute_graph_kernel(const int32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                                     int64_t N, int k, const int32_t* __restrict__ col,
                                     const float* __restrict__ w, int32_t* __restrict__ colp,
                                     float* __restrict__ wp) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, j = e % k;
        const int64_t o = (int64_t)perm[i] * k + j;
        colp[e] = inv[col[o]];
        if (w) wp[e] = w[o];
    }
}

__global__ void map_modes_kernel(const int32_t* __restrict__ inv, const int32_t* __restrict__ modes,
                                 int L, int32_t* __restrict__ out) {
    for (int l = threadIdx.x; l < L; l += blockDim.x) out[l] = inv[modes[l]];
}

__global__ void unpermute_small_kernel(const int32_t* __restrict__ perm, int64_t N, int L,
                                       const int32_t* __restrict__ labels_p,
                                       const int32_t* __restrict__ modes_p,
                                       int32_t* __restrict__ labels, int32_t* __restrict__ modes) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        labels[perm[i]] = labels_p[i];
        if (i < L) modes[i] = perm[modes_p[i]];
    }
}

unsigned grid_for(const slk_ctx* ctx, int64_t work, int per_block) {
    int64_t g = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)ctx->num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

size_t locality_ws_bytes(int64_t N, int L) {
    const int nb = (int)((N + kSortChunk - 1) / kSortChunk);
    return align_up(sizeof(int32_t) * N, 256) + align_up(sizeof(int32_t) * (size_t)nb * L, 256) +
           align_up(sizeof(int64_t) * (size_t)nb * L, 256) + align_up(sizeof(int64_t) * (L + 1), 256) +
           1024;
}

slk_status locality_perm_launch(slk_ctx* ctx, const float* A, int64_t N, int L, int32_t* perm,
                                int32_t* inv, void* ws) {
    cudaStream_t s = ctx->stream;
    const int nb = (int)((N + kSortChunk - 1) / kSortChunk);
    WsCarver wc(ws);
    int32_t* lab = wc.take<int32_t>(N);
    int32_t* counts = wc.take<int32_t>((size_t)nb * L);
    int64_t* base = wc.take<int64_t>((size_t)nb * L);
    int64_t* off = wc.take<int64_t>(L + 1);
    SLK_COUNT_LAUNCH(ctx, 5);
    row_argmax_kernel<<<grid_for(ctx, N, 256), 256, 0, s>>>(A, N, L, lab);
    label_count_kernel<<<nb, 256, sizeof(int) * L, s>>>(lab, N, L, counts);
    label_scan_kernel<<<1, 256, 0, s>>>(counts, nb, L, base, off);
    label_scatter_kernel<<<nb, 256, sizeof(int) * 9 * L, s>>>(lab, N, L, base, perm);
    inverse_perm_kernel<<<grid_for(ctx, N, 256), 256, 0, s>>>(perm, N, inv);
    SLK_LAUNCH_CHECK(ctx, "locality order");
    return SLK_OK;
}

slk_status permute_problem_launch(slk_ctx* ctx, const int32_t* perm, const int32_t* inv,
                                  int64_t N, int D, int L, int k, const float* X, const float* A,
                                  const float* Z0, const int32_t* col_idx, const float* w,
                                  float* Xp, float* Ap, float* Z0p, int32_t* colp, float* wp) {
    cudaStream_t s = ctx->stream;
    const unsigned rg = grid_for(ctx, N, 8);
    SLK_COUNT_LAUNCH(ctx, 4);
    gather_rows_kernel<<<rg, 256, 0, s>>>(X, perm, N, D, Xp);
    gather_rows_kernel<<<rg, 256, 0, s>>>(A, perm, N, L, Ap);
    gather_rows_kernel<<<rg, 256, 0, s>>>(Z0, perm, N, L, Z0p);
    permute_graph_kernel<<<grid_for(ctx, N * k, 256), 256, 0, s>>>(perm, inv, N, k, col_idx, w, colp, wp);
    SLK_LAUNCH_CHECK(ctx, "permute problem");
    return SLK_OK;
}

slk_status unpermute_launch(slk_ctx* ctx, const int32_t* perm, int64_t N, int L, const float* Zp,
                            const int32_t* labels_p, const int32_t* modes_p, float* Z,
                            int32_t* labels, int32_t* modes) {
    cudaStream_t s = ctx->stream;
    SLK_COUNT_LAUNCH(ctx, 2);
    scatter_rows_kernel<<<grid_for(ctx, N, 8), 256, 0, s>>>(Zp, perm, N, L, Z);
    unpermute_small_kernel<<<grid_for(ctx, N, 256), 256, 0, s>>>(perm, N, L, labels_p, modes_p,
                                                                 labels, modes);
    SLK_LAUNCH_CHECK(ctx, "unpermute");
    return SLK_OK;
}

slk_status map_modes_launch(slk_ctx* ctx, const int32_t* inv, const int32_t* modes, int L,
                            int32_t* out) {
    SLK_COUNT_LAUNCH(ctx, 1);
    map_modes_kernel<<<1, 256, 0, ctx->stream>>>(inv, modes, L, out);
    SLK_LAUNCH_CHECK(ctx, "map_modes_kernel");
    return SLK_OK;
}
