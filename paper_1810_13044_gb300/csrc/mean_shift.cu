// SLK-MS mode update: Eq. (mean-shift) iterated with the assignments fixed
// (Algorithm 1, SLK-MS branch):
//   m_l <- sum_p z_{p,l} k(x_p, m_l) x_p / sum_p z_{p,l} k(x_p, m_l),
// k the Gaussian kernel of Section 4.2.  The weight of point p for mode l is
// computed in the log domain, s_{p,l} = log z_{p,l} - ||x_p - m_l||^2 / (2
// sigma^2), and every sum is kept relative to a running maximum of s (the
// factor cancels in the ratio), so neither saturated z nor modes far from
// every point lose the weights to float32 underflow.
//
// One pass over X per iteration, one persistent cooperative kernel for all
// iterations:
//   phase 1  every CTA takes one (row range, label group) unit.  Row tiles
//            of R rows arrive by bulk copy (cp.async.bulk, mbarrier) into a
//            double buffer; for each tile
//              A  exact float32 distances ||x_p - m_l||^2 (direct differences;
//                 warp = 4 rows x the group's labels x part of the features,
//                 lane sums folded by a 32-lane reduce-scatter),
//              B  s, the tile maximum per label, rescale factor of the
//                 running sums, weights w = exp(s - max),
//              C  acc[l][d] = acc[l][d] * rescale + sum_p w_{p,l} x_{p,d}
//                 (thread = all labels of the group x CPT features, registers),
//            then writes (max, sum of weights, acc) of the unit;
//   barrier
//   phase 2  warps combine the units of every label in float64, write the new
//            modes (float64 state and float32 copies) and add the squared
//            move of each label;
//   barrier  the last block decides: stop when max_l ||m_l^new - m_l^old||_2
//            <= tol * sigma, or at max_iters.
// Waits (bulk copies, barriers) are bounded; on a timeout the kernel raises
// an error word, lets its own copies drain (bounded) and returns.
#include <math.h>
#include <stdint.h>

#include "slk_internal.cuh"
#include "sync.cuh"

namespace {

constexpr int kMsThreads = 256;
constexpr int kMsWarps = kMsThreads / 32;
#define kNegInf __int_as_float(0xff800000)

struct MsArgs {
    const float* X;
    int64_t N;
    int D, Dp;          // Dp: shared-memory row stride (D rounded up to 4)
    int bulk;           // 1: tiles arrive by bulk copy (D % 4 == 0, X 16-byte aligned)
    const float* LZ;    // N x L log z
    int L;
    const float* sigma_dev;
    double* M64;        // L x D state
    float* Mout;        // L x D caller's modes (read in iteration 0, written every iteration)
    float* Mbuf[2];     // L x D ping-pong copies read by phase 1 after iteration 0
    float* part;        // [units][LG][D] weighted sums
    float* part_mu;     // [units][LG] running maxima
    float* part_s;      // [units][LG] sums of weights
    int groups, P, units;
    int64_t tiles;      // ceil(N / R)
    int max_iters;
    float tol;
    MsStatus* ms;
};

template <int R, int LG>
struct MsSmem {
    float red[kMsWarps / (R / 4)][LG][R];  // per feature part: distances of the tile (label-major)
    float w[R][LG];
    float alpha[LG];
    float mu[LG];        // running maximum of s per label
    float ssum[LG];      // running sum of weights per label (relative to mu)
    unsigned long long bar[2];
    int abort;
};

// Reduce-scatter of 64 values over the 32 lanes: afterwards lane holds the
// full sums of original indices base, base + 1, base = 2 * bitreverse5(lane).
__device__ __forceinline__ void reduce_scatter64(float (&v)[64], int lane) {
#pragma unroll
    for (int o = 16, n = 64; o >= 1; o >>= 1, n >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const float keep = up ? v[i + n / 2] : v[i];
            const float send = up ? v[i] : v[i + n / 2];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

// Shared-memory row stride and tile bytes.
__host__ __device__ __forceinline__ int round4(int d) { return (d + 3) & ~3; }

template <int R, int LG, int CPT>
__device__ void ms_load_tile_plain(const MsArgs& a, float* xs, int64_t row0, int nrows) {
    for (int i = threadIdx.x; i < R * a.Dp; i += kMsThreads) {
        const int r = i / a.Dp, c = i % a.Dp;
        xs[i] = (r < nrows && c < a.D) ? a.X[(row0 + r) * a.D + c] : 0.f;
    }
}

// Phase 1 of one unit: the weighted sums of label group g over row range pr.
template <int R, int LG, int CPT>
__device__ bool ms_unit(const MsArgs& a, int u, const float* Mc, float* xs0, float* xs1,
                        float* msm, MsSmem<R, LG>& sh, uint32_t (&par)[2]) {
    constexpr int QUADS = R / 4;
    constexpr int HP = kMsWarps / QUADS;  // feature parts per row quad
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int pr = u / a.groups, g = u % a.groups;
    const int l0 = g * LG;
    const int lg = min(LG, a.L - l0);
    const int64_t t_begin = a.tiles * pr / a.P, t_end = a.tiles * (pr + 1) / a.P;
    const int D = a.D, Dp = a.Dp;
    const float sg = *a.sigma_dev;
    const float inv2s2 = 1.0f / (2.0f * sg * sg);

    // modes of the group (zero rows beyond lg)
    for (int i = t; i < LG * Dp; i += kMsThreads) {
        const int l = i / Dp, c = i % Dp;
        msm[i] = (l < lg && c < D) ? __ldcg(Mc + (int64_t)(l0 + l) * D + c) : 0.f;
    }
    if (t < LG) {
        sh.mu[t] = kNegInf;
        sh.ssum[t] = 0.f;
    }
    float acc[LG][CPT];
#pragma unroll
    for (int l = 0; l < LG; ++l)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[l][c] = 0.f;
    __syncthreads();

    auto issue = [&](int64_t ti, int b) {
        const int64_t row0 = ti * R;
        const int nrows = (int)min((int64_t)R, a.N - row0);
        float* dst = b ? xs1 : xs0;
        if (a.bulk) {
            if (t == 0) {
                const uint32_t bytes = (uint32_t)nrows * (uint32_t)D * 4u;
                fence_proxy_async_smem();
                mbar_arrive_tx(&sh.bar[b], bytes);
                bulk_g2s(dst, a.X + row0 * D, bytes, &sh.bar[b]);
            }
        } else {
            ms_load_tile_plain<R, LG, CPT>(a, dst, row0, nrows);
        }
    };

    if (t_begin < t_end) issue(t_begin, 0);
    for (int64_t ti = t_begin; ti < t_end; ++ti) {
        const int b = (int)((ti - t_begin) & 1);
        const int64_t row0 = ti * R;
        const int nrows = (int)min((int64_t)R, a.N - row0);
        const float* xs = b ? xs1 : xs0;
        if (ti + 1 < t_end) issue(ti + 1, b ^ 1);
        if (a.bulk) {
            const bool ok = mbar_wait_parity(&sh.bar[b], par[b]);
            if (__syncthreads_or(!ok)) {
                if (t == 0) sh.abort = 1;
                return false;  // par[b] still names the phase of the copy in flight
            }
            par[b] ^= 1u;
        } else {
            __syncthreads();
        }

        // ---- A: distances of 4 rows x LG labels over a part of the features
        {
            const int q = warp % QUADS, h = warp / QUADS;
            float v[64];
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = 0.f;
            const float* x0 = xs + (4 * q) * Dp;
            for (int c0 = h * 32; c0 < D; c0 += HP * 32) {
                const int d = c0 + lane;
                if (d < D) {
                    const float x[4] = {x0[d], x0[Dp + d], x0[2 * Dp + d], x0[3 * Dp + d]};
#pragma unroll
                    for (int l = 0; l < LG; ++l) {
                        const float m = msm[l * Dp + d];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float df = x[i] - m;
                            v[i * 16 + l] = fmaf(df, df, v[i * 16 + l]);
                        }
                    }
                }
            }
            reduce_scatter64(v, lane);
            const int base = (((lane >> 4) & 1) << 5) | (((lane >> 3) & 1) << 4) |
                             (((lane >> 2) & 1) << 3) | (((lane >> 1) & 1) << 2) | ((lane & 1) << 1);
            const int i = base >> 4, l = base & 15;
            if (l < LG) sh.red[h][l][4 * q + i] = v[0];
            if (l + 1 < LG) sh.red[h][l + 1][4 * q + i] = v[1];
        }
        __syncthreads();
        // ---- B: a warp per label (labels warp, warp + 8, ...), lanes over the
        // rows: s, tile maximum, rescale factor of the running sums, weights
        // relative to the new maximum
        for (int l = warp; l < LG; l += kMsWarps) {
            float sv = kNegInf;
            if (lane < R && lane < nrows && l < lg) {
                float d2 = 0.f;
#pragma unroll
                for (int hh = 0; hh < HP; ++hh) d2 += sh.red[hh][l][lane];
                sv = __ldg(a.LZ + (row0 + lane) * a.L + l0 + l) - d2 * inv2s2;
            }
            float tm = sv;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tm = fmaxf(tm, __shfl_xor_sync(0xffffffffu, tm, o));
            const float mo = sh.mu[l];
            const float mn = fmaxf(mo, tm);
            const float wt = (sv == kNegInf) ? 0.f : expf(sv - mn);
            if (lane < R) sh.w[lane][l] = wt;
            float sw = wt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(0xffffffffu, sw, o);
            if (lane == 0) {
                const float al = (mn == kNegInf) ? 1.f : expf(mo - mn);
                sh.alpha[l] = al;
                sh.mu[l] = mn;
                sh.ssum[l] = sh.ssum[l] * al + sw;
            }
        }
        __syncthreads();
        // ---- C: rescale and accumulate the weighted rows
        {
            float al[LG];
#pragma unroll
            for (int l = 0; l < LG; ++l) al[l] = sh.alpha[l];
#pragma unroll
            for (int l = 0; l < LG; ++l)
#pragma unroll
                for (int c = 0; c < CPT; ++c) acc[l][c] *= al[l];
            for (int r = 0; r < nrows; ++r) {
                float wv[LG];
#pragma unroll
                for (int l = 0; l < LG; l += 4) {
                    const float4 w4 = *reinterpret_cast<const float4*>(&sh.w[r][l]);
                    wv[l] = w4.x; wv[l + 1] = w4.y; wv[l + 2] = w4.z; wv[l + 3] = w4.w;
                }
                const float* xr = xs + r * Dp;
                float xv[CPT];
                if constexpr (CPT >= 4) {
#pragma unroll
                    for (int j = 0; j < CPT / 4; ++j) {
                        const int q4 = t + kMsThreads * j;
                        float4 x4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (4 * q4 < Dp) x4 = *reinterpret_cast<const float4*>(xr + 4 * q4);
                        xv[4 * j] = x4.x; xv[4 * j + 1] = x4.y; xv[4 * j + 2] = x4.z; xv[4 * j + 3] = x4.w;
                    }
                } else if constexpr (CPT == 2) {
                    float2 x2 = make_float2(0.f, 0.f);
                    if (2 * t < Dp) x2 = *reinterpret_cast<const float2*>(xr + 2 * t);
                    xv[0] = x2.x;
                    xv[1] = x2.y;
                } else {
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        const int col = t * CPT + c;
                        xv[c] = (col < Dp) ? xr[col] : 0.f;
                    }
                }
#pragma unroll
                for (int l = 0; l < LG; ++l)
#pragma unroll
                    for (int c = 0; c < CPT; ++c) acc[l][c] = fmaf(wv[l], xv[c], acc[l][c]);
            }
        }
        __syncthreads();  // the buffer and the tile's weights are free again
    }

    // unit results
    float* pu = a.part + (int64_t)u * LG * D;
#pragma unroll
    for (int l = 0; l < LG; ++l) {
        if (l >= lg) break;
        if constexpr (CPT >= 4) {
#pragma unroll
            for (int j = 0; j < CPT / 4; ++j) {
                const int q4 = t + kMsThreads * j;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int col = 4 * q4 + c;
                    if (col < D) pu[l * D + col] = acc[l][4 * j + c];
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int col = t * CPT + c;
                if (col < D) pu[l * D + col] = acc[l][c];
            }
        }
    }
    if (t < lg) {
        a.part_mu[u * LG + t] = sh.mu[t];
        a.part_s[u * LG + t] = sh.ssum[t];
    }
    __syncthreads();
    return true;
}

// Phase 2: warps over (label, 32 features): combine the units of the
// label's group in float64, new mode, squared move added per label.
template <int LG>
__device__ void ms_finish(const MsArgs& a, int it, float* Mnext) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kMsWarps + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * kMsWarps;
    const int D = a.D;
    const int nblk = (D + 31) / 32;
    double* sh2 = a.ms->shift2[it % 3];
    for (int64_t task = gw; task < (int64_t)a.L * nblk; task += nw) {
        const int l = (int)(task / nblk);
        const int d = (int)(task % nblk) * 32 + lane;
        const int g = l / LG, li = l % LG;
        float mu = kNegInf;
        for (int p = 0; p < a.P; ++p) mu = fmaxf(mu, __ldcg(a.part_mu + (p * a.groups + g) * LG + li));
        double num = 0.0, den = 0.0;
        for (int p = 0; p < a.P; ++p) {
            const int uu = p * a.groups + g;
            const float mp = __ldcg(a.part_mu + uu * LG + li);
            const double c = (mp == kNegInf) ? 0.0 : (double)expf(mp - mu);
            den += c * (double)__ldcg(a.part_s + uu * LG + li);
            if (d < D) num += c * (double)__ldcg(a.part + ((int64_t)uu * LG + li) * D + d);
        }
        double mv = 0.0;
        if (d < D) {
            const int64_t o = (int64_t)l * D + d;
            const double mnew = num / den;
            const double mold = a.M64[o];
            a.M64[o] = mnew;
            const float mf = (float)mnew;
            Mnext[o] = mf;
            a.Mout[o] = mf;
            mv = (mnew - mold) * (mnew - mold);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mv += __shfl_xor_sync(0xffffffffu, mv, o);
        if (lane == 0) atomicAdd(&sh2[l], mv);
    }
}

// Decision of iteration `it` (one thread): records the count and the move.
__device__ __forceinline__ bool ms_decide(const MsArgs& a, int it) {
    double mx = 0.0;
    for (int l = 0; l < a.L; ++l) mx = fmax(mx, __ldcg(&a.ms->shift2[it % 3][l]));
    const float shift = (float)sqrt(mx);
    a.ms->last_shift = shift;
    a.ms->iters_done = it + 1;
    return a.tol >= 0.f && shift <= a.tol * *a.sigma_dev;
}

template <int R, int LG, int CPT>
struct MsLayout {
    static size_t bytes(int Dp) {
        return 1024 + sizeof(MsSmem<R, LG>) + sizeof(float) * ((size_t)2 * R * Dp + (size_t)LG * Dp);
    }
};

template <int R, int LG, int CPT>
__device__ __forceinline__ void ms_carve(unsigned char* raw, int Dp, MsSmem<R, LG>*& sh,
                                         float*& xs0, float*& xs1, float*& msm) {
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
    xs0 = reinterpret_cast<float*>(base);
    xs1 = xs0 + (size_t)R * Dp;
    msm = xs1 + (size_t)R * Dp;
    sh = reinterpret_cast<MsSmem<R, LG>*>(msm + (size_t)LG * Dp);
}

template <int R, int LG, int CPT>
__global__ void __launch_bounds__(kMsThreads, 1) ms_persistent_kernel(MsArgs a) {
    extern __shared__ unsigned char ms_raw[];
    MsSmem<R, LG>* sh;
    float *xs0, *xs1, *msm;
    ms_carve<R, LG, CPT>(ms_raw, a.Dp, sh, xs0, xs1, msm);
    GridBarrier* gb = reinterpret_cast<GridBarrier*>(a.ms);
    if (threadIdx.x == 0) {
        mbar_init1(&sh->bar[0]);
        mbar_init1(&sh->bar[1]);
        sh->abort = 0;
    }
    __syncthreads();
    uint32_t par[2] = {0u, 0u};
    bool ok = true;
    for (int it = 0; it < a.max_iters; ++it) {
        const float* Mc = (it == 0) ? a.Mout : a.Mbuf[(it - 1) & 1];
        if (blockIdx.x == 0)
            for (int l = threadIdx.x; l < a.L; l += kMsThreads) a.ms->shift2[(it + 1) % 3][l] = 0.0;
        for (int u = blockIdx.x; u < a.units && ok; u += gridDim.x)
            ok = ms_unit<R, LG, CPT>(a, u, Mc, xs0, xs1, msm, *sh, par);
        if (!ok) {
            if (threadIdx.x == 0) atomicOr(&gb->error, 2u);
            break;
        }
        if (grid_barrier(gb, gridDim.x, [] { return false; }) < 0) break;
        ms_finish<LG>(a, it, a.Mbuf[it & 1]);
        const int r = grid_barrier(gb, gridDim.x, [&] { return ms_decide(a, it); });
        if (r != 0) break;
    }
    if (!ok && a.bulk && threadIdx.x == 0) {
        // let copies still in flight land before the shared memory is released
        for (int b = 0; b < 2; ++b) mbar_wait_parity(&sh->bar[b], par[b]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_inval(&sh->bar[0]);
        mbar_inval(&sh->bar[1]);
    }
}

// Without cooperative launch: one launch per phase and iteration; a launch
// after the decision has stopped the loop returns at once.
template <int R, int LG, int CPT>
__global__ void __launch_bounds__(kMsThreads, 1) ms_accum_kernel(MsArgs a, int it) {
    if (*(volatile unsigned*)&a.ms->stop != 0u) return;
    extern __shared__ unsigned char ms_raw[];
    MsSmem<R, LG>* sh;
    float *xs0, *xs1, *msm;
    ms_carve<R, LG, CPT>(ms_raw, a.Dp, sh, xs0, xs1, msm);
    if (threadIdx.x == 0) {
        mbar_init1(&sh->bar[0]);
        mbar_init1(&sh->bar[1]);
        sh->abort = 0;
    }
    __syncthreads();
    const float* Mc = (it == 0) ? a.Mout : a.Mbuf[(it - 1) & 1];
    if (blockIdx.x == 0)
        for (int l = threadIdx.x; l < a.L; l += kMsThreads) a.ms->shift2[(it + 1) % 3][l] = 0.0;
    uint32_t par[2] = {0u, 0u};
    bool ok = true;
    for (int u = blockIdx.x; u < a.units && ok; u += gridDim.x)
        ok = ms_unit<R, LG, CPT>(a, u, Mc, xs0, xs1, msm, *sh, par);
    if (!ok && threadIdx.x == 0) {
        atomicOr(&a.ms->error, 2u);
        for (int b = 0; b < 2; ++b) mbar_wait_parity(&sh->bar[b], par[b]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_inval(&sh->bar[0]);
        mbar_inval(&sh->bar[1]);
    }
}

template <int LG>
__global__ void __launch_bounds__(kMsThreads) ms_finish_kernel(MsArgs a, int it) {
    if (*(volatile unsigned*)&a.ms->stop != 0u || *(volatile unsigned*)&a.ms->error != 0u) return;
    ms_finish<LG>(a, it, a.Mbuf[it & 1]);
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atom_add_ar(&a.ms->arrive, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        a.ms->arrive = 0;
        if (ms_decide(a, it)) a.ms->stop = 1u;
    }
}

__global__ void ms_gather_kernel(const float* __restrict__ X, int D, const int32_t* __restrict__ idx,
                                 int L, float* __restrict__ M, double* __restrict__ M64) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < (int64_t)L * D;
         o += (int64_t)gridDim.x * blockDim.x) {
        const float v = X[(int64_t)idx[o / D] * D + o % D];
        M[o] = v;
        M64[o] = (double)v;
    }
}

__global__ void ms_split_kernel(const double* __restrict__ M64, int64_t n, float* __restrict__ Mhi,
                                float* __restrict__ Mlo) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        const double m = M64[o];
        const float hi = (float)m;
        Mhi[o] = hi;
        Mlo[o] = (float)(m - (double)hi);
    }
}

__global__ void ms_widen_kernel(const float* __restrict__ M, int64_t n, double* __restrict__ M64) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x)
        M64[o] = (double)M[o];
}

// One block: warp w takes labels w, w + 8, ...; max over labels of the norm.
__global__ void __launch_bounds__(256)
ms_moved_kernel(const double* __restrict__ M64, const double* __restrict__ M0, int D, int L,
                MsStatus* ms) {
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double mx = 0.0;
    for (int l = warp; l < L; l += 8) {
        double s = 0.0;
        for (int d = lane; d < D; d += 32) {
            const double df = M64[(int64_t)l * D + d] - M0[(int64_t)l * D + d];
            s += df * df;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = fmax(mx, s);
    }
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < 8; ++i) m = fmax(m, red[i]);
        ms->moved = (float)sqrt(m);
    }
}

// Launch shape for a feature count: rows per tile, labels per group,
// features per thread in phase C.
struct MsShape {
    int R, LG, CPT;
};
MsShape ms_shape(int D, int L) {
    if (D <= 1024) {
        const int cpt = D <= 256 ? 1 : D <= 512 ? 2 : 4;
        const int lg = L <= 4 ? 4 : L <= 8 ? 8 : L <= 12 ? 12 : 16;
        return {16, lg, cpt};
    }
    if (D <= 2048) return {8, L <= 4 ? 4 : 8, 8};
    return {4, 4, 16};
}

template <int R, int LG, int CPT>
slk_status ms_run(slk_ctx* ctx, MsArgs& a) {
    const size_t smem = MsLayout<R, LG, CPT>::bytes(a.Dp);
    auto kp = ms_persistent_kernel<R, LG, CPT>;
    auto ka = ms_accum_kernel<R, LG, CPT>;
    SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SLK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp, kMsThreads, smem));
    if (per_sm < 1) return set_err(ctx, SLK_ERR_CUDA, "mean-shift kernel does not fit on an SM");
    // the workspace holds the partial sums of at most 2 CTAs per SM
    const int64_t max_grid = (int64_t)ctx->num_sms * (per_sm < 2 ? per_sm : 2);
    int64_t P = max_grid / a.groups;
    if (P < 1) P = 1;
    if (P > a.tiles) P = a.tiles;
    a.P = (int)P;
    a.units = a.groups * a.P;
    const int64_t grid = a.units < max_grid ? a.units : max_grid;
    if (ctx->coop_supported) {
        SLK_COUNT_LAUNCH(ctx, 1);
        void* args[] = {&a};
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)kp, dim3((unsigned)grid),
                                                    dim3(kMsThreads), args, smem, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "ms_persistent_kernel");
    } else {
        SLK_COUNT_LAUNCH(ctx, 2 * a.max_iters);
        for (int it = 0; it < a.max_iters; ++it) {
            ka<<<(unsigned)grid, kMsThreads, smem, ctx->stream>>>(a, it);
            ms_finish_kernel<LG><<<(unsigned)grid, kMsThreads, 0, ctx->stream>>>(a, it);
        }
        SLK_LAUNCH_CHECK(ctx, "ms_accum_kernel / ms_finish_kernel");
    }
    return SLK_OK;
}

}  // namespace

size_t ms_ws_bytes(const slk_ctx* ctx, int64_t N, int D, int L) {
    const MsShape s = ms_shape(D, L);
    const int groups = (L + s.LG - 1) / s.LG;
    const int64_t units = (int64_t)ctx->num_sms * 2 * groups;  // at most 2 CTAs per SM
    return 256 * 6 + sizeof(float) * (size_t)L * D * 2 +
           sizeof(float) * (size_t)units * s.LG * ((size_t)D + 2);
}

slk_status ms_launch(slk_ctx* ctx, const float* X, int64_t N, int D, const float* LZ, int L,
                     const float* sigma_dev, double* M64, float* M, int max_iters, float tol,
                     MsStatus* ms, void* ws) {
    if (D > 4096) return set_err(ctx, SLK_ERR_INVALID_ARG, "mean-shift modes: D = %d > 4096", D);
    const MsShape s = ms_shape(D, L);
    MsArgs a{};
    a.X = X;
    a.N = N;
    a.D = D;
    a.Dp = round4(D);
    a.bulk = (D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0) ? 1 : 0;
    a.LZ = LZ;
    a.L = L;
    a.sigma_dev = sigma_dev;
    a.M64 = M64;
    a.Mout = M;
    a.groups = (L + s.LG - 1) / s.LG;
    a.tiles = (N + s.R - 1) / s.R;
    a.max_iters = max_iters;
    a.tol = tol;
    a.ms = ms;
    WsCarver wc(ws);
    a.Mbuf[0] = wc.take<float>((size_t)L * D);
    a.Mbuf[1] = wc.take<float>((size_t)L * D);
    const int64_t units_max = (int64_t)ctx->num_sms * 2 * a.groups;
    a.part_mu = wc.take<float>((size_t)units_max * s.LG);
    a.part_s = wc.take<float>((size_t)units_max * s.LG);
    a.part = wc.take<float>((size_t)units_max * s.LG * D);
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(ms, 0, sizeof(MsStatus), ctx->stream));
    if (max_iters <= 0) return SLK_OK;
    PhaseScope ps(ctx, SLK_PHASE_MEANSHIFT);
#define SLK_MS(R_, LG_, CPT_) \
    if (s.R == R_ && s.LG == LG_ && s.CPT == CPT_) return ms_run<R_, LG_, CPT_>(ctx, a);
    SLK_MS(16, 4, 1) SLK_MS(16, 8, 1) SLK_MS(16, 12, 1) SLK_MS(16, 16, 1)
    SLK_MS(16, 4, 2) SLK_MS(16, 8, 2) SLK_MS(16, 12, 2) SLK_MS(16, 16, 2)
    SLK_MS(16, 4, 4) SLK_MS(16, 8, 4) SLK_MS(16, 12, 4) SLK_MS(16, 16, 4)
    SLK_MS(8, 4, 8) SLK_MS(8, 8, 8)
    SLK_MS(4, 4, 16)
#undef SLK_MS
    return set_err(ctx, SLK_ERR_INVALID_ARG, "mean-shift modes: no launch shape");
}

slk_status ms_gather_launch(slk_ctx* ctx, const float* X, int D, const int32_t* idx, int L,
                            float* M, double* M64) {
    SLK_COUNT_LAUNCH(ctx, 1);
    const int64_t n = (int64_t)L * D;
    const unsigned grid = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    ms_gather_kernel<<<grid, 256, 0, ctx->stream>>>(X, D, idx, L, M, M64);
    SLK_LAUNCH_CHECK(ctx, "ms_gather_kernel");
    return SLK_OK;
}

slk_status ms_widen_launch(slk_ctx* ctx, const float* M, int64_t n, double* M64) {
    SLK_COUNT_LAUNCH(ctx, 1);
    const unsigned grid = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    ms_widen_kernel<<<grid, 256, 0, ctx->stream>>>(M, n, M64);
    SLK_LAUNCH_CHECK(ctx, "ms_widen_kernel");
    return SLK_OK;
}

slk_status ms_moved_launch(slk_ctx* ctx, const double* M64, const double* M64_start, int D, int L,
                           MsStatus* ms) {
    SLK_COUNT_LAUNCH(ctx, 1);
    ms_moved_kernel<<<1, 256, 0, ctx->stream>>>(M64, M64_start, D, L, ms);
    SLK_LAUNCH_CHECK(ctx, "ms_moved_kernel");
    return SLK_OK;
}

slk_status ms_split_launch(slk_ctx* ctx, const double* M64, int64_t n, float* Mhi, float* Mlo) {
    SLK_COUNT_LAUNCH(ctx, 1);
    const unsigned grid = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    ms_split_kernel<<<grid, 256, 0, ctx->stream>>>(M64, n, Mhi, Mlo);
    SLK_LAUNCH_CHECK(ctx, "ms_split_kernel");
    return SLK_OK;
}
