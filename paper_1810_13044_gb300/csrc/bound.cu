// Bound iterations (inner loop of Algorithm 1) and the SLK-BO mode update.
//
// z-update, Eq. (soft-max):   z_p <- exp(a_p + lambda b_p) / 1^t exp(a_p + lambda b_p)
// pairwise term, Eq. (general-third): b_{p,l} = sum_{e in row p} w_e z_{col(e), l}
// mode update, Eq. (mode_byproduct):  m_l = argmax_q z_{q,l}
//
// Layout: a "group" of G lanes (G = 4, 8, 16 or 32) owns one row p; lane i of
// the group owns labels i, i + G, ..., so the L floats of a Z row are read as
// one coalesced segment.  The group loads up to G column indices of its row
// with one coalesced load and broadcasts them by shuffle; the neighbour rows
// of Z are then gathered label-parallel.  Row max and row sum use xor
// shuffles inside the group.  Every update of all rows is one pass of a
// persistent cooperative kernel; passes are separated by a device-wide
// barrier whose waits are bounded in time (SLK_ERR_TIMEOUT instead of a hang).
#include <cuda.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "slk_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Device-wide step barrier of the persistent inner loop.  Every block has
// already folded its max |dz| into delta_bits[it % 3] (a reduction without
// return); it adds one to a monotonic arrival counter (release) and waits
// (acquire) until the counter reaches nblocks (it + 1), compared modulo 2^32.
// By then every block's max is in the slot, so each block reads the same
// final delta and takes the same decision (delta <= tol) itself.  Block 0
// clears the slot of update it + 2 (its last readers passed this barrier)
// and records the delta.  Returns 1 (converged), 0 (go on) or -1 (a wait
// gave up after timeout_ns, or another block's did).
__device__ int grid_step(DevState* st, unsigned nblocks, int it, float tol,
                         unsigned long long timeout_ns = kBarrierTimeoutNs) {
    __shared__ int s_res;
    __syncthreads();
    if (threadIdx.x == 0) {
        int res = 0;
        const unsigned target = nblocks * (unsigned)(it + 1);
        red_add_release_gpu(&st->barrier_arrive, 1u);
        const unsigned long long t0 = globaltimer_ns();
        unsigned polls = 0;
        while ((int)(ld_acquire_gpu(&st->barrier_arrive) - target) < 0) {
            if ((++polls & 63u) == 0u) {
                if (ld_acquire_gpu(&st->error) != 0u) { res = -1; break; }
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicOr(&st->error, ERR_BARRIER_TIMEOUT);
                    res = -1;
                    break;
                }
            }
        }
        if (res == 0) {
            const float dl = __uint_as_float(ld_acquire_gpu(&st->delta_bits[it % 3]));
            if (blockIdx.x == 0) {
                st->delta_bits[(it + 2) % 3] = 0u;
                st->last_delta = dl;
            }
            res = (dl <= tol) ? 1 : 0;
        }
        s_res = res;
    }
    __syncthreads();
    return s_res;
}

template <int G>
__device__ __forceinline__ float group_max(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, G));
    return v;
}
// Maximum over the 32 lanes of a warp in one instruction (exact, as the
// butterfly of fmaxf).
__device__ __forceinline__ float warp_max_all(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

// Logits s_{p,l} = a_{p,l} + lambda b_{p,l} of row p for this lane's labels
// l = gl + G j (l >= L gets -inf).  b sums the row's edges in CSR order.
template <int G, int LPL>
__device__ __forceinline__ void row_logits(int64_t p, int gl, unsigned gmask,
                                           const float* __restrict__ A,
                                           const int64_t* __restrict__ row_ptr,
                                           const int32_t* __restrict__ col_idx,
                                           const float* __restrict__ w, const float* Zin,
                                           int L, float lambda, bool with_pair, float (&s)[LPL]) {
    float b[LPL];
#pragma unroll
    for (int j = 0; j < LPL; ++j) b[j] = 0.f;
    if (with_pair) {
        const int64_t e0 = __ldg(row_ptr + p), e1 = __ldg(row_ptr + p + 1);
        for (int64_t base = e0; base < e1; base += G) {
            const int cnt = (int)((e1 - base) < G ? (e1 - base) : G);
            int myq = 0;
            float myw = 1.f;
            if (gl < cnt) {
                myq = __ldg(col_idx + base + gl);
                if (w) myw = __ldg(w + base + gl);
            }
            for (int t = 0; t < cnt; ++t) {
                const int q = __shfl_sync(gmask, myq, t, G);
                const float wq = __shfl_sync(gmask, myw, t, G);
                const float* zq = Zin + (int64_t)q * L;
#pragma unroll
                for (int j = 0; j < LPL; ++j) {
                    const int l = gl + G * j;
                    if (l < L) b[j] = fmaf(wq, __ldcg(zq + l), b[j]);
                }
            }
        }
    }
    const float* ap = A + p * (int64_t)L;
#pragma unroll
    for (int j = 0; j < LPL; ++j) {
        const int l = gl + G * j;
        s[j] = (l < L) ? fmaf(lambda, b[j], __ldg(ap + l)) : -INFINITY;
    }
}

// One z-update of row p: Zout[p] = softmax(s_p); returns max |z_new - z_old|
// over this lane's labels.
template <int G, int LPL>
__device__ __forceinline__ float row_update(int64_t p, int gl, unsigned gmask, const float* A,
                                            const int64_t* row_ptr, const int32_t* col_idx,
                                            const float* w, const float* Zin, float* Zout,
                                            int L, float lambda) {
    float s[LPL];
    row_logits<G, LPL>(p, gl, gmask, A, row_ptr, col_idx, w, Zin, L, lambda, true, s);
    float m = s[0];
#pragma unroll
    for (int j = 1; j < LPL; ++j) m = fmaxf(m, s[j]);
    m = group_max<G>(m, gmask);
    float e[LPL], sum = 0.f;
#pragma unroll
    for (int j = 0; j < LPL; ++j) {
        e[j] = (gl + G * j < L) ? expf(s[j] - m) : 0.f;
        sum += e[j];
    }
    sum = group_sum<G>(sum, gmask);
    float d = 0.f;
    const int64_t off = p * (int64_t)L;
#pragma unroll
    for (int j = 0; j < LPL; ++j) {
        const int l = gl + G * j;
        if (l < L) {
            const float z = e[j] / sum;
            d = fmaxf(d, fabsf(z - __ldcg(Zin + off + l)));
            __stcg(Zout + off + l, z);
        }
    }
    return d;
}

// RPG z-updates per lane group at once: rows p0, p0 + stride, ...  Each
// row's own unary term and previous z are loaded first; neighbour rows of Z
// are then gathered in windows of W per row, RPG x W loads issued before any
// of their FMAs, so that their L2 latencies overlap.  Per row the edges are
// summed in CSR order.  kdeg > 0 means every row has kdeg entries
// (row_ptr[p] = kdeg p) and skips the row_ptr loads.  Returns max
// |z_new - z_old| over this lane's entries.
template <int G, int LPL, int RPG, int W>
__device__ __forceinline__ float rows_update(int64_t p0, int64_t stride, int64_t N, int gl,
                                             unsigned gmask, const float* __restrict__ A,
                                             const int64_t* __restrict__ row_ptr, int kdeg,
                                             const int32_t* __restrict__ col_idx,
                                             const float* __restrict__ w, const float* Zin,
                                             float* Zout, int L, float lambda) {
    int64_t p[RPG], e0[RPG];
    int cnt[RPG];
    int maxc = 0;
    float av[RPG][LPL], zo[RPG][LPL], b[RPG][LPL];
#pragma unroll
    for (int i = 0; i < RPG; ++i) {
        p[i] = p0 + i * stride;
        const bool live = p[i] < N;
        e0[i] = 0;
        cnt[i] = 0;
        if (live) {
            if (kdeg > 0) {
                e0[i] = p[i] * kdeg;
                cnt[i] = kdeg;
            } else {
                e0[i] = __ldg(row_ptr + p[i]);
                cnt[i] = (int)(__ldg(row_ptr + p[i] + 1) - e0[i]);
            }
        }
        maxc = max(maxc, cnt[i]);
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            const bool ok = live && l < L;
            av[i][j] = ok ? __ldg(A + p[i] * (int64_t)L + l) : 0.f;
            zo[i][j] = ok ? __ldcg(Zin + p[i] * (int64_t)L + l) : 0.f;
            b[i][j] = 0.f;
        }
    }
    for (int c0 = 0; c0 < maxc; c0 += G) {
        int myq[RPG];
        float myw[RPG];
#pragma unroll
        for (int i = 0; i < RPG; ++i) {
            myq[i] = 0;
            myw[i] = 1.f;
            if (gl < cnt[i] - c0) {
                myq[i] = __ldg(col_idx + e0[i] + c0 + gl);
                if (w) myw[i] = __ldg(w + e0[i] + c0 + gl);
            }
        }
        const int cm = min(G, maxc - c0);
        for (int t0 = 0; t0 < cm; t0 += W) {
            float zz[RPG][W][LPL], ww[RPG][W];
#pragma unroll
            for (int i = 0; i < RPG; ++i)
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const int t = t0 + u;   // < G: W divides G and t0 < cm <= G
                    const int q = __shfl_sync(gmask, myq[i], t, G);
                    ww[i][u] = __shfl_sync(gmask, myw[i], t, G);
                    const bool ok = t < cnt[i] - c0;
                    const float* zq = Zin + (int64_t)q * L;
#pragma unroll
                    for (int j = 0; j < LPL; ++j) {
                        const int l = gl + G * j;
                        zz[i][u][j] = (ok && l < L) ? __ldcg(zq + l) : 0.f;
                    }
                }
#pragma unroll
            for (int i = 0; i < RPG; ++i)
#pragma unroll
                for (int u = 0; u < W; ++u)
                    if (t0 + u < cnt[i] - c0)
#pragma unroll
                        for (int j = 0; j < LPL; ++j) b[i][j] = fmaf(ww[i][u], zz[i][u][j], b[i][j]);
        }
    }
    float dmax = 0.f;
#pragma unroll
    for (int i = 0; i < RPG; ++i) {
        if (p[i] >= N) continue;  // uniform within the group
        float sv[LPL];
        float m = -INFINITY;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            sv[j] = (l < L) ? fmaf(lambda, b[i][j], av[i][j]) : -INFINITY;
            m = fmaxf(m, sv[j]);
        }
        m = group_max<G>(m, gmask);
        float e[LPL], sum = 0.f;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            e[j] = (gl + G * j < L) ? expf(sv[j] - m) : 0.f;
            sum += e[j];
        }
        sum = group_sum<G>(sum, gmask);
        const int64_t off = p[i] * (int64_t)L;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            if (l < L) {
                const float z = e[j] / sum;
                dmax = fmaxf(dmax, fabsf(z - zo[i][j]));
                __stcg(Zout + off + l, z);
            }
        }
    }
    return dmax;
}

// Rows per group and gather window per row: about 32 loads in flight per lane.
template <int G, int LPL>
#ifndef SLK_BOUND_RPG4
#define SLK_BOUND_RPG4 1
#endif
#ifndef SLK_BOUND_W4
#define SLK_BOUND_W4 4
#endif
#ifndef SLK_BOUND_MINB
#define SLK_BOUND_MINB 1
#endif
struct Tiling {
    static constexpr int rpg = (LPL == 1) ? 4 : (LPL == 2 ? 2 : (LPL == 4 ? SLK_BOUND_RPG4 : 1));
    static constexpr int w = (LPL <= 2) ? (G < 8 ? G : 8) : (LPL == 4 ? SLK_BOUND_W4 : 2);
};

__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float m = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
    return m;  // valid on thread 0
}

// Persistent inner loop.  Update it reads buffer it % 2 and writes the other;
// Z0 holds the starting iterate.
template <int G, int LPL>
__global__ void __launch_bounds__(kThreads, SLK_BOUND_MINB)
bound_persistent_kernel(const float* __restrict__ A, const int64_t* __restrict__ row_ptr,
                        const int32_t* __restrict__ col_idx, const float* __restrict__ w,
                        int64_t N, int L, float lambda, float* Z0, float* Z1, int max_iters,
                        float tol, int kdeg, DevState* st) {
    constexpr int RPW = 32 / G;
    __shared__ float red[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int64_t nwarps = (int64_t)gridDim.x * (kThreads / 32);
    const int64_t gwarp = (int64_t)blockIdx.x * (kThreads / 32) + warp;
    int it = 0;
    while (it < max_iters) {
        const float* Zin = (it & 1) ? Z1 : Z0;
        float* Zout = (it & 1) ? Z0 : Z1;
        float d = 0.f;
        constexpr int RPG = Tiling<G, LPL>::rpg;
        const int64_t stride = nwarps * RPW;
        for (int64_t base = gwarp * RPW + grp; base < N; base += stride * RPG)
            d = fmaxf(d, rows_update<G, LPL, RPG, Tiling<G, LPL>::w>(base, stride, N, gl, gmask, A,
                                                                    row_ptr, kdeg, col_idx, w,
                                                                    Zin, Zout, L, lambda));
        const float bm = block_max(d, red);
        if (threadIdx.x == 0) atomicMax(&st->delta_bits[it % 3], __float_as_uint(bm));
        const int r = grid_step(st, gridDim.x, it, tol);
        if (r < 0) return;
        ++it;
        if (r == 1) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->iters_done = it;
}

// ------------------------------------------------ 16-byte form for 64 < L <= 128
//
// For L a multiple of 4 in (64, 128] one warp owns a row and lane v owns the
// labels 4v .. 4v + 3 (v < L/4), so every row of A and Z -- a unary row, the
// row's previous z and each neighbour's z -- is one 16-byte load per lane,
// and all neighbour rows of a window are in flight together.  The arithmetic
// is that of rows_update<32, 4>, bit for bit: each label sums its edges in
// CSR order, and the row sum of the soft-max is formed in that kernel's
// order (lane s adds the labels s, s + 32, s + 64, s + 96 from 0, then the
// xor butterfly over the 32 lanes), its addends fetched by shuffles.
__device__ __forceinline__ float4 ld4_cg(const float4* p) { return __ldcg(p); }

template <int W, int RPG>
__device__ __forceinline__ float rows_update_vec4(int64_t p0, int64_t stride, int64_t N, int lane,
                                                  const float4* __restrict__ A4,
                                                  const int64_t* __restrict__ row_ptr, int kdeg,
                                                  const int32_t* __restrict__ col_idx,
                                                  const float* __restrict__ w, const float4* Zin4,
                                                  float4* Zout4, int L4, float lambda) {
    const bool act = lane < L4;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int64_t p[RPG], e0[RPG];
    int cnt[RPG];
    int maxc = 0;
    float4 av[RPG], zo[RPG], b[RPG];
#pragma unroll
    for (int i = 0; i < RPG; ++i) {
        p[i] = p0 + i * stride;
        const bool live = p[i] < N;
        e0[i] = 0;
        cnt[i] = 0;
        if (live) {
            if (kdeg > 0) {
                e0[i] = p[i] * kdeg;
                cnt[i] = kdeg;
            } else {
                e0[i] = __ldg(row_ptr + p[i]);
                cnt[i] = (int)(__ldg(row_ptr + p[i] + 1) - e0[i]);
            }
        }
        maxc = max(maxc, cnt[i]);
        av[i] = (live && act) ? __ldg(A4 + p[i] * L4 + lane) : z4;
        zo[i] = (live && act) ? ld4_cg(Zin4 + p[i] * L4 + lane) : z4;
        b[i] = z4;
    }
    for (int c0 = 0; c0 < maxc; c0 += 32) {
        int myq[RPG];
        float myw[RPG];
#pragma unroll
        for (int i = 0; i < RPG; ++i) {
            myq[i] = 0;
            myw[i] = 1.f;
            if (lane < cnt[i] - c0) {
                myq[i] = __ldg(col_idx + e0[i] + c0 + lane);
                if (w) myw[i] = __ldg(w + e0[i] + c0 + lane);
            }
        }
        const int cm = min(32, maxc - c0);
        for (int t0 = 0; t0 < cm; t0 += W) {
            float4 zz[RPG][W];
            float ww[RPG][W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (t0 + u >= cm) break;   // uniform over the warp
#pragma unroll
                for (int i = 0; i < RPG; ++i) {
                    const int q = __shfl_sync(0xffffffffu, myq[i], t0 + u);
                    ww[i][u] = __shfl_sync(0xffffffffu, myw[i], t0 + u);
                    const bool ok = act && (t0 + u < cnt[i] - c0);
                    zz[i][u] = ok ? ld4_cg(Zin4 + (int64_t)q * L4 + lane) : z4;
                }
            }
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (t0 + u >= cm) break;
#pragma unroll
                for (int i = 0; i < RPG; ++i) {
                    if (t0 + u < cnt[i] - c0) {
                        b[i].x = fmaf(ww[i][u], zz[i][u].x, b[i].x);
                        b[i].y = fmaf(ww[i][u], zz[i][u].y, b[i].y);
                        b[i].z = fmaf(ww[i][u], zz[i][u].z, b[i].z);
                        b[i].w = fmaf(ww[i][u], zz[i][u].w, b[i].w);
                    }
                }
            }
        }
    }
    float dmax = 0.f;
#pragma unroll
    for (int i = 0; i < RPG; ++i) {
        if (p[i] >= N) continue;  // uniform over the warp
        float4 sv;
        sv.x = act ? fmaf(lambda, b[i].x, av[i].x) : -INFINITY;
        sv.y = act ? fmaf(lambda, b[i].y, av[i].y) : -INFINITY;
        sv.z = act ? fmaf(lambda, b[i].z, av[i].z) : -INFINITY;
        sv.w = act ? fmaf(lambda, b[i].w, av[i].w) : -INFINITY;
        float m = fmaxf(fmaxf(sv.x, sv.y), fmaxf(sv.z, sv.w));
        m = group_max<32>(m, 0xffffffffu);
        float4 e;
        e.x = act ? expf(sv.x - m) : 0.f;
        e.y = act ? expf(sv.y - m) : 0.f;
        e.z = act ? expf(sv.z - m) : 0.f;
        e.w = act ? expf(sv.w - m) : 0.f;
        // lane s adds labels s + 32 j (j = 0..3), held by lane s/4 + 8 j as
        // component s % 4, in the order of the label-strided kernel
        float part = 0.f;
        const int c = lane & 3;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int src = (lane >> 2) + 8 * j;
            const float ex = __shfl_sync(0xffffffffu, e.x, src);
            const float ey = __shfl_sync(0xffffffffu, e.y, src);
            const float ez = __shfl_sync(0xffffffffu, e.z, src);
            const float ew = __shfl_sync(0xffffffffu, e.w, src);
            part += (c == 0) ? ex : (c == 1) ? ey : (c == 2) ? ez : ew;
        }
        const float sum = group_sum<32>(part, 0xffffffffu);
        if (act) {
            float4 z;
            z.x = e.x / sum;
            z.y = e.y / sum;
            z.z = e.z / sum;
            z.w = e.w / sum;
            dmax = fmaxf(dmax, fmaxf(fmaxf(fabsf(z.x - zo[i].x), fabsf(z.y - zo[i].y)),
                                     fmaxf(fabsf(z.z - zo[i].z), fabsf(z.w - zo[i].w))));
            __stcg(Zout4 + p[i] * L4 + lane, z);
        }
    }
    return dmax;
}

#ifndef SLK_BOUND_VEC_W
#define SLK_BOUND_VEC_W 12
#endif
#ifndef SLK_BOUND_VEC_RPG
#define SLK_BOUND_VEC_RPG 1
#endif

// Persistent inner loop in the 16-byte form (64 < L <= 128, L % 4 == 0,
// 16-byte aligned A, Z0, Z1); barrier, convergence and results as
// bound_persistent_kernel<32, 4>.
__global__ void __launch_bounds__(kThreads, SLK_BOUND_MINB)
bound_vec4_kernel(const float* __restrict__ A, const int64_t* __restrict__ row_ptr,
                  const int32_t* __restrict__ col_idx, const float* __restrict__ w, int64_t N,
                  int L, float lambda, float* Z0, float* Z1, int max_iters, float tol, int kdeg,
                  DevState* st) {
    __shared__ float red[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (kThreads / 32);
    const int64_t gwarp = (int64_t)blockIdx.x * (kThreads / 32) + warp;
    const int L4 = L >> 2;
    const float4* A4 = reinterpret_cast<const float4*>(A);
    constexpr int RPG = SLK_BOUND_VEC_RPG;
    int it = 0;
    while (it < max_iters) {
        const float4* Zin4 = reinterpret_cast<const float4*>((it & 1) ? Z1 : Z0);
        float4* Zout4 = reinterpret_cast<float4*>((it & 1) ? Z0 : Z1);
        float d = 0.f;
        for (int64_t base = gwarp; base < N; base += nwarps * RPG)
            d = fmaxf(d, rows_update_vec4<SLK_BOUND_VEC_W, RPG>(base, nwarps, N, lane, A4, row_ptr,
                                                                 kdeg, col_idx, w, Zin4, Zout4, L4,
                                                                 lambda));
        const float bm = block_max(d, red);
        if (threadIdx.x == 0) atomicMax(&st->delta_bits[it % 3], __float_as_uint(bm));
        const int r = grid_step(st, gridDim.x, it, tol);
        if (r < 0) return;
        ++it;
        if (r == 1) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->iters_done = it;
}

// ------------------------------------- staged form for large N (64 < L <= 128)
//
// The 16-byte form above keeps about 16 rows per SM in flight, each waiting
// on its names, then on its neighbours' rows: at 1e6 rows the z-updates are
// bound by that latency and by the instructions per row, not by HBM (a
// graph of self-loops runs as slowly as a random one).  Here every warp
// runs a pipeline of S row stages in shared memory: while it computes row
// j, the cp.async copies of rows j+1 .. j+S-1 (unary row, previous z row
// and the kdeg neighbour z rows, 16 bytes a lane) are in flight, and the
// neighbour names of rows j+S .. j+2S-1 arrive in a ring of 2S slots S rows
// ahead of their gathers, so no row waits on its names.  Each label sums
// its edges in CSR order as in the other forms; the soft-max takes the row
// sum from each lane's own four terms and one reciprocal per row (z = e
// (1 / sum), within 1.5 ulp of e / sum), fewer instructions than the
// label-strided order of the other forms, whose bits it therefore does not
// repeat.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int P>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(P) : "memory");
}

// Shared memory of one warp: S stages of (2 + kdeg) rows of L4 float4 (unary
// row, previous z row, neighbour z rows), then 2S slots of kdeg names and
// kdeg weights.
__host__ __device__ constexpr size_t staged_warp_bytes(int S, int kdeg, int L4) {
    return (size_t)S * (2 + kdeg) * L4 * 16 + (size_t)2 * S * kdeg * 8;
}

// K > 0: every row has K edges, known at compile time (loops unrolled);
// K = 0: kdeg_rt edges.  Element offsets are 32-bit (N L / 4 < 2^31).
template <int S, int WPB, int K>
__global__ void __launch_bounds__(WPB * 32, 1)
bound_staged_kernel(const float* __restrict__ A, const int32_t* __restrict__ col_idx,
                    const float* __restrict__ w, int64_t N, int L, float lambda, float* Z0,
                    float* Z1, int max_iters, float tol, int kdeg_rt, DevState* st) {
    extern __shared__ __align__(16) unsigned char stage_sm[];
    __shared__ float red[WPB];
    const int kdeg = K > 0 ? K : kdeg_rt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwarps = gridDim.x * WPB;
    const uint32_t gwarp = blockIdx.x * WPB + warp;
    const uint32_t L4 = (uint32_t)L >> 2;
    const bool act = (uint32_t)lane < L4;
    const int srows = 2 + kdeg;
    unsigned char* mine = stage_sm + (size_t)warp * staged_warp_bytes(S, kdeg, (int)L4);
    float4* stg = reinterpret_cast<float4*>(mine);                        // [S][srows][L4]
    int32_t* qring = reinterpret_cast<int32_t*>(mine + (size_t)S * srows * L4 * 16);   // [2S][kdeg]
    float* wring = reinterpret_cast<float*>(qring + 2 * S * kdeg);                     // [2S][kdeg]
    const float4* A4 = reinterpret_cast<const float4*>(A);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // rows of this warp: gwarp + j nwarps, j < nj
    const uint32_t nj = ((uint64_t)N > gwarp) ? (uint32_t)(((uint64_t)N - gwarp + nwarps - 1) / nwarps) : 0u;
    int it = 0;
    while (it < max_iters) {
        const float4* Zin4 = reinterpret_cast<const float4*>((it & 1) ? Z1 : Z0);
        float4* Zout4 = reinterpret_cast<float4*>((it & 1) ? Z0 : Z1);
        // names and weights of row j into ring slot j % 2S
        auto fetch_names = [&](uint32_t j) {
            if (j < nj && lane < kdeg) {
                const uint32_t e = (gwarp + j * nwarps) * (uint32_t)kdeg + lane;
                const int slot = (int)(j % (2 * S));
                cp_async4(qring + slot * kdeg + lane, col_idx + e);
                if (w) cp_async4(wring + slot * kdeg + lane, w + e);
            }
        };
        // unary row, previous z row and neighbour rows of row j into stage j % S
        auto fetch_rows = [&](uint32_t j) {
            if (j < nj && act) {
                const uint32_t o = (gwarp + j * nwarps) * L4 + lane;
                float4* sb = stg + (j % S) * srows * L4 + lane;
                const int32_t* qs = qring + (j % (2 * S)) * kdeg;
                cp_async16(sb, A4 + o);
                cp_async16(sb + L4, Zin4 + o);
#pragma unroll
                for (int t = 0; t < kdeg; ++t)
                    cp_async16(sb + (2 + t) * L4, Zin4 + ((uint32_t)qs[t] * L4 + lane));
            }
        };
        // prologue: names of rows 0 .. S-1 (waited for), then the stages of
        // rows 0 .. S-2 with the names of rows S .. 2S-2 (one group each)
        for (int j = 0; j < S; ++j) fetch_names(j);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        for (int j = 0; j < S - 1; ++j) {
            fetch_rows(j);
            fetch_names(j + S);
            cp_async_commit();
        }
        float d = 0.f;
        for (uint32_t j = 0; j < nj; ++j) {
            // group j + S - 1: the stage of row j+S-1 (its names arrived with
            // group j-1, waited for in the previous iteration) and the names
            // of row j+2S-1
            fetch_rows(j + S - 1);
            fetch_names(j + 2 * S - 1);
            cp_async_commit();
            cp_async_wait<S - 1>();   // group j: the stage of row j
            __syncwarp();
            const uint32_t o = (gwarp + j * nwarps) * L4 + lane;
            const float4* sb = stg + (j % S) * srows * L4 + lane;
            const float* ws = wring + (j % (2 * S)) * kdeg;
            float4 b = z4;
            if (act) {
#pragma unroll
                for (int t = 0; t < kdeg; ++t) {
                    const float wt = w ? ws[t] : 1.f;
                    const float4 zq = sb[(2 + t) * L4];
                    b.x = fmaf(wt, zq.x, b.x);
                    b.y = fmaf(wt, zq.y, b.y);
                    b.z = fmaf(wt, zq.z, b.z);
                    b.w = fmaf(wt, zq.w, b.w);
                }
            }
            const float4 av = act ? sb[0] : z4;
            const float4 zo = act ? sb[L4] : z4;
            float4 sv;
            sv.x = act ? fmaf(lambda, b.x, av.x) : -INFINITY;
            sv.y = act ? fmaf(lambda, b.y, av.y) : -INFINITY;
            sv.z = act ? fmaf(lambda, b.z, av.z) : -INFINITY;
            sv.w = act ? fmaf(lambda, b.w, av.w) : -INFINITY;
            const float m = warp_max_all(fmaxf(fmaxf(sv.x, sv.y), fmaxf(sv.z, sv.w)));
            // exp(x), x = s - m <= 0, by the fast intrinsic: its error of at
            // most (2 + 1.16 |x|) ulp of e^x is below 2e-7 absolute for every
            // x <= 0 (e^x (2 + 1.16 |x|) peaks at x = 0), so z moves by less
            // than that
            float4 e;
            e.x = act ? __expf(sv.x - m) : 0.f;
            e.y = act ? __expf(sv.y - m) : 0.f;
            e.z = act ? __expf(sv.z - m) : 0.f;
            e.w = act ? __expf(sv.w - m) : 0.f;
            // the row sum from the lanes' own four terms, and one reciprocal
            // per row: z = e (1 / sum), within 1.5 ulp of e / sum
            const float sum = group_sum<32>((e.x + e.y) + (e.z + e.w), 0xffffffffu);
            const float inv = 1.f / sum;
            if (act) {
                float4 z;
                z.x = e.x * inv;
                z.y = e.y * inv;
                z.z = e.z * inv;
                z.w = e.w * inv;
                d = fmaxf(d, fmaxf(fmaxf(fabsf(z.x - zo.x), fabsf(z.y - zo.y)),
                                   fmaxf(fabsf(z.z - zo.z), fabsf(z.w - zo.w))));
                __stcg(Zout4 + o, z);
            }
            __syncwarp();   // the stage is refilled by the next iteration's copies
        }
        cp_async_wait<0>();
        __syncwarp();
        const float bm = block_max(d, red);
        if (threadIdx.x == 0) atomicMax(&st->delta_bits[it % 3], __float_as_uint(bm));
        const int r = grid_step(st, gridDim.x, it, tol);
        if (r < 0) return;
        ++it;
        if (r == 1) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->iters_done = it;
}

// rows_update on operands cached in shared memory: the CTA's rows
// [r0, r0 + nr) keep their unary terms sA[lr][L], column indices
// sQ[lr][kdeg] and weights sW[lr][kdeg] (lr = p - r0) there for the whole
// inner loop, so an update reads only Z from L2.  Rows lr0, lr0 + lstride,
// ...; the arithmetic (edge order, windows, soft-max) is that of rows_update.
template <int G, int LPL, int RPG, int W>
__device__ __forceinline__ float rows_update_cached(int lr0, int lstride, int nr, int64_t r0, int gl,
                                                    unsigned gmask, const float* sA, const int* sQ,
                                                    const float* sW, int kdeg, const float* Zin,
                                                    float* Zout, int L, float lambda) {
    int lr[RPG], cnt[RPG];
    int maxc = 0;
    float av[RPG][LPL], zo[RPG][LPL], b[RPG][LPL];
#pragma unroll
    for (int i = 0; i < RPG; ++i) {
        lr[i] = lr0 + i * lstride;
        const bool live = lr[i] < nr;
        cnt[i] = live ? kdeg : 0;
        maxc = max(maxc, cnt[i]);
        const int64_t p = r0 + lr[i];
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            const bool ok = live && l < L;
            av[i][j] = ok ? sA[lr[i] * L + l] : 0.f;
            zo[i][j] = ok ? __ldcg(Zin + p * (int64_t)L + l) : 0.f;
            b[i][j] = 0.f;
        }
    }
    // neighbour names and weights straight from shared memory (every lane of
    // a group reads the same word); windows of W edges, slots beyond the
    // row's degree skipped with a warp-uniform test
    for (int t0 = 0; t0 < maxc; t0 += W) {
        float zz[RPG][W][LPL], ww[RPG][W];
#pragma unroll
        for (int u = 0; u < W; ++u) {
            if (t0 + u >= maxc) break;   // maxc = kdeg for every live row: uniform
#pragma unroll
            for (int i = 0; i < RPG; ++i) {
                const bool ok = t0 + u < cnt[i];
                const int q = ok ? sQ[lr[i] * kdeg + t0 + u] : 0;
                ww[i][u] = (ok && sW) ? sW[lr[i] * kdeg + t0 + u] : 1.f;
                const float* zq = Zin + (int64_t)q * L;
#pragma unroll
                for (int j = 0; j < LPL; ++j) {
                    const int l = gl + G * j;
                    zz[i][u][j] = (ok && l < L) ? __ldcg(zq + l) : 0.f;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < W; ++u) {
            if (t0 + u >= maxc) break;
#pragma unroll
            for (int i = 0; i < RPG; ++i)
                if (t0 + u < cnt[i])
#pragma unroll
                    for (int j = 0; j < LPL; ++j) b[i][j] = fmaf(ww[i][u], zz[i][u][j], b[i][j]);
        }
    }
    float dmax = 0.f;
#pragma unroll
    for (int i = 0; i < RPG; ++i) {
        if (lr[i] >= nr) continue;  // uniform within the group
        float sv[LPL];
        float m = -INFINITY;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            sv[j] = (l < L) ? fmaf(lambda, b[i][j], av[i][j]) : -INFINITY;
            m = fmaxf(m, sv[j]);
        }
        m = group_max<G>(m, gmask);
        float e[LPL], sum = 0.f;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            e[j] = (gl + G * j < L) ? expf(sv[j] - m) : 0.f;
            sum += e[j];
        }
        sum = group_sum<G>(sum, gmask);
        const int64_t off = (r0 + lr[i]) * (int64_t)L;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            if (l < L) {
                const float z = e[j] / sum;
                dmax = fmaxf(dmax, fabsf(z - zo[i][j]));
                __stcg(Zout + off + l, z);
            }
        }
    }
    return dmax;
}

#ifndef SLK_BOUND_CACHED_RPG2
#define SLK_BOUND_CACHED_RPG2 2
#endif
template <int LPL>
struct CachedTiling {
    static constexpr int rpg = (LPL == 1) ? 4 : (LPL == 2 ? SLK_BOUND_CACHED_RPG2 : (LPL == 4 ? 2 : 1));
};

// Persistent inner loop over a fixed-degree graph (kdeg edges per row) with
// each CTA's operands cached in shared memory: CTA b owns rows
// [b rpc, (b + 1) rpc).  Same updates, barrier and results as
// bound_persistent_kernel.
template <int G, int LPL>
__global__ void __launch_bounds__(kThreads, SLK_BOUND_MINB)
bound_cached_kernel(const float* __restrict__ A, const int32_t* __restrict__ col_idx,
                    const float* __restrict__ w, int64_t N, int L, float lambda, float* Z0,
                    float* Z1, int max_iters, float tol, int kdeg, int rpc, DevState* st) {
    extern __shared__ __align__(16) float csm[];
    constexpr int RPW = 32 / G;
    __shared__ float red[kThreads / 32];
    const int64_t r0 = (int64_t)blockIdx.x * rpc;
    const int nr = (int)(N - r0 < (int64_t)rpc ? (N - r0 > 0 ? N - r0 : 0) : rpc);
    float* sA = csm;                                            // [rpc][L]
    int* sQ = reinterpret_cast<int*>(sA + (size_t)rpc * L);     // [rpc][kdeg]
    float* sW = w ? reinterpret_cast<float*>(sQ + (size_t)rpc * kdeg) : nullptr;   // [rpc][kdeg]
    for (int i = threadIdx.x; i < nr * L; i += kThreads) sA[i] = __ldg(A + r0 * L + i);
    for (int i = threadIdx.x; i < nr * kdeg; i += kThreads) {
        sQ[i] = __ldg(col_idx + r0 * kdeg + i);
        if (w) sW[i] = __ldg(w + r0 * kdeg + i);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int gidx = warp * RPW + grp;
    constexpr int ng = (kThreads / 32) * RPW;   // groups per CTA
    constexpr int RPG = CachedTiling<LPL>::rpg;
    int it = 0;
    while (it < max_iters) {
        const float* Zin = (it & 1) ? Z1 : Z0;
        float* Zout = (it & 1) ? Z0 : Z1;
        float d = 0.f;
        for (int lr0 = gidx; lr0 < nr; lr0 += ng * RPG)
            d = fmaxf(d, rows_update_cached<G, LPL, RPG, Tiling<G, LPL>::w>(
                             lr0, ng, nr, r0, gl, gmask, sA, sQ, sW, kdeg, Zin, Zout, L, lambda));
        const float bm = block_max(d, red);
        if (threadIdx.x == 0) atomicMax(&st->delta_bits[it % 3], __float_as_uint(bm));
        const int r = grid_step(st, gridDim.x, it, tol);
        if (r < 0) return;
        ++it;
        if (r == 1) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->iters_done = it;
}

// One update per launch (used when cooperative launch is unavailable).  The
// launch for update `it` first looks at the previous update's delta and, once
// converged, does nothing.
template <int G, int LPL>
__global__ void __launch_bounds__(kThreads)
bound_step_kernel(const float* __restrict__ A, const int64_t* __restrict__ row_ptr,
                  const int32_t* __restrict__ col_idx, const float* __restrict__ w, int64_t N,
                  int L, float lambda, float* Z0, float* Z1, int it, float tol, DevState* st) {
    constexpr int RPW = 32 / G;
    __shared__ float red[kThreads / 32];
    if (it > 0) {
        const float prev = __uint_as_float(*(volatile unsigned*)&st->delta_bits[(it - 1) % 3]);
        if (*(volatile int*)&st->iters_done >= 0 || prev <= tol) {
            if (blockIdx.x == 0 && threadIdx.x == 0 && st->iters_done < 0) {
                st->iters_done = it;
                st->last_delta = prev;
            }
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->delta_bits[(it + 1) % 3] = 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const float* Zin = (it & 1) ? Z1 : Z0;
    float* Zout = (it & 1) ? Z0 : Z1;
    const int64_t p = ((int64_t)blockIdx.x * (kThreads / 32) + warp) * RPW + grp;
    float d = 0.f;
    if (p < N) d = row_update<G, LPL>(p, gl, gmask, A, row_ptr, col_idx, w, Zin, Zout, L, lambda);
    const float bm = block_max(d, red);
    if (threadIdx.x == 0) atomicMax(&st->delta_bits[it % 3], __float_as_uint(bm));
}

// The device-wide barrier of the persistent kernels, waited on by one block
// against an arrival target of nblocks_expected blocks that no other block
// will join: its wait must give up after timeout_ns and set the error bit.
__global__ void barrier_probe_kernel(DevState* st, unsigned nblocks_expected,
                                     unsigned long long timeout_ns) {
    grid_step(st, nblocks_expected, 0, -1.f, timeout_ns);
}

__global__ void bound_finish_kernel(int max_iters, DevState* st) {
    if (st->iters_done < 0) {
        st->iters_done = max_iters;
        st->last_delta = max_iters > 0 ? __uint_as_float(st->delta_bits[(max_iters - 1) % 3]) : 0.f;
    }
}

// After the loop the last iterate sits in buffer iters_done % 2; move it to Z.
// iters_done < 0 (a barrier wait gave up) leaves both buffers as they are.
__global__ void swap_if_odd_kernel(float* Z, float* Zp, int64_t n, const DevState* st) {
    if (st->iters_done < 0 || (st->iters_done & 1) == 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float a = Z[i];
        Z[i] = Zp[i];
        Zp[i] = a;
    }
}

// --------------------------------------------------------------------------- mode update

// Per row q: logits s (from Z_prev, or s = a when there was no update),
// label = argmax_l s (ties to the smaller l) and keys
// log z_{q,l} = (s_l - m) - log1p(sum_{j != j*} exp(s_j - m)).  Each block
// keeps the best (key, q) of every label in shared memory, packed so that one
// 64-bit max picks the larger key and, on equal keys, the smaller q.
template <int G, int LPL>
__global__ void __launch_bounds__(kThreads)
mode_rows_kernel(const float* __restrict__ A, const float* __restrict__ Zp,
                 const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                 const float* __restrict__ w, int64_t N, int L, float lambda, int use_iters_flag,
                 int32_t* __restrict__ labels, const int32_t* __restrict__ orig, DevState* st) {
    constexpr int RPW = 32 / G;
    __shared__ unsigned long long best[SLK_MAX_L];
    for (int l = threadIdx.x; l < L; l += kThreads) best[l] = 0ull;
    __syncthreads();
    const bool with_pair = (Zp != nullptr) && (!use_iters_flag || st->iters_done > 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int64_t nwarps = (int64_t)gridDim.x * (kThreads / 32);
    const int64_t gwarp = (int64_t)blockIdx.x * (kThreads / 32) + warp;
    for (int64_t base = gwarp * RPW; base < N; base += nwarps * RPW) {
        const int64_t q = base + grp;
        if (q >= N) continue;  // whole group skips together
        float s[LPL];
        row_logits<G, LPL>(q, gl, gmask, A, row_ptr, col_idx, w, Zp, L, lambda, with_pair, s);
        // group argmax with ties to the smaller label
        float m = s[0];
        int jl = gl;
#pragma unroll
        for (int j = 1; j < LPL; ++j)
            if (s[j] > m) { m = s[j]; jl = gl + G * j; }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const float om = __shfl_xor_sync(gmask, m, o, G);
            const int ol = __shfl_xor_sync(gmask, jl, o, G);
            if (om > m || (om == m && ol < jl)) { m = om; jl = ol; }
        }
        float r = 0.f;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            if (l < L && l != jl) r += expf(s[j] - m);
        }
        r = group_sum<G>(r, gmask);
        const float lse1 = log1pf(r);
        if (gl == 0 && labels) labels[q] = jl;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            if (l < L) {
                const float key = (s[j] - m) - lse1;
                // ties go to the smaller original point index
                const unsigned qo = orig ? (unsigned)orig[q] : (unsigned)q;
                const unsigned long long packed =
                    ((unsigned long long)float_to_ordered(key) << 32) |
                    (unsigned long long)(0xffffffffu - qo);
                atomicMax(&best[l], packed);
            }
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += kThreads)
        if (best[l]) atomicMax(&st->mode_best[l], best[l]);
}

// log z of every row and label (SLK-MS weights, Eq. mean-shift) and labels:
// logits from the previous iterate as in mode_rows_kernel, then
// log z_{q,l} = (s_l - max s) - log1p(sum_{j != argmax} exp(s_j - max s)).
template <int G, int LPL>
__global__ void __launch_bounds__(kThreads)
logz_rows_kernel(const float* __restrict__ A, const float* __restrict__ Zp,
                 const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                 const float* __restrict__ w, int64_t N, int L, float lambda, int use_iters_flag,
                 int32_t* __restrict__ labels, float* __restrict__ LZ, const DevState* st) {
    constexpr int RPW = 32 / G;
    const bool with_pair = (Zp != nullptr) && (!use_iters_flag || st->iters_done > 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int64_t nwarps = (int64_t)gridDim.x * (kThreads / 32);
    const int64_t gwarp = (int64_t)blockIdx.x * (kThreads / 32) + warp;
    for (int64_t base = gwarp * RPW; base < N; base += nwarps * RPW) {
        const int64_t q = base + grp;
        if (q >= N) continue;  // whole group skips together
        float s[LPL];
        row_logits<G, LPL>(q, gl, gmask, A, row_ptr, col_idx, w, Zp, L, lambda, with_pair, s);
        float m = s[0];
        int jl = gl;
#pragma unroll
        for (int j = 1; j < LPL; ++j)
            if (s[j] > m) { m = s[j]; jl = gl + G * j; }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const float om = __shfl_xor_sync(gmask, m, o, G);
            const int ol = __shfl_xor_sync(gmask, jl, o, G);
            if (om > m || (om == m && ol < jl)) { m = om; jl = ol; }
        }
        float r = 0.f;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            if (l < L && l != jl) r += expf(s[j] - m);
        }
        r = group_sum<G>(r, gmask);
        const float lse1 = log1pf(r);
        if (gl == 0 && labels) labels[q] = jl;
#pragma unroll
        for (int j = 0; j < LPL; ++j) {
            const int l = gl + G * j;
            if (l < L) LZ[q * L + l] = (s[j] - m) - lse1;
        }
    }
}

__global__ void mode_finish_kernel(int L, int32_t* modes, float* mode_key, const int32_t* inv,
                                   DevState* st) {
    __shared__ int changed;
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const unsigned long long b = st->mode_best[l];
        const int qo = (int)(0xffffffffu - (unsigned)(b & 0xffffffffull));
        const int q = inv ? inv[qo] : qo;   // back to the rows' (permuted) order
        if (q != modes[l]) changed = 1;  // benign race: every writer stores 1
        modes[l] = q;
        if (mode_key) mode_key[l] = ordered_to_float((unsigned)(b >> 32));
        st->mode_best[l] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) st->changed = changed;
}

// ---------------------------------------------------------------- dispatch on L

struct Shape {
    int G, LPL;
};
Shape shape_for(int L) {
    if (L <= 4) return {4, 1};
    if (L <= 8) return {8, 1};
    if (L <= 16) return {8, 2};
    if (L <= 32) return {16, 2};
    if (L <= 64) return {32, 2};
    if (L <= 128) return {32, 4};
    return {32, 8};
}

#define SLK_DISPATCH_L(L, MACRO)                 \
    do {                                         \
        Shape _s = shape_for(L);                 \
        if (_s.G == 4) { MACRO(4, 1); }          \
        else if (_s.G == 8 && _s.LPL == 1) { MACRO(8, 1); }     \
        else if (_s.G == 8) { MACRO(8, 2); }     \
        else if (_s.G == 16) { MACRO(16, 2); }   \
        else if (_s.LPL == 2) { MACRO(32, 2); }  \
        else if (_s.LPL == 4) { MACRO(32, 4); }  \
        else { MACRO(32, 8); }                   \
    } while (0)

constexpr size_t kCachedSmemMax = 96 * 1024;   // bytes of cached operands per CTA
constexpr size_t kStagedSmemMax = 200 * 1024;  // stages of the pipelined kernel per CTA
constexpr int64_t kStagedMinRows = 100000;     // below: the graph sits in L2, latency is short

// Launches bound_cached_kernel when the graph has a fixed degree and every
// CTA's share of A, col_idx and w fits kCachedSmemMax with all CTAs resident;
// *used says whether it did.
template <int G, int LPL>
cudaError_t launch_cached(slk_ctx* ctx, const float* A, const int32_t* col_idx, const float* w,
                          int64_t N, int L, float lambda, float* Z, float* Z_prev, int max_iters,
                          float tol, int kdeg, DevState* st, bool* used) {
    *used = false;
    auto kern = bound_cached_kernel<G, LPL>;
    const size_t per_row = sizeof(float) * L + sizeof(int) * kdeg + (w ? sizeof(float) * kdeg : 0);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    for (int tries = 0; tries < 4 && per_sm >= 1; ++tries) {
        const int64_t grid = (int64_t)per_sm * ctx->num_sms;
        const int64_t rpc = (N + grid - 1) / grid;
        const size_t smem = per_row * (size_t)rpc;
        if (smem > kCachedSmemMax) return cudaSuccess;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int fit = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, kThreads, smem);
        if (e != cudaSuccess) return e;
        if (fit >= per_sm) {
            const int64_t g2 = (N + rpc - 1) / rpc;   // <= grid: every CTA is resident
            const float* a_ = A; const int32_t* ci_ = col_idx; const float* w_ = w;
            int64_t n_ = N; int l_ = L; float lam_ = lambda; float* z0_ = Z; float* z1_ = Z_prev;
            int mi_ = max_iters; float tol_ = tol; int kd_ = kdeg; int rpc_ = (int)rpc;
            DevState* st_ = st;
            void* args[] = {&a_, &ci_, &w_, &n_, &l_, &lam_, &z0_, &z1_, &mi_, &tol_, &kd_, &rpc_, &st_};
            *used = true;
            return cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)g2), dim3(kThreads),
                                               args, smem, ctx->stream);
        }
        per_sm = fit;
    }
    return cudaSuccess;
}

// Launches bound_staged_kernel<S, WPB> when its stages fit kStagedSmemMax
// with one resident CTA per SM; *used says whether it did.
template <int S, int WPB>
cudaError_t launch_staged(slk_ctx* ctx, const float* A, const int32_t* col_idx, const float* w,
                          int64_t N, int L, float lambda, float* Z, float* Z_prev, int max_iters,
                          float tol, int kdeg, DevState* st, bool* used) {
    *used = false;
    auto kern = kdeg == 10 ? bound_staged_kernel<S, WPB, 10>
              : kdeg == 5  ? bound_staged_kernel<S, WPB, 5>
                           : bound_staged_kernel<S, WPB, 0>;
    const size_t smem = WPB * staged_warp_bytes(S, kdeg, L / 4);
    if (smem > kStagedSmemMax) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPB * 32, smem);
    if (e != cudaSuccess || per_sm < 1) return e;
    int64_t grid = (int64_t)per_sm * ctx->num_sms;
    const int64_t vblocks = (N + WPB - 1) / WPB;
    if (grid > vblocks) grid = vblocks;
    const float* a_ = A; const int32_t* ci_ = col_idx; const float* w_ = w;
    int64_t n_ = N; int l_ = L; float lam_ = lambda; float* z0_ = Z; float* z1_ = Z_prev;
    int mi_ = max_iters; float tol_ = tol; int kd_ = kdeg; DevState* st_ = st;
    void* args[] = {&a_, &ci_, &w_, &n_, &l_, &lam_, &z0_, &z1_, &mi_, &tol_, &kd_, &st_};
    *used = true;
    return cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(WPB * 32), args,
                                       smem, ctx->stream);
}

}  // namespace

slk_status bound_launch(slk_ctx* ctx, const float* A, const int64_t* row_ptr,
                        const int32_t* col_idx, const float* w, int64_t N, int L, float lambda,
                        float* Z, float* Z_prev, int max_iters, float tol, DevState* st,
                        int kdeg) {
    PhaseScope ps(ctx, SLK_PHASE_BOUND);
    // reset barrier / delta state; iters_done = -1 marks "not finished"
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(st, 0, offsetof(DevState, iters_done), ctx->stream));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->iters_done, 0xff, sizeof(int), ctx->stream));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->delta_bits[0], 0, sizeof(st->delta_bits), ctx->stream));
    if (max_iters == 0) {
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->iters_done, 0, sizeof(int), ctx->stream));
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->last_delta, 0, sizeof(float), ctx->stream));
        return SLK_OK;
    }
    const Shape sh = shape_for(L);
    const int rows_per_block = (kThreads / 32) * (32 / sh.G);
    const int64_t blocks_needed = (N + rows_per_block - 1) / rows_per_block;
    cudaError_t e = cudaSuccess;
    if (ctx->coop_supported) {
        SLK_COUNT_LAUNCH(ctx, 1);
        bool cached = false;
#define SLK_LAUNCH_CACHED(G_, LPL_)                                                            \
    e = launch_cached<G_, LPL_>(ctx, A, col_idx, w, N, L, lambda, Z, Z_prev, max_iters, tol,   \
                                kdeg, st, &cached);
        if (kdeg > 0) SLK_DISPATCH_L(L, SLK_LAUNCH_CACHED);
#undef SLK_LAUNCH_CACHED
        if (e != cudaSuccess) return cuda_err(ctx, e, "bound_cached_kernel");
        const bool aligned16 = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Z) |
                                 reinterpret_cast<uintptr_t>(Z_prev)) & 15) == 0;
        if (!cached && L % 4 == 0 && L > 64 && L <= 128 && aligned16 && kdeg > 0 &&
            kdeg <= SLK_MAX_K && N >= kStagedMinRows && N * (int64_t)L < ((int64_t)1 << 32)) {
            // shared-memory pipeline: SLK_BOUND_WPB warps per CTA, the
            // deepest stage count that fits
#ifndef SLK_BOUND_WPB
#define SLK_BOUND_WPB 16
#endif

            constexpr int WPB = SLK_BOUND_WPB;
            e = launch_staged<5, WPB>(ctx, A, col_idx, w, N, L, lambda, Z, Z_prev, max_iters, tol,
                                      kdeg, st, &cached);
            if (e == cudaSuccess && !cached)
                e = launch_staged<4, WPB>(ctx, A, col_idx, w, N, L, lambda, Z, Z_prev, max_iters,
                                          tol, kdeg, st, &cached);
            if (e == cudaSuccess && !cached)
                e = launch_staged<3, WPB>(ctx, A, col_idx, w, N, L, lambda, Z, Z_prev, max_iters,
                                          tol, kdeg, st, &cached);
            if (e == cudaSuccess && !cached)
                e = launch_staged<2, WPB>(ctx, A, col_idx, w, N, L, lambda, Z, Z_prev, max_iters,
                                          tol, kdeg, st, &cached);
            if (e != cudaSuccess) return cuda_err(ctx, e, "bound_staged_kernel");
        }
        if (!cached && L % 4 == 0 && L > 64 && L <= 128 && aligned16) {
            auto kern = bound_vec4_kernel;
            int per_sm = 0;
            SLK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
            if (per_sm < 1) return set_err(ctx, SLK_ERR_CUDA, "bound kernel cannot be resident");
            int64_t grid = (int64_t)per_sm * ctx->num_sms;
            const int64_t vblocks = (N + (kThreads / 32) - 1) / (kThreads / 32);
            if (grid > vblocks) grid = vblocks;
            const float* a_ = A; const int64_t* rp_ = row_ptr; const int32_t* ci_ = col_idx;
            const float* w_ = w; int64_t n_ = N; int l_ = L; float lam_ = lambda;
            float* z0_ = Z; float* z1_ = Z_prev; int mi_ = max_iters; float tol_ = tol;
            int kd_ = kdeg; DevState* st_ = st;
            void* args[] = {&a_, &rp_, &ci_, &w_, &n_, &l_, &lam_, &z0_, &z1_, &mi_, &tol_, &kd_, &st_};
            e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(kThreads),
                                            args, 0, ctx->stream);
            if (e != cudaSuccess) return cuda_err(ctx, e, "bound_vec4_kernel");
            cached = true;   // launched: skip the label-strided kernel below
        }
#define SLK_LAUNCH_PERSISTENT(G_, LPL_)                                                        \
    if (!cached) {                                                                             \
        auto kern = bound_persistent_kernel<G_, LPL_>;                                         \
        int per_sm = 0;                                                                        \
        SLK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0)); \
        if (per_sm < 1) return set_err(ctx, SLK_ERR_CUDA, "bound kernel cannot be resident"); \
        int64_t grid = (int64_t)per_sm * ctx->num_sms;                                         \
        if (grid > blocks_needed) grid = blocks_needed;                                        \
        const float* a_ = A; const int64_t* rp_ = row_ptr; const int32_t* ci_ = col_idx;       \
        const float* w_ = w; int64_t n_ = N; int l_ = L; float lam_ = lambda;                  \
        float* z0_ = Z; float* z1_ = Z_prev; int mi_ = max_iters; float tol_ = tol;            \
        int kd_ = kdeg; DevState* st_ = st;                                                    \
        void* args[] = {&a_, &rp_, &ci_, &w_, &n_, &l_, &lam_, &z0_, &z1_, &mi_, &tol_, &kd_, &st_}; \
        e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(kThreads), \
                                        args, 0, ctx->stream);                                 \
    }
        SLK_DISPATCH_L(L, SLK_LAUNCH_PERSISTENT);
#undef SLK_LAUNCH_PERSISTENT
        if (e != cudaSuccess) return cuda_err(ctx, e, "bound_persistent_kernel");
    } else {
        SLK_COUNT_LAUNCH(ctx, max_iters + 1);
#define SLK_LAUNCH_STEPS(G_, LPL_)                                                             \
    for (int it = 0; it < max_iters; ++it)                                                     \
        bound_step_kernel<G_, LPL_><<<(unsigned)blocks_needed, kThreads, 0, ctx->stream>>>(    \
            A, row_ptr, col_idx, w, N, L, lambda, Z, Z_prev, it, tol, st);
        SLK_DISPATCH_L(L, SLK_LAUNCH_STEPS);
#undef SLK_LAUNCH_STEPS
        SLK_LAUNCH_CHECK(ctx, "bound_step_kernel");
        bound_finish_kernel<<<1, 1, 0, ctx->stream>>>(max_iters, st);
        SLK_LAUNCH_CHECK(ctx, "bound_finish_kernel");
    }
    const int64_t n = N * (int64_t)L;
    int64_t sgrid = (n + 255) / 256;
    if (sgrid > (int64_t)ctx->num_sms * 8) sgrid = (int64_t)ctx->num_sms * 8;
    SLK_COUNT_LAUNCH(ctx, 1);
    swap_if_odd_kernel<<<(unsigned)sgrid, 256, 0, ctx->stream>>>(Z, Z_prev, n, st);
    SLK_LAUNCH_CHECK(ctx, "swap_if_odd_kernel");
    return SLK_OK;
}

__global__ void degree_check_kernel(const int64_t* __restrict__ row_ptr, int64_t N,
                                    unsigned int* __restrict__ mixed) {
    const int64_t k = row_ptr[1] - row_ptr[0];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x)
        if (row_ptr[p] != k * p || row_ptr[p + 1] - row_ptr[p] != k) atomicOr(mixed, 1u);
}

slk_status uniform_degree(slk_ctx* ctx, const int64_t* row_ptr, int64_t N, DevState* st, int* kdeg) {
    *kdeg = 0;
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->deg_mixed, 0, sizeof(unsigned int), ctx->stream));
    int64_t g = (N + 255) / 256;
    if (g > (int64_t)ctx->num_sms * 8) g = (int64_t)ctx->num_sms * 8;
    SLK_COUNT_LAUNCH(ctx, 1);
    degree_check_kernel<<<(unsigned)g, 256, 0, ctx->stream>>>(row_ptr, N, &st->deg_mixed);
    SLK_LAUNCH_CHECK(ctx, "degree_check_kernel");
    int64_t rp[2] = {0, 0};
    unsigned int mixed = 1;
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(rp, row_ptr, sizeof(rp), cudaMemcpyDeviceToHost, ctx->stream));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(&mixed, &st->deg_mixed, sizeof(mixed), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    SLK_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t k = rp[1] - rp[0];
    if (!mixed && k >= 1 && k <= SLK_MAX_K) *kdeg = (int)k;
    return SLK_OK;
}

slk_status barrier_probe_launch(slk_ctx* ctx, DevState* st, unsigned long long timeout_ns) {
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(st, 0, offsetof(DevState, iters_done), ctx->stream));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->delta_bits[0], 0, sizeof(st->delta_bits), ctx->stream));
    SLK_COUNT_LAUNCH(ctx, 1);
    // one block waits for a second one that is never launched
    barrier_probe_kernel<<<1, 32, 0, ctx->stream>>>(st, 2u, timeout_ns);
    SLK_LAUNCH_CHECK(ctx, "barrier_probe_kernel");
    return SLK_OK;
}

slk_status mode_launch(slk_ctx* ctx, const float* A, const float* Z_prev,
                       const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                       int64_t N, int L, float lambda, int32_t* modes, int32_t* labels,
                       float* mode_key, bool use_iters_flag, DevState* st, const int32_t* orig,
                       const int32_t* inv) {
    PhaseScope ps(ctx, SLK_PHASE_MODE);
    SLK_COUNT_LAUNCH(ctx, 2);
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(&st->mode_best[0], 0, sizeof(unsigned long long) * L,
                                      ctx->stream));
    const Shape sh = shape_for(L);
    const int rows_per_block = (kThreads / 32) * (32 / sh.G);
    int64_t grid = (N + rows_per_block - 1) / rows_per_block;
    if (grid > (int64_t)ctx->num_sms * 8) grid = (int64_t)ctx->num_sms * 8;
#define SLK_LAUNCH_MODE(G_, LPL_)                                                        \
    mode_rows_kernel<G_, LPL_><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(            \
        A, Z_prev, row_ptr, col_idx, w, N, L, lambda, use_iters_flag ? 1 : 0, labels, orig, st);
    SLK_DISPATCH_L(L, SLK_LAUNCH_MODE);
#undef SLK_LAUNCH_MODE
    SLK_LAUNCH_CHECK(ctx, "mode_rows_kernel");
    mode_finish_kernel<<<1, 256, 0, ctx->stream>>>(L, modes, mode_key, inv, st);
    SLK_LAUNCH_CHECK(ctx, "mode_finish_kernel");
    return SLK_OK;
}

slk_status logz_launch(slk_ctx* ctx, const float* A, const float* Z_prev,
                       const int64_t* row_ptr, const int32_t* col_idx, const float* w,
                       int64_t N, int L, float lambda, int32_t* labels, float* LZ,
                       bool use_iters_flag, const DevState* st) {
    SLK_COUNT_LAUNCH(ctx, 1);
    const Shape sh = shape_for(L);
    const int rows_per_block = (kThreads / 32) * (32 / sh.G);
    int64_t grid = (N + rows_per_block - 1) / rows_per_block;
    if (grid > (int64_t)ctx->num_sms * 8) grid = (int64_t)ctx->num_sms * 8;
#define SLK_LAUNCH_LOGZ(G_, LPL_)                                                        \
    logz_rows_kernel<G_, LPL_><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(            \
        A, Z_prev, row_ptr, col_idx, w, N, L, lambda, use_iters_flag ? 1 : 0, labels, LZ, st);
    SLK_DISPATCH_L(L, SLK_LAUNCH_LOGZ);
#undef SLK_LAUNCH_LOGZ
    SLK_LAUNCH_CHECK(ctx, "logz_rows_kernel");
    return SLK_OK;
}

// ------------------------------------------------- allocation-free variant
//
// Scratch of slk_bound_iterate_noalloc: a 4 KiB status block followed by the
// ping-pong iterate.  Host code must not pass this symbol to a kernel (on
// the host it names a stand-in, not device memory); its device address is
// looked up once per device with cudaGetSymbolAddress.

static __device__ __align__(256) unsigned char g_noalloc_scratch[SLK_NOALLOC_SCRATCH_BYTES];
static_assert(sizeof(DevState) <= 4096, "status block must fit the reserved 4 KiB");

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx_id[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (0 if unknown), read
// through the driver entry points the runtime hands out, so the library does
// not link the driver library itself.  A device reset makes a new context
// with a new id, and the static array's address is looked up again.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}
}  // namespace

extern "C" slk_status slk_bound_iterate_noalloc(void* stream, const float* A, const int64_t* row_ptr,
                                                const int32_t* col_idx, const float* w, int64_t N,
                                                int32_t L, float lambda, float* Z, int32_t max_iters,
                                                float tol, int32_t* iters_done, float* last_delta) {
    if (!A || !row_ptr || !col_idx || !Z) return SLK_ERR_INVALID_ARG;
    if (N < 1 || N >= (int64_t)0x7fffffff || L < 1 || L > SLK_MAX_L || max_iters < 0)
        return SLK_ERR_INVALID_ARG;
    if (N * (int64_t)L > (int64_t)SLK_NOALLOC_MAX_ELEMS) return SLK_ERR_SCRATCH_LIMIT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SLK_ERR_NO_DEVICE;
    }
    void* base = nullptr;
    {
        // set-up once per device and context: the array's device address
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        const unsigned long long cid = current_context_id();   // 0: no context current yet
        if (!g_noalloc_addr[dev] || cid == 0 || cid != g_noalloc_ctx_id[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                g_noalloc_addr[dev] = nullptr;
                return SLK_ERR_CUDA;
            }
            g_noalloc_addr[dev] = p;
            // the lookup made the device's context current if none was
            g_noalloc_ctx_id[dev] = current_context_id();
        }
        base = g_noalloc_addr[dev];
    }
    DevState* st = static_cast<DevState*>(base);
    float* Zs = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + 4096);

    // the status words this call relies on start at zero; iters_done = -1
    if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess ||
        cudaMemsetAsync(&st->iters_done, 0xff, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return SLK_ERR_CUDA;
    }
    int num_sms = 0, coop = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
        cudaGetLastError();
        return SLK_ERR_CUDA;
    }
    cudaError_t e = cudaSuccess;
    if (max_iters == 0) {
        e = cudaMemsetAsync(&st->iters_done, 0, sizeof(int), s);
    } else {
        const Shape sh = shape_for(L);
        const int rows_per_block = (kThreads / 32) * (32 / sh.G);
        const int64_t blocks_needed = (N + rows_per_block - 1) / rows_per_block;
#define SLK_NOALLOC_LAUNCH(G_, LPL_)                                                           \
    {                                                                                          \
        auto kern = bound_persistent_kernel<G_, LPL_>;                                         \
        int per_sm = 0;                                                                        \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);         \
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;                 \
        if (e == cudaSuccess) {                                                                \
            int64_t grid = (int64_t)per_sm * num_sms;                                          \
            if (grid > blocks_needed) grid = blocks_needed;                                    \
            const float* a_ = A; const int64_t* rp_ = row_ptr; const int32_t* ci_ = col_idx;   \
            const float* w_ = w; int64_t n_ = N; int l_ = L; float lam_ = lambda;              \
            float* z0_ = Z; float* z1_ = Zs; int mi_ = max_iters; float tol_ = tol;            \
            int kd_ = 0; DevState* st_ = st;                                                   \
            void* args[] = {&a_, &rp_, &ci_, &w_, &n_, &l_, &lam_, &z0_, &z1_, &mi_, &tol_, &kd_, &st_}; \
            e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid),           \
                                            dim3(kThreads), args, 0, s);                       \
        }                                                                                      \
    }
        SLK_DISPATCH_L(L, SLK_NOALLOC_LAUNCH);
#undef SLK_NOALLOC_LAUNCH
        if (e == cudaSuccess) {
            const int64_t n = N * (int64_t)L;
            int64_t sgrid = (n + 255) / 256;
            if (sgrid > (int64_t)num_sms * 8) sgrid = (int64_t)num_sms * 8;
            swap_if_odd_kernel<<<(unsigned)sgrid, 256, 0, s>>>(Z, Zs, n, st);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SLK_ERR_CUDA;
    }
    // read the status block (iters_done, delta, error) into a host copy of
    // the same type (pageable memory: the copy is synchronous for the host)
    DevState hs;
    e = cudaMemcpyAsync(&hs, st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SLK_ERR_CUDA;
    }
    if (hs.error & ERR_BARRIER_TIMEOUT) return SLK_ERR_TIMEOUT;
    if (iters_done) *iters_done = hs.iters_done;
    if (last_delta) *last_delta = hs.last_delta;
    return SLK_OK;
}
