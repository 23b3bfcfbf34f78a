// Continuous-batching server for SLK-BO requests (slk_server_*, include/slk.h).
//
// Requests wait in a FIFO queue until a slot is free and their device state
// (kNN graph, unary term A, scratch iterate, and -- while the graph is being
// built -- kNN scratch) fits in the server's memory arena.  An admitted
// request's graph and sigma are built on one of several auxiliary streams,
// overlapping whatever runs on the main stream.  Each slk_server_step then
// advances every request that has its graph, all in segment-indexed launches
// over the slots:
//   srv_unary_kernel    start of an outer iteration: a, z = softmax(a)
//   srv_bound_kernel    up to `quantum` z-updates (persistent, cooperative);
//                       each slot continues its own update count and delta
//                       ring, so its arithmetic is the same whatever else runs
//   srv_swap / srv_mode / srv_mode_finish / srv_energy / srv_outer_update
//                       for the slots whose inner loop ended in this step
// A slot whose modes stopped changing (or that hit max_outer) is done: its
// caller-owned Z, labels and modes hold the result, its memory and slot are
// released on the host.
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <vector>

#include "seg_common.cuh"

namespace {

enum : int { SLOT_IDLE = 0, SLOT_START = 1, SLOT_ITER = 2, SLOT_DONE = 3 };
// Auxiliary streams for graph builds (requests take them in turn).  Measured
// on a 2000-request stream: 1, 2 and 4 streams serve within 2 % of each other
// (the tile kernels of large graphs fill every SM, so builds do not overlap).
#ifndef SLK_SRV_AUX
#define SLK_SRV_AUX 4
#endif
constexpr int kSrvAux = SLK_SRV_AUX;

struct SlotDev {
    int* mode;          // SLOT_*
    int* it_base;       // z-updates done in the current inner loop
    int* fin;           // -1, or the update count the inner loop ended with
    unsigned* delta;    // [3 S] ring of max |dz| per update
    int* outer;
    int* inner_total;
    int* changed;
    double* energy;
    double* energy_out;
    float* sigma;
    unsigned long long* best;  // [S * SLK_BATCH_MAX_L]
};

// Exclusive prefix over slots of the tile counts of slots satisfying `pred`
// (same answer in every block), computed into shared memory pref[S + 1].
template <int THREADS, class Pred, class Tiles>
__device__ void slot_scan(int S, int* pref, int* wsum, Pred pred, Tiles tiles_of) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int per = (S + THREADS - 1) / THREADS;
    const int s0 = threadIdx.x * per;
    int local = 0;
    for (int s = s0; s < min(S, s0 + per); ++s) {
        const int c = pred(s) ? tiles_of(s) : 0;
        pref[s] = c;
        local += c;
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int v = lane < THREADS / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < THREADS / 32) wsum[lane] = v;
    }
    __syncthreads();
    int run = incl - local + (wid > 0 ? wsum[wid - 1] : 0);
    for (int s = s0; s < min(S, s0 + per); ++s) {
        const int c = pref[s];
        pref[s] = run;
        run += c;
    }
    if (threadIdx.x == THREADS - 1) pref[S] = run;
    __syncthreads();
}

__device__ __forceinline__ int find_slot(const int* pref, int S, int64_t wi) {
    int lo = 0, hi = S;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pref[mid] <= wi) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int rows_per_tile(const SegInfo& si) { return 32 / si.G; }
__device__ __forceinline__ int n_tiles(const SegInfo& si) {
    const int r = rows_per_tile(si);
    return (int)((si.N + r - 1) / r);
}

// ---- start of an outer iteration: a = k(x, m), z = softmax(a); slot -> ITER
__global__ void __launch_bounds__(256)
srv_unary_kernel(const SegInfo* __restrict__ seg, int S, SlotDev sd) {
    extern __shared__ int pref[];
    __shared__ int wsum[8];
    __shared__ float xs[32][33];
    __shared__ float ms[SLK_BATCH_MAX_L][33];
    __shared__ float at[32][SLK_BATCH_MAX_L + 1];
    __shared__ int mrow[SLK_BATCH_MAX_L];
    slot_scan<256>(S, pref, wsum, [&](int s) { return sd.mode[s] == SLOT_START; },
                   [&](int s) { return (int)((seg[s].N + 31) / 32); });
    const int total = pref[S];
    for (int64_t wi = blockIdx.x; wi < total; wi += gridDim.x) {
        const int s = find_slot(pref, S, wi);
        const SegInfo si = seg[s];
        const int tile = (int)(wi - pref[s]);
        const int64_t row0 = (int64_t)tile * 32;
        const int nrows = (int)((si.N - row0) < 32 ? (si.N - row0) : 32);
        const int t = threadIdx.x, pl = t & 31, lb = t >> 5;
        const int L = si.L, D = si.D;
        constexpr int LPT = SLK_BATCH_MAX_L / 8;
        __syncthreads();
        for (int l = t; l < L; l += 256) mrow[l] = si.modes[l];
        double acc[LPT];
#pragma unroll
        for (int j = 0; j < LPT; ++j) acc[j] = 0.0;
        __syncthreads();
        for (int d0 = 0; d0 < D; d0 += 32) {
            const int dc = min(32, D - d0);
            for (int i = t; i < 32 * 32; i += 256) {
                const int r = i >> 5, c = i & 31;
                xs[r][c] = (r < nrows && c < dc) ? si.X[(row0 + r) * D + d0 + c] : 0.f;
            }
            for (int i = t; i < L * 32; i += 256) {
                const int r = i >> 5, c = i & 31;
                ms[r][c] = (c < dc) ? si.X[(int64_t)mrow[r] * D + d0 + c] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < LPT; ++j) {
                const int l = lb + 8 * j;
                if (l < L) {
                    float part = 0.f;
                    for (int c = 0; c < dc; ++c) {
                        const float df = xs[pl][c] - ms[l][c];
                        part = fmaf(df, df, part);
                    }
                    acc[j] += (double)part;
                }
            }
            __syncthreads();
        }
        const float sg = *si.sigma;
        const float inv2s2 = 1.0f / (2.0f * sg * sg);
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int l = lb + 8 * j;
            if (l < L) {
                const float a = expf(-(float)acc[j] * inv2s2);
                at[pl][l] = a;
                if (pl < nrows) si.A[(row0 + pl) * L + l] = a;
            }
        }
        __syncthreads();
        if (t < nrows) {
            float m = at[t][0];
            for (int l = 1; l < L; ++l) m = fmaxf(m, at[t][l]);
            float sm = 0.f;
            for (int l = 0; l < L; ++l) sm += expf(at[t][l] - m);
            float* zr = si.Z + (row0 + t) * L;
            for (int l = 0; l < L; ++l) zr[l] = expf(at[t][l] - m) / sm;
        }
    }
}

// The slots that started an outer iteration are now iterating.
__global__ void srv_start_inner_kernel(int S, SlotDev sd, SegState* ss) {
    __shared__ int n_iter;
    if (threadIdx.x == 0) n_iter = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        if (sd.mode[s] == SLOT_START) {
            sd.mode[s] = SLOT_ITER;
            sd.it_base[s] = 0;
            sd.fin[s] = -1;
            sd.delta[3 * s] = sd.delta[3 * s + 1] = sd.delta[3 * s + 2] = 0u;
            sd.energy[s] = 0.0;
        }
        if (sd.mode[s] == SLOT_ITER && sd.fin[s] < 0) atomicAdd(&n_iter, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ss->active_inner = n_iter;
        ss->arrive = 0;
    }
}

// ---- up to `quantum` z-updates of every iterating slot
// Resident CTAs per SM and neighbour window of the z-update kernel, measured
// on eight requests of 120633 x 18 (k = 10, 300 updates each) served
// together: 1 CTA / window 8 (155 registers) 470 ms, 2 / 8 307 ms,
// 3 / 8 301 ms (spills), 3 / 4 258 ms, 3 / 2 262 ms, 4 / 2 283 ms.
// Lanes per row of the segment-indexed kernels (0: as the plain z-update
// kernels, so that a request's soft-max sums run in the plain kernels' order;
// 1: the fewest that hold L at kLPL labels per lane, at least 4).  Measured
// on eight requests of 120633 x 18 served together: 262 ms with 0, 185 ms
// with 1 (the plain loop: 178 ms).  On the 2000-request stream 1 served
// 92.4 requests/s against 91.2 for the plain loop, but only 163 of the
// first 200 requests kept the plain loop's labels and modes (190 with 0):
// the other summation order moves trajectories that pass near a tie or the
// tolerance
#ifndef SLK_SRV_G_RULE
#define SLK_SRV_G_RULE 0
#endif
#ifndef SLK_SRV_BOUND_MINB
#define SLK_SRV_BOUND_MINB 3
#endif
#ifndef SLK_SRV_BOUND_W
#define SLK_SRV_BOUND_W 4
#endif
template <int THREADS, int W>
__global__ void __launch_bounds__(THREADS, SLK_SRV_BOUND_MINB)
srv_bound_kernel(const SegInfo* __restrict__ seg, int S, SlotDev sd, int quantum, int max_inner,
                 float tol, SegState* ss) {
    extern __shared__ int pref[];
    __shared__ int wsum[THREADS / 32];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (THREADS / 32);
    const int64_t gwarp = (int64_t)blockIdx.x * (THREADS / 32) + (threadIdx.x >> 5);
    for (int it = 0; it < quantum; ++it) {
        // live slots of this update; block 0 records the ones whose inner loop
        // ends here (converged, or max_inner updates done)
        auto live = [&](int s) -> bool {
            if (sd.mode[s] != SLOT_ITER) return false;
            const int u = sd.it_base[s] + it;
            const int f = *(volatile int*)&sd.fin[s];
            if (f >= 0 && f < u) return false;
            bool stop = u >= max_inner;
            if (!stop && u > 0) stop = __uint_as_float(ld_acq(&sd.delta[3 * s + (u - 1) % 3])) <= tol;
            if (stop) {
                if (blockIdx.x == 0 && atomicCAS(&sd.fin[s], -1, u) == -1) atomicSub(&ss->active_inner, 1);
                return false;
            }
            if (blockIdx.x == 0) sd.delta[3 * s + (u + 1) % 3] = 0u;
            return true;
        };
        slot_scan<THREADS>(S, pref, wsum, live, [&](int s) { return n_tiles(seg[s]); });
        const int total = pref[S];
        // each lane's max |dz| over this warp's tiles of one slot, published
        // with one atomic when the warp moves to another slot (a warp's tiles
        // are consecutive in slot order)
        int cur = -1, cur_u = 0;
        float dacc = 0.f;
        auto flush = [&]() {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dacc = fmaxf(dacc, __shfl_xor_sync(0xffffffffu, dacc, o));
            if (lane == 0 && cur >= 0 && dacc > 0.f)
                atomicMax(&sd.delta[3 * cur + cur_u % 3], __float_as_uint(dacc));
            dacc = 0.f;
        };
        SegInfo si;
        int cur_end = 0;   // the first tile past the current slot's
        for (int64_t wi = gwarp; wi < total; wi += nwarps) {
            if (cur < 0 || wi >= cur_end) {
                flush();
                cur = find_slot(pref, S, wi);
                cur_end = pref[cur + 1];
                load_seg(seg, cur, si);
                cur_u = sd.it_base[cur] + it;
            }
            const int s = cur, u = cur_u;
            const int rpt = rows_per_tile(si);
            const int64_t row0 = (wi - pref[s]) * (int64_t)rpt;
            const int nrows = (int)((si.N - row0) < rpt ? (si.N - row0) : (int64_t)rpt);
            const int G = si.G, grp = lane / G, gl = lane % G;
            const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
            const float* Zin = (u & 1) ? si.Zs : si.Z;
            float* Zout = (u & 1) ? si.Z : si.Zs;
            float d = 0.f;
            if (grp < nrows) {
                const int64_t p = row0 + grp;
                const int64_t off = p * (int64_t)si.L;
                // the row's unary term and previous iterate, loaded before the
                // neighbour gathers so that their latency overlaps them
                float av[kLPL], zo[kLPL];
#pragma unroll
                for (int j = 0; j < kLPL; ++j) {
                    const int l = gl + G * j;
                    av[j] = (l < si.L) ? __ldg(si.A + off + l) : 0.f;
                    zo[j] = (l < si.L) ? __ldcg(Zin + off + l) : 0.f;
                }
                float sv[kLPL];
                seg_pair<W>(si, p, gl, gm, Zin, true, sv);
#pragma unroll
                for (int j = 0; j < kLPL; ++j)
                    sv[j] = (gl + G * j < si.L) ? fmaf(si.lambda, sv[j], av[j]) : -INFINITY;
                float m = sv[0];
#pragma unroll
                for (int j = 1; j < kLPL; ++j) m = fmaxf(m, sv[j]);
                m = gmax(m, gm, G);
                float e[kLPL], sum = 0.f;
#pragma unroll
                for (int j = 0; j < kLPL; ++j) {
                    e[j] = (gl + G * j < si.L) ? expf(sv[j] - m) : 0.f;
                    sum += e[j];
                }
                sum = gsum(sum, gm, G);
#pragma unroll
                for (int j = 0; j < kLPL; ++j) {
                    const int l = gl + G * j;
                    if (l < si.L) {
                        const float z = e[j] / sum;
                        d = fmaxf(d, fabsf(z - zo[j]));
                        __stcg(Zout + off + l, z);
                    }
                }
            }
            dacc = fmaxf(dacc, d);
        }
        flush();
        const int r = seg_step(ss, gridDim.x);
        if (r < 0) return;
        if (r == 1) break;
    }
}

// Iterating slots still running carry their count into the next step.
__global__ void srv_post_bound_kernel(int S, int quantum, SlotDev sd) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x)
        if (sd.mode[s] == SLOT_ITER && sd.fin[s] < 0) sd.it_base[s] += quantum;
}

__device__ __forceinline__ bool ending(const SlotDev& sd, int s) {
    return sd.mode[s] == SLOT_ITER && sd.fin[s] >= 0;
}

// The last iterate of a slot whose inner loop ended sits in Zs after an odd count.
__global__ void srv_swap_kernel(const SegInfo* __restrict__ seg, int S, SlotDev sd) {
    const int s = blockIdx.y;
    if (s >= S || !ending(sd, s) || (sd.fin[s] & 1) == 0) return;
    const SegInfo si = seg[s];
    const int64_t n = si.N * (int64_t)si.L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float a = si.Z[i];
        si.Z[i] = si.Zs[i];
        si.Zs[i] = a;
    }
}

template <int W>
__global__ void __launch_bounds__(256)
srv_mode_kernel(const SegInfo* __restrict__ seg, int S, SlotDev sd) {
    extern __shared__ int pref[];
    __shared__ int wsum[8];
    const int lane = threadIdx.x & 31;
    slot_scan<256>(S, pref, wsum, [&](int s) { return ending(sd, s); },
                   [&](int s) { return n_tiles(seg[s]); });
    const int total = pref[S];
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    // each lane's best keys over this warp's tiles of one slot (its labels
    // gl + G j), merged across groups and published when the warp moves to
    // another slot
    int cur = -1, cur_G = 32, cur_L = 0;
    unsigned long long best[kLPL];
#pragma unroll
    for (int j = 0; j < kLPL; ++j) best[j] = 0ull;
    auto flush = [&]() {
#pragma unroll
        for (int j = 0; j < kLPL; ++j) {
            for (int o = cur_G; o < 32; o <<= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best[j], o);
                if (ob > best[j]) best[j] = ob;
            }
            const int l = lane + cur_G * j;
            if (cur >= 0 && lane < cur_G && l < cur_L && best[j])
                atomicMax(&sd.best[(int64_t)cur * SLK_BATCH_MAX_L + l], best[j]);
            best[j] = 0ull;
        }
    };
    for (int64_t wi = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); wi < total; wi += nwarps) {
        const int s = find_slot(pref, S, wi);
        SegInfo si;
        load_seg(seg, s, si);
        if (s != cur) {
            flush();
            cur = s;
            cur_G = si.G;
            cur_L = si.L;
        }
        const int rpt = rows_per_tile(si);
        const int64_t row0 = (wi - pref[s]) * (int64_t)rpt;
        const int nrows = (int)((si.N - row0) < rpt ? (si.N - row0) : (int64_t)rpt);
        const int G = si.G, grp = lane / G, gl = lane % G;
        const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
        const bool live = grp < nrows;
        const int64_t p = row0 + (live ? grp : 0);
        if (live) {
            float sv[kLPL];
            seg_logits<W>(si, p, gl, gm, si.Zs, sd.fin[s] > 0, sv);
            float m = sv[0];
            int jl = gl;
#pragma unroll
            for (int j = 1; j < kLPL; ++j)
                if (sv[j] > m) { m = sv[j]; jl = gl + G * j; }
            for (int o = G >> 1; o > 0; o >>= 1) {
                const float om = __shfl_xor_sync(gm, m, o, G);
                const int ol = __shfl_xor_sync(gm, jl, o, G);
                if (om > m || (om == m && ol < jl)) { m = om; jl = ol; }
            }
            float r = 0.f;
#pragma unroll
            for (int j = 0; j < kLPL; ++j) {
                const int l = gl + G * j;
                if (l < si.L && l != jl) r += expf(sv[j] - m);
            }
            r = gsum(r, gm, G);
            const float lse1 = log1pf(r);
            if (gl == 0) si.labels[p] = jl;
#pragma unroll
            for (int j = 0; j < kLPL; ++j) {
                const int l = gl + G * j;
                if (l < si.L) {
                    const unsigned long long key =
                        ((unsigned long long)float_to_ordered((sv[j] - m) - lse1) << 32) |
                        (unsigned long long)(0xffffffffu - (unsigned)p);
                    if (key > best[j]) best[j] = key;
                }
            }
        }
    }
    flush();
}

__global__ void srv_mode_finish_kernel(const SegInfo* __restrict__ seg, int S, SlotDev sd) {
    const int s = blockIdx.x;
    if (s >= S || !ending(sd, s)) return;
    const SegInfo si = seg[s];
    __shared__ int ch;
    if (threadIdx.x == 0) ch = 0;
    __syncthreads();
    for (int l = threadIdx.x; l < si.L; l += blockDim.x) {
        unsigned long long* b = &sd.best[(int64_t)s * SLK_BATCH_MAX_L + l];
        const int q = (int)(0xffffffffu - (unsigned)(*b & 0xffffffffull));
        if (q != si.modes[l]) ch = 1;
        si.modes[l] = q;
        *b = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) sd.changed[s] = ch;
}

__global__ void __launch_bounds__(256)
srv_energy_kernel(const SegInfo* __restrict__ seg, int S, SlotDev sd) {
    extern __shared__ int pref[];
    __shared__ int wsum[8];
    const int lane = threadIdx.x & 31;
    slot_scan<256>(S, pref, wsum, [&](int s) { return ending(sd, s); },
                   [&](int s) { return n_tiles(seg[s]); });
    const int total = pref[S];
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    // each lane's float64 sum over this warp's tiles of one slot, added to the
    // slot's energy when the warp moves to another slot
    int cur = -1;
    double acc = 0.0;
    auto flush = [&]() {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && cur >= 0) atomicAdd(&sd.energy[cur], acc);
        acc = 0.0;
    };
    for (int64_t wi = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); wi < total; wi += nwarps) {
        const int s = find_slot(pref, S, wi);
        SegInfo si;
        load_seg(seg, s, si);
        if (s != cur) {
            flush();
            cur = s;
        }
        const int rpt = rows_per_tile(si);
        const int64_t row0 = (wi - pref[s]) * (int64_t)rpt;
        const int nrows = (int)((si.N - row0) < rpt ? (si.N - row0) : (int64_t)rpt);
        const double sg = (double)*si.sigma;
        const double inv2s2 = 1.0 / (2.0 * sg * sg);
        double my_d2 = 0.0, my_cut = 0.0;
        bool mine = false;
        int slot = 0;
        for (int r = 0; r < nrows; ++r) {
            const int64_t p = row0 + r;
            const int lp = si.labels[p];
            const float* xp = si.X + p * si.D;
            const float* xm = si.X + (int64_t)si.modes[lp] * si.D;
            const double d2 = warp_sq_dist(xp, xm, nullptr, si.D, lane);
            const int64_t e0 = p * si.kdeg, e1 = e0 + si.kdeg;
            float ch = 0.f, cl = 0.f;   // cut weight as a float pair
            for (int64_t e = e0 + lane; e < e1; e += 32)
                if (si.labels[si.col[e]] != lp) fpair_add(ch, cl, si.w ? si.w[e] : 1.f, 0.f);
            for (int o = 16; o > 0; o >>= 1)
                fpair_add(ch, cl, __shfl_xor_sync(0xffffffffu, ch, o), __shfl_xor_sync(0xffffffffu, cl, o));
            // lane `slot` keeps this row; the float64 kernel values of 32 rows
            // are then one warp-wide sequence
            if (lane == slot) {
                my_d2 = d2;
                my_cut = (double)ch + (double)cl;
                mine = true;
            }
            if (++slot == 32) {
                if (mine) acc += -exp(-my_d2 * inv2s2) + 0.5 * (double)si.lambda * 2.0 * my_cut;
                mine = false;
                slot = 0;
            }
        }
        if (mine) acc += -exp(-my_d2 * inv2s2) + 0.5 * (double)si.lambda * 2.0 * my_cut;
    }
    flush();
}

// End of an outer iteration: count it, then either the next outer iteration
// (modes changed, below max_outer) or done.
__global__ void srv_outer_update_kernel(int S, int max_outer, SlotDev sd) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        if (!ending(sd, s)) continue;
        sd.outer[s] += 1;
        sd.inner_total[s] += sd.fin[s];
        sd.energy_out[s] = sd.energy[s];
        sd.mode[s] = (sd.changed[s] && sd.outer[s] < max_outer) ? SLOT_START : SLOT_DONE;
    }
}

// ------------------------------------------------------------------ host side

struct Block {
    size_t off, size;
};

struct Request {
    slk_instance spec;
    int state = 0;  // 0 queued, 1 building graph, 2 iterating, 3 done
    int slot = -1;
    int aux = 0;
    Block mem{0, 0}, scratch{0, 0};
    cudaEvent_t ev = nullptr;
    slk_stats stats{};
};

}  // namespace

struct slk_server {
    slk_ctx* ctx = nullptr;
    slk_server_config cfg{};
    slk_params p{};
    char* arena = nullptr;
    size_t arena_bytes = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> size
    int S = 0;
    SegInfo* d_seg = nullptr;
    SegState* d_ss = nullptr;
    SlotDev sd{};
    void* d_base = nullptr;
    int* h_mode = nullptr;   // pinned status copies
    int* h_outer = nullptr;
    int* h_inner = nullptr;
    double* h_energy = nullptr;
    float* h_sigma = nullptr;
    SegState* h_ss = nullptr;
    DevState* aux_st = nullptr;
    cudaStream_t aux[kSrvAux] = {};
    std::vector<int64_t> slot_req;
    std::deque<int64_t> queue;
    std::map<int64_t, Request> reqs;
    int64_t next_id = 1;
    int next_aux = 0;
};

namespace {

bool arena_alloc(slk_server* sv, size_t bytes, Block& out) {
    bytes = align_up(std::max<size_t>(bytes, 256), 256);
    for (auto it = sv->free_blocks.begin(); it != sv->free_blocks.end(); ++it) {
        if (it->second >= bytes) {
            out = {it->first, bytes};
            const size_t rest = it->second - bytes, roff = it->first + bytes;
            sv->free_blocks.erase(it);
            if (rest) sv->free_blocks[roff] = rest;
            return true;
        }
    }
    return false;
}

void arena_free(slk_server* sv, Block b) {
    if (!b.size) return;
    auto it = sv->free_blocks.emplace(b.off, b.size).first;
    auto nx = std::next(it);
    if (nx != sv->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        sv->free_blocks.erase(nx);
    }
    if (it != sv->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            sv->free_blocks.erase(it);
        }
    }
}

size_t request_bytes(const slk_server* sv, const slk_instance& q) {
    size_t b = align_up(sizeof(int64_t) * (q.N + 1), 256) + 2 * align_up(sizeof(float) * q.N * q.k, 256) +
               align_up(sizeof(int32_t) * q.N * q.k, 256) + 2 * align_up(sizeof(float) * q.N * q.L, 256);
    if (sv->p.affinity == SLK_AFFINITY_HEAT) b += align_up(sizeof(float) * q.N * q.k, 256);
    return b + 1024;
}

template <class T>
T* carve(char* base, size_t& off, size_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * count;
    return p;
}

}  // namespace

extern "C" slk_status slk_server_create(slk_ctx* ctx, const slk_server_config* cfg,
                                        const slk_params* params, slk_server** out) {
    if (!ctx || !cfg || !out) return SLK_ERR_INVALID_ARG;
    *out = nullptr;
    ctx->err.clear();
    if (cfg->max_slots < 1 || cfg->max_slots > SLK_BATCH_MAX_COUNT || cfg->memory_bytes < (1 << 20) ||
        cfg->quantum < 1)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "bad server configuration");
    if (params && params->symmetrize != 0)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "the server runs on the directed kNN graph only");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    slk_server* sv = new slk_server();
    sv->ctx = ctx;
    sv->cfg = *cfg;
    if (params) sv->p = *params; else slk_default_params(&sv->p);
    sv->S = cfg->max_slots;
    const int S = sv->S;
    auto fail = [&](cudaError_t e, const char* what) {
        slk_status st = cuda_err(ctx, e, what);
        slk_server_destroy(sv);
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    };
    cudaError_t e = cudaMalloc(&sv->arena, (size_t)cfg->memory_bytes);
    if (e != cudaSuccess) return fail(e, "server arena");
    sv->arena_bytes = (size_t)cfg->memory_bytes;
    sv->free_blocks[0] = sv->arena_bytes;
    // slot arrays (one allocation)
    size_t bytes = 0;
    bytes += align_up(sizeof(SegInfo) * S, 256) + align_up(sizeof(SegState), 256);
    bytes += 7 * align_up(sizeof(int) * S, 256) + align_up(sizeof(unsigned) * 3 * S, 256);
    bytes += 2 * align_up(sizeof(double) * S, 256) + align_up(sizeof(float) * S, 256);
    bytes += align_up(sizeof(unsigned long long) * S * SLK_BATCH_MAX_L, 256);
    bytes += kSrvAux * align_up(sizeof(DevState), 256) + 4096;
    e = cudaMalloc(&sv->d_base, bytes);
    if (e != cudaSuccess) return fail(e, "server slot tables");
    e = cudaMemset(sv->d_base, 0, bytes);
    if (e != cudaSuccess) return fail(e, "server slot tables");
    size_t off = 0;
    char* base = static_cast<char*>(sv->d_base);
    sv->d_seg = carve<SegInfo>(base, off, S);
    sv->d_ss = carve<SegState>(base, off, 1);
    sv->sd.mode = carve<int>(base, off, S);
    sv->sd.it_base = carve<int>(base, off, S);
    sv->sd.fin = carve<int>(base, off, S);
    sv->sd.outer = carve<int>(base, off, S);
    sv->sd.inner_total = carve<int>(base, off, S);
    sv->sd.changed = carve<int>(base, off, S);
    sv->sd.delta = carve<unsigned>(base, off, 3 * S);
    sv->sd.energy = carve<double>(base, off, S);
    sv->sd.energy_out = carve<double>(base, off, S);
    sv->sd.sigma = carve<float>(base, off, S);
    sv->sd.best = carve<unsigned long long>(base, off, (size_t)S * SLK_BATCH_MAX_L);
    sv->aux_st = carve<DevState>(base, off, kSrvAux);
    void* hp = nullptr;
    e = cudaMallocHost(&hp, sizeof(int) * 3 * S + sizeof(double) * S + sizeof(float) * S + sizeof(SegState) + 256);
    if (e != cudaSuccess) return fail(e, "server status buffer");
    sv->h_mode = static_cast<int*>(hp);
    sv->h_outer = sv->h_mode + S;
    sv->h_inner = sv->h_outer + S;
    sv->h_energy = reinterpret_cast<double*>(align_up(reinterpret_cast<uintptr_t>(sv->h_inner + S), 8));
    sv->h_sigma = reinterpret_cast<float*>(sv->h_energy + S);
    sv->h_ss = reinterpret_cast<SegState*>(align_up(reinterpret_cast<uintptr_t>(sv->h_sigma + S), 16));
    for (int i = 0; i < kSrvAux; ++i) {
        e = cudaStreamCreateWithFlags(&sv->aux[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(e, "server streams");
    }
    sv->slot_req.assign(S, -1);
    if (prev >= 0) cudaSetDevice(prev);
    *out = sv;
    return SLK_OK;
}

extern "C" slk_status slk_server_destroy(slk_server* sv) {
    if (!sv) return SLK_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : sv->reqs)
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    for (int i = 0; i < kSrvAux; ++i)
        if (sv->aux[i]) cudaStreamDestroy(sv->aux[i]);
    if (sv->h_mode) cudaFreeHost(sv->h_mode);
    if (sv->d_base) cudaFree(sv->d_base);
    if (sv->arena) cudaFree(sv->arena);
    delete sv;
    if (prev >= 0) cudaSetDevice(prev);
    return SLK_OK;
}

extern "C" slk_status slk_server_submit(slk_server* sv, const slk_instance* q, int64_t* ticket) {
    if (!sv || !q || !ticket) return SLK_ERR_INVALID_ARG;
    slk_ctx* ctx = sv->ctx;
    ctx->err.clear();
    if (!q->X || !q->init_modes || !q->Z || !q->labels || !q->modes)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "request: required pointer is NULL");
    if (q->N < 2 || q->N >= (int64_t)0x7fffffff || q->D < 1 || q->L < 1 || q->L > SLK_BATCH_MAX_L ||
        q->L > q->N || q->k < 1 || q->k > SLK_MAX_K || q->k > q->N - 1)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "request: bad sizes");
    const size_t need = request_bytes(sv, *q) + knn_ws_bytes(ctx, q->N, q->D, q->k, sv->p.knn_precision);
    if (need > sv->arena_bytes)
        return set_err(ctx, SLK_ERR_OOM, "request needs %zu bytes, the server arena has %zu", need,
                       sv->arena_bytes);
    const int64_t id = sv->next_id++;
    Request r;
    r.spec = *q;
    sv->reqs[id] = r;
    sv->queue.push_back(id);
    *ticket = id;
    return SLK_OK;
}

extern "C" slk_status slk_server_request_bytes(slk_server* sv, const slk_instance* q, int64_t* bytes) {
    if (!sv || !q || !bytes) return SLK_ERR_INVALID_ARG;
    *bytes = (int64_t)(align_up(request_bytes(sv, *q), 256) +
                       align_up(knn_ws_bytes(sv->ctx, q->N, q->D, q->k, sv->p.knn_precision), 256));
    return SLK_OK;
}

extern "C" slk_status slk_server_poll(slk_server* sv, int64_t ticket, int32_t* state, slk_stats* stats) {
    if (!sv || !state) return SLK_ERR_INVALID_ARG;
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return set_err(sv->ctx, SLK_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
    *state = it->second.state;
    if (stats && it->second.state == 3) *stats = it->second.stats;
    if (it->second.state == 3) sv->reqs.erase(it);   // a finished ticket is reported once
    return SLK_OK;
}

namespace {

slk_status admit(slk_server* sv, int64_t id) {
    slk_ctx* ctx = sv->ctx;
    Request& r = sv->reqs[id];
    const slk_instance& q = r.spec;
    int slot = -1;
    for (int s = 0; s < sv->S; ++s)
        if (sv->slot_req[s] < 0) { slot = s; break; }
    if (slot < 0) return SLK_ERR_OOM;
    Block mem, scr;
    if (!arena_alloc(sv, request_bytes(sv, q), mem)) return SLK_ERR_OOM;
    if (!arena_alloc(sv, knn_ws_bytes(ctx, q.N, q.D, q.k, sv->p.knn_precision), scr)) {
        arena_free(sv, mem);
        return SLK_ERR_OOM;
    }
    r.slot = slot;
    r.mem = mem;
    r.scratch = scr;
    r.aux = sv->next_aux;
    sv->next_aux = (sv->next_aux + 1) % kSrvAux;
    sv->slot_req[slot] = id;
    // carve the request's buffers and describe the slot
    char* base = sv->arena + mem.off;
    size_t off = 0;
    SegInfo si{};
    int64_t* row_ptr = carve<int64_t>(base, off, q.N + 1);
    int32_t* col = carve<int32_t>(base, off, q.N * q.k);
    float* dist2 = carve<float>(base, off, q.N * q.k);
    float* wts = (sv->p.affinity == SLK_AFFINITY_HEAT) ? carve<float>(base, off, q.N * q.k) : nullptr;
    si.A = carve<float>(base, off, q.N * q.L);
    si.Zs = carve<float>(base, off, q.N * q.L);
    si.X = q.X;
    si.Z = q.Z;
    si.labels = q.labels;
    si.modes = q.modes;
    si.row_ptr = row_ptr;
    si.col = col;
    si.w = wts;
    si.sigma = sv->sd.sigma + slot;
    si.N = q.N;
    si.L = q.L;
    si.D = q.D;
#if SLK_SRV_G_RULE == 1
    // lanes per row: the fewest (a power of two, at least 4) that hold the
    // row's labels at kLPL per lane -- more rows per warp for the gathers in
    // flight
    int g = 4;
    while (g * kLPL < q.L) g <<= 1;
    si.G = g;
#else
    // lanes per row: every label of L <= 8 on its own lane; above, two
    // labels per lane up to L = 32 (8 or 16 lanes), then 32 lanes with up to
    // kLPL labels each -- more rows per warp for the gathers in flight
    int g = 1;
    while (g < q.L && g < 8) g <<= 1;
    si.G = q.L <= 8 ? g : q.L <= 16 ? 8 : q.L <= 32 ? 16 : 32;
#endif
    si.moff = slot * SLK_BATCH_MAX_L;
    si.lambda = q.lambda;
    si.kdeg = q.k;
    // graph, sigma and weights on the request's auxiliary stream
    cudaStream_t main_s = ctx->stream;
    ctx->stream = sv->aux[r.aux];
    DevState* st = sv->aux_st + r.aux;
    slk_status rs = knn_graph_launch(ctx, q.X, q.N, q.D, q.k, sv->p.knn_precision, row_ptr, col, dist2,
                                     sv->arena + scr.off, st);
    if (rs == SLK_OK)
        rs = (q.sigma > 0.f) ? set_sigma_launch(ctx, q.sigma, st)
                             : sigma_launch(ctx, dist2, q.N * (int64_t)q.k, sv->p.sigma_rule, st);
    cudaError_t ce = cudaSuccess;
    if (rs == SLK_OK)
        ce = cudaMemcpyAsync(sv->sd.sigma + slot, &st->sigma, sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
    if (rs == SLK_OK && ce == cudaSuccess && wts)
        rs = weights_launch(ctx, dist2, q.N * (int64_t)q.k, SLK_AFFINITY_HEAT, sv->sd.sigma + slot, wts);
    if (rs == SLK_OK && ce == cudaSuccess)
        ce = cudaMemcpyAsync(q.modes, q.init_modes, sizeof(int32_t) * q.L, cudaMemcpyDeviceToDevice, ctx->stream);
    if (rs == SLK_OK && ce == cudaSuccess)
        ce = cudaMemcpyAsync(sv->d_seg + slot, &si, sizeof(SegInfo), cudaMemcpyHostToDevice, ctx->stream);
    if (rs == SLK_OK && ce == cudaSuccess && !r.ev) ce = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming);
    if (rs == SLK_OK && ce == cudaSuccess) ce = cudaEventRecord(r.ev, ctx->stream);
    ctx->stream = main_s;
    if (ce != cudaSuccess) return cuda_err(ctx, ce, "request admission");
    if (rs != SLK_OK) return rs;
    r.state = 1;
    return SLK_OK;
}

}  // namespace

extern "C" slk_status slk_server_step(slk_server* sv, int32_t* n_running, int32_t* n_queued) {
    if (!sv) return SLK_ERR_INVALID_ARG;
    slk_ctx* ctx = sv->ctx;
    ctx->err.clear();
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    struct Restore {
        int d;
        ~Restore() { if (d >= 0) cudaSetDevice(d); }
    } restore{prev};
    cudaStream_t s = ctx->stream;
    const int S = sv->S;
    // 1. admission, FIFO while a slot and memory are free
    while (!sv->queue.empty()) {
        const slk_status r = admit(sv, sv->queue.front());
        if (r == SLK_ERR_OOM) { ctx->err.clear(); break; }
        if (r != SLK_OK) return r;
        sv->queue.pop_front();
    }
    // 2. requests whose graph is ready start their first outer iteration
    bool any_iter = false;
    for (int slot = 0; slot < S; ++slot) {
        const int64_t id = sv->slot_req[slot];
        if (id < 0) continue;
        Request& r = sv->reqs[id];
        if (r.state == 1) {
            const cudaError_t q = cudaEventQuery(r.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return cuda_err(ctx, q, "request graph build");
            arena_free(sv, r.scratch);
            r.scratch = {0, 0};
            const int zero = 0, start = SLOT_START;
            SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->sd.mode + slot, &start, sizeof(int), cudaMemcpyHostToDevice, s));
            SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->sd.outer + slot, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
            SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->sd.inner_total + slot, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
            r.state = 2;
        }
        if (r.state == 2) any_iter = true;
    }
    // 3. one step of every iterating request
    if (any_iter) {
        const size_t pref_smem = sizeof(int) * (S + 1);
        const int grid_tiles = ctx->num_sms * 4;
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(srv_unary_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pref_smem));
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(srv_mode_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pref_smem));
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(srv_energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pref_smem));
        srv_unary_kernel<<<grid_tiles, 256, pref_smem, s>>>(sv->d_seg, S, sv->sd);
        srv_start_inner_kernel<<<1, 256, 0, s>>>(S, sv->sd, sv->d_ss);
        auto kern = srv_bound_kernel<256, SLK_SRV_BOUND_W>;
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pref_smem));
        int per_sm = 0;
        SLK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, pref_smem));
        if (per_sm < 1) return set_err(ctx, SLK_ERR_CUDA, "server bound kernel cannot be resident");
        const SegInfo* seg = sv->d_seg;
        int S_ = S, quantum = sv->cfg.quantum, max_inner = sv->p.max_inner;
        float tol = sv->p.tol_inner;
        SlotDev sd = sv->sd;
        SegState* ss = sv->d_ss;
        void* args[] = {(void*)&seg, (void*)&S_, (void*)&sd, (void*)&quantum, (void*)&max_inner, (void*)&tol,
                        (void*)&ss};
        SLK_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)kern, dim3(per_sm * ctx->num_sms), dim3(256),
                                                      args, pref_smem, s));
        srv_post_bound_kernel<<<(S + 255) / 256, 256, 0, s>>>(S, quantum, sv->sd);
        srv_swap_kernel<<<dim3(64, S), 256, 0, s>>>(sv->d_seg, S, sv->sd);
        srv_mode_kernel<8><<<grid_tiles, 256, pref_smem, s>>>(sv->d_seg, S, sv->sd);
        srv_mode_finish_kernel<<<S, 128, 0, s>>>(sv->d_seg, S, sv->sd);
        srv_energy_kernel<<<grid_tiles, 256, pref_smem, s>>>(sv->d_seg, S, sv->sd);
        srv_outer_update_kernel<<<(S + 255) / 256, 256, 0, s>>>(S, sv->p.max_outer, sv->sd);
        SLK_LAUNCH_CHECK(ctx, "server step");
        SLK_COUNT_LAUNCH(ctx, 10);
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->h_mode, sv->sd.mode, sizeof(int) * S, cudaMemcpyDeviceToHost, s));
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->h_outer, sv->sd.outer, sizeof(int) * S, cudaMemcpyDeviceToHost, s));
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->h_inner, sv->sd.inner_total, sizeof(int) * S, cudaMemcpyDeviceToHost, s));
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->h_energy, sv->sd.energy_out, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->h_sigma, sv->sd.sigma, sizeof(float) * S, cudaMemcpyDeviceToHost, s));
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->h_ss, sv->d_ss, sizeof(SegState), cudaMemcpyDeviceToHost, s));
        SLK_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (sv->h_ss->error) return set_err(ctx, SLK_ERR_TIMEOUT, "device-wide barrier of the server timed out");
        // 4. finished requests release their slot and memory
        for (int slot = 0; slot < S; ++slot) {
            const int64_t id = sv->slot_req[slot];
            if (id < 0 || sv->h_mode[slot] != SLOT_DONE) continue;
            Request& r = sv->reqs[id];
            r.stats.outer_iters = sv->h_outer[slot];
            r.stats.inner_iters_total = sv->h_inner[slot];
            r.stats.converged = sv->h_outer[slot] < sv->p.max_outer ? 1 : 0;
            r.stats.sigma = sv->h_sigma[slot];
            r.stats.energy = sv->h_energy[slot];
            r.stats.knn_fallback_rows = -1;
            r.stats.knn_float32_rows = -1;
            r.stats.knn_exact_rows = -1;
            r.state = 3;
            arena_free(sv, r.mem);
            r.mem = {0, 0};
            if (r.ev) { cudaEventDestroy(r.ev); r.ev = nullptr; }
            sv->slot_req[slot] = -1;
            const int idle = SLOT_IDLE;
            SLK_CUDA_TRY(ctx, cudaMemcpyAsync(sv->sd.mode + slot, &idle, sizeof(int), cudaMemcpyHostToDevice, s));
        }
    }
    int running = 0;
    for (int slot = 0; slot < S; ++slot) running += sv->slot_req[slot] >= 0;
    if (n_running) *n_running = running;
    if (n_queued) *n_queued = (int32_t)sv->queue.size();
    return SLK_OK;
}
