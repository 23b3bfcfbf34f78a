// Device code shared by the segment-indexed kernels (batched.cu, serve.cu):
// per-problem descriptors, the device-wide step barrier and the logits of one
// row with windowed neighbour gathers.
#pragma once

#include <math.h>

#include "slk_internal.cuh"
#include "sync.cuh"

namespace {

constexpr int kLPL = 4;  // labels per lane: L <= 128 with 32 lanes
constexpr unsigned long long kTimeoutNs = kSyncTimeoutNs;

struct SegInfo {
    const float* X;
    float* Z;            // caller's iterate (holds the result)
    float* Zs;           // scratch iterate (ping-pong partner)
    float* A;
    int32_t* labels;
    int32_t* modes;
    const int64_t* row_ptr;  // instance-local CSR
    const int32_t* col;
    const float* w;
    const float* sigma;      // device scalar
    int64_t N;
    int32_t L, D, G, moff;   // moff: first slot of this instance in mode_best
    float lambda;
    int32_t kdeg;
};

struct SegTile {
    int32_t inst, row, nrows, pad;
};

// Global words of the batched loops.
struct SegState {
    unsigned int arrive, gen, error, pad;
    int active_inner;  // instances still iterating in the current inner loop
    int active_outer;  // instances whose outer loop still runs
};

// Device-wide step barrier; the last block to arrive publishes "every
// instance has converged" (active_inner == 0) with the new generation.
// Returns 1 (all converged), 0 (go on), -1 (a wait gave up).
__device__ int seg_step(SegState* ss, unsigned nblocks) {
    __shared__ int s_res;
    __syncthreads();
    if (threadIdx.x == 0) {
        int res = 0;
        const unsigned gen = ld_acq(&ss->gen);
        __threadfence();
        const unsigned prev = atom_add_ar(&ss->arrive, 1u);
        if (prev == nblocks - 1) {
            ss->arrive = 0;
            const unsigned done = (ld_acq_i(&ss->active_inner) <= 0) ? 0x80000000u : 0u;
            st_rel(&ss->gen, ((gen + 1u) & 0x7fffffffu) | done);
            res = done ? 1 : 0;
        } else {
            const unsigned long long t0 = globaltimer_ns();
            unsigned polls = 0, v;
            while ((v = ld_acq(&ss->gen)) == gen) {
                if ((++polls & 63u) == 0u) {
                    if (ld_acq(&ss->error) != 0u) { res = -1; break; }
                    if (globaltimer_ns() - t0 > kTimeoutNs) {
                        atomicOr(&ss->error, 1u);
                        res = -1;
                        break;
                    }
                }
            }
            if (res == 0) res = (v & 0x80000000u) ? 1 : 0;
        }
        s_res = res;
    }
    __syncthreads();
    return s_res;
}

__device__ __forceinline__ float gmax(float v, unsigned m, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(m, v, o, G));
    return v;
}
__device__ __forceinline__ float gsum(float v, unsigned m, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o, G);
    return v;
}

// Pairwise term b of row p (lane gl of a G-lane group; labels gl + G j):
// the neighbours' iterates summed in CSR order with windowed gathers from Zin.
template <int W>
__device__ __forceinline__ void seg_pair(const SegInfo& si, int64_t p, int gl, unsigned gm,
                                         const float* Zin, bool with_pair, float (&b)[kLPL]) {
    const int G = si.G, L = si.L;
#pragma unroll
    for (int j = 0; j < kLPL; ++j) b[j] = 0.f;
    if (with_pair) {
        int64_t e0;
        int cnt;
        if (si.kdeg > 0) {
            e0 = p * si.kdeg;
            cnt = si.kdeg;
        } else {
            e0 = si.row_ptr[p];
            cnt = (int)(si.row_ptr[p + 1] - e0);
        }
        for (int c0 = 0; c0 < cnt; c0 += G) {
            int myq = 0;
            float myw = 1.f;
            if (gl < cnt - c0) {
                myq = __ldg(si.col + e0 + c0 + gl);
                if (si.w) myw = __ldg(si.w + e0 + c0 + gl);
            }
            const int cm = min(G, cnt - c0);
            for (int t0 = 0; t0 < cm; t0 += W) {
                float zz[W][kLPL], ww[W];
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const int t = t0 + u;
                    if (t >= cm) break;   // uniform within the group (one row)
                    const int src = t < G ? t : 0;
                    const int q = __shfl_sync(gm, myq, src, G);
                    ww[u] = __shfl_sync(gm, myw, src, G);
                    const float* zq = Zin + (int64_t)q * L;
#pragma unroll
                    for (int j = 0; j < kLPL; ++j) {
                        const int l = gl + G * j;
                        zz[u][j] = (t < cm && l < L) ? __ldcg(zq + l) : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    if (t0 + u >= cm) break;
#pragma unroll
                    for (int j = 0; j < kLPL; ++j) b[j] = fmaf(ww[u], zz[u][j], b[j]);
                }
            }
        }
    }
}

// Logits s = a + lambda b of row p (b as in seg_pair).
template <int W>
__device__ __forceinline__ void seg_logits(const SegInfo& si, int64_t p, int gl, unsigned gm,
                                           const float* Zin, bool with_pair, float (&s)[kLPL]) {
    const int G = si.G, L = si.L;
    float b[kLPL];
    seg_pair<W>(si, p, gl, gm, Zin, with_pair, b);
    const float* ap = si.A + p * (int64_t)L;
#pragma unroll
    for (int j = 0; j < kLPL; ++j) {
        const int l = gl + G * j;
        s[j] = (l < L) ? fmaf(si.lambda, b[j], __ldg(ap + l)) : -INFINITY;
    }
}

__device__ __forceinline__ void load_seg(const SegInfo* seg, int b, SegInfo& si) { si = seg[b]; }

}  // namespace
