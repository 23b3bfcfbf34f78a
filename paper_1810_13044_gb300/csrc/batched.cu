// Batched SLK-BO: many independent problems of different N, D, L in one
// pass of segment-indexed kernels (slk_solve_batched, include/slk.h).
//
// Every problem ("instance") keeps its own buffers (caller's Z, labels,
// modes; its own kNN CSR with local indices, A and a scratch iterate).  A
// table of per-instance descriptors (SegInfo) and a table of work tiles
// (SegTile: a few consecutive rows of one instance) drive the kernels:
//   seg_unary_kernel        a_{p,l} = k(x_p, m_l), z_p = softmax(a_p)      [Eq. general-second, Alg. 1]
//   seg_bound_kernel        persistent z-updates, Eq. (soft-max), for all instances, with a
//                           per-instance convergence test (its own delta ring and count)
//   seg_mode_kernel         modes, Eq. (mode_byproduct), on log z; labels
//   seg_energy_kernel       Eq. (1) in float64 per instance
// A warp works on one tile at a time; the G lanes of a group own one row
// (G = the power of two >= L of that instance, at most 32, two labels per
// lane beyond 32).  Instances whose outer loop has stopped are skipped.
#include <math.h>
#include <string.h>

#include <map>
#include <vector>

#include "seg_common.cuh"

namespace {

// ------------------------------------------------------------------ unary

// One block per 32-row tile of one instance: a_{p,l} = exp(-||x_p - x_{m_l}||^2
// / (2 sigma^2)) (float32 chunk sums, float64 total), z_p = softmax(a_p).
__global__ void __launch_bounds__(256)
seg_unary_kernel(const SegInfo* __restrict__ seg, const SegTile* __restrict__ tiles,
                 const int* __restrict__ outer_active) {
    __shared__ float xs[32][33];
    __shared__ float ms[SLK_BATCH_MAX_L][33];
    __shared__ float at[32][SLK_BATCH_MAX_L + 1];
    __shared__ int mrow[SLK_BATCH_MAX_L];
    const SegTile tl = tiles[blockIdx.x];
    if (!outer_active[tl.inst]) return;
    SegInfo si;
    load_seg(seg, tl.inst, si);
    const int t = threadIdx.x, pl = t & 31, lb = t >> 5;
    const int L = si.L, D = si.D;
    for (int l = t; l < L; l += 256) mrow[l] = si.modes[l];
    constexpr int LPT = SLK_BATCH_MAX_L / 8;   // labels per thread
    double acc[LPT];
#pragma unroll
    for (int j = 0; j < LPT; ++j) acc[j] = 0.0;
    __syncthreads();
    for (int d0 = 0; d0 < D; d0 += 32) {
        const int dc = min(32, D - d0);
        for (int i = t; i < 32 * 32; i += 256) {
            const int r = i >> 5, c = i & 31;
            xs[r][c] = (r < tl.nrows && c < dc) ? si.X[(int64_t)(tl.row + r) * D + d0 + c] : 0.f;
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
            if (pl < tl.nrows) si.A[(int64_t)(tl.row + pl) * L + l] = a;
        }
    }
    __syncthreads();
    if (t < tl.nrows) {
        float m = at[t][0];
        for (int l = 1; l < L; ++l) m = fmaxf(m, at[t][l]);
        float sm = 0.f;
        for (int l = 0; l < L; ++l) sm += expf(at[t][l] - m);
        float* zr = si.Z + (int64_t)(tl.row + t) * L;
        for (int l = 0; l < L; ++l) zr[l] = expf(at[t][l] - m) / sm;
    }
}

// ------------------------------------------------------------------ z-updates

// Persistent inner loop over all instances.  Update `it` of instance b reads
// its buffer it % 2 (Z, then Zs) and writes the other.  Instance b stops at
// the first update whose predecessor's max |dz| (delta[3 b + slot]) was <=
// tol, which block 0 records in iters[b] (leaving the active count).  At the
// start of every update each block lists the instances still updating
// (the same list in every block: it only reads values that are final for
// this update) and scans their tile counts in shared memory, so the warps
// spread only the live tiles; the loop ends when no instance is active.
template <int THREADS, int W>
__global__ void __launch_bounds__(THREADS)
seg_bound_kernel(const SegInfo* __restrict__ seg, const SegTile* __restrict__ tiles,
                 const int* __restrict__ tile0, int count, int max_iters, float tol, SegState* ss,
                 unsigned* __restrict__ delta, int* __restrict__ iters,
                 const int* __restrict__ outer_active) {
    extern __shared__ int pref[];   // [count + 1]: exclusive prefix of live tiles
    __shared__ int wsum[THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (THREADS / 32);
    const int64_t gwarp = (int64_t)blockIdx.x * (THREADS / 32) + wid;
    const int per = (count + THREADS - 1) / THREADS;
    for (int it = 0; it < max_iters; ++it) {
        // ---- live instances of this update and their tile counts
        int local = 0;
        const int b0 = threadIdx.x * per;
        for (int b = b0; b < min(count, b0 + per); ++b) {
            bool act = outer_active[b] != 0;
            if (act) {
                const int ib = *(volatile int*)&iters[b];
                if (ib >= 0 && ib < it) act = false;
            }
            if (act && it > 0) {
                const float dprev = __uint_as_float(ld_acq(&delta[3 * b + (it - 1) % 3]));
                if (dprev <= tol) {
                    act = false;
                    if (blockIdx.x == 0 && atomicCAS(&iters[b], -1, it) == -1)
                        atomicSub(&ss->active_inner, 1);
                }
            }
            if (act && blockIdx.x == 0) delta[3 * b + (it + 1) % 3] = 0u;
            const int c = act ? tile0[b + 1] - tile0[b] : 0;
            pref[b] = c;
            local += c;
        }
        // block scan of the per-thread sums
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
        for (int b = b0; b < min(count, b0 + per); ++b) {
            const int c = pref[b];
            pref[b] = run;
            run += c;
        }
        if (threadIdx.x == THREADS - 1) pref[count] = run;
        __syncthreads();
        const int total = pref[count];
        // ---- the live tiles, spread over all warps
        for (int64_t wi = gwarp; wi < total; wi += nwarps) {
            int lo = 0, hi = count;   // last b with pref[b] <= wi
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pref[mid] <= wi) lo = mid; else hi = mid;
            }
            const int b = lo;
            const SegTile tl = tiles[tile0[b] + (wi - pref[b])];
            SegInfo si;
            load_seg(seg, b, si);
            const int G = si.G, grp = lane / G, gl = lane % G;
            const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
            const float* Zin = (it & 1) ? si.Zs : si.Z;
            float* Zout = (it & 1) ? si.Z : si.Zs;
            float d = 0.f;
            if (grp < tl.nrows) {
                const int64_t p = tl.row + grp;
                float sv[kLPL];
                seg_logits<W>(si, p, gl, gm, Zin, true, sv);
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
                const int64_t off = p * (int64_t)si.L;
#pragma unroll
                for (int j = 0; j < kLPL; ++j) {
                    const int l = gl + G * j;
                    if (l < si.L) {
                        const float z = e[j] / sum;
                        d = fmaxf(d, fabsf(z - __ldcg(Zin + off + l)));
                        __stcg(Zout + off + l, z);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
            if (lane == 0) atomicMax(&delta[3 * b + it % 3], __float_as_uint(d));
        }
        const int r = seg_step(ss, gridDim.x);
        if (r < 0) return;
        if (r == 1) break;
    }
}

// Instances still running after max_iters ran all of them; then move every
// instance's last iterate into Z (it sits in Zs after an odd count).
__global__ void seg_finish_iters_kernel(int count, int max_iters, int* iters,
                                        const int* outer_active) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x)
        if (outer_active[b] && iters[b] < 0) iters[b] = max_iters;
}

__global__ void seg_swap_kernel(const SegInfo* __restrict__ seg, const SegTile* __restrict__ tiles,
                                const int* __restrict__ iters, const int* __restrict__ outer_active) {
    const SegTile tl = tiles[blockIdx.x];
    if (!outer_active[tl.inst] || (iters[tl.inst] & 1) == 0) return;
    const SegInfo si = seg[tl.inst];
    const int64_t base = (int64_t)tl.row * si.L;
    const int64_t n = (int64_t)tl.nrows * si.L;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float a = si.Z[base + i];
        si.Z[base + i] = si.Zs[base + i];
        si.Zs[base + i] = a;
    }
}

// ------------------------------------------------------------------ modes

// Per row: logits from the previous iterate (Zs after the swap; s = a when
// no update ran), label = argmax_l s (ties to smaller l), keys
// log z = (s_l - max s) - log1p(sum_{j != argmax} exp(s_j - max s)); the
// warp reduces each label's best (key, ~row) over its rows, then one 64-bit
// max per label and tile.
template <int W>
__global__ void __launch_bounds__(256)
seg_mode_kernel(const SegInfo* __restrict__ seg, const SegTile* __restrict__ tiles,
                int64_t ntiles, const int* __restrict__ iters, const int* __restrict__ outer_active,
                unsigned long long* __restrict__ mode_best) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    for (int64_t ti = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); ti < ntiles; ti += nwarps) {
        const SegTile tl = tiles[ti];
        const int b = tl.inst;
        if (!outer_active[b]) continue;
        SegInfo si;
        load_seg(seg, b, si);
        const int G = si.G, grp = lane / G, gl = lane % G;
        const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
        const bool live = grp < tl.nrows;
        const int64_t p = tl.row + (live ? grp : 0);
        unsigned long long best[kLPL];
#pragma unroll
        for (int j = 0; j < kLPL; ++j) best[j] = 0ull;
        if (live) {
            float s[kLPL];
            seg_logits<W>(si, p, gl, gm, si.Zs, iters[b] > 0, s);
            float m = s[0];
            int jl = gl;
#pragma unroll
            for (int j = 1; j < kLPL; ++j)
                if (s[j] > m) { m = s[j]; jl = gl + G * j; }
            for (int o = G >> 1; o > 0; o >>= 1) {
                const float om = __shfl_xor_sync(gm, m, o, G);
                const int ol = __shfl_xor_sync(gm, jl, o, G);
                if (om > m || (om == m && ol < jl)) { m = om; jl = ol; }
            }
            float r = 0.f;
#pragma unroll
            for (int j = 0; j < kLPL; ++j) {
                const int l = gl + G * j;
                if (l < si.L && l != jl) r += expf(s[j] - m);
            }
            r = gsum(r, gm, G);
            const float lse1 = log1pf(r);
            if (gl == 0) si.labels[p] = jl;
#pragma unroll
            for (int j = 0; j < kLPL; ++j) {
                const int l = gl + G * j;
                if (l < si.L)
                    best[j] = ((unsigned long long)float_to_ordered((s[j] - m) - lse1) << 32) |
                              (unsigned long long)(0xffffffffu - (unsigned)p);
            }
        }
        // reduce across the groups of the warp (same label slot, other rows)
#pragma unroll
        for (int j = 0; j < kLPL; ++j) {
            for (int o = G; o < 32; o <<= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best[j], o);
                if (ob > best[j]) best[j] = ob;
            }
            const int l = lane + G * j;
            if (lane < G && l < si.L && best[j]) atomicMax(&mode_best[si.moff + l], best[j]);
        }
    }
}

// Per instance: new modes from the packed maxima, changed flag.
__global__ void seg_mode_finish_kernel(const SegInfo* __restrict__ seg, int count,
                                       const int* __restrict__ outer_active,
                                       unsigned long long* __restrict__ mode_best,
                                       int* __restrict__ changed) {
    const int b = blockIdx.x;
    if (b >= count || !outer_active[b]) return;
    const SegInfo si = seg[b];
    __shared__ int ch;
    if (threadIdx.x == 0) ch = 0;
    __syncthreads();
    for (int l = threadIdx.x; l < si.L; l += blockDim.x) {
        const unsigned long long v = mode_best[si.moff + l];
        const int q = (int)(0xffffffffu - (unsigned)(v & 0xffffffffull));
        if (q != si.modes[l]) ch = 1;
        si.modes[l] = q;
        mode_best[si.moff + l] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) changed[b] = ch;
}

// ------------------------------------------------------------------ energy

__global__ void __launch_bounds__(256)
seg_energy_kernel(const SegInfo* __restrict__ seg, const SegTile* __restrict__ tiles,
                  int64_t ntiles, const int* __restrict__ outer_active, double* __restrict__ energy) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    for (int64_t ti = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); ti < ntiles; ti += nwarps) {
        const SegTile tl = tiles[ti];
        const int b = tl.inst;
        if (!outer_active[b]) continue;
        SegInfo si;
        load_seg(seg, b, si);
        const double sg = (double)*si.sigma;
        const double inv2s2 = 1.0 / (2.0 * sg * sg);
        double acc = 0.0, my_d2 = 0.0, my_cut = 0.0;
        bool mine = false;
        int slot = 0;
        for (int r = 0; r < tl.nrows; ++r) {
            const int64_t p = tl.row + r;
            const int lp = si.labels[p];
            const float* xp = si.X + p * si.D;
            const float* xm = si.X + (int64_t)si.modes[lp] * si.D;
            const double d2 = warp_sq_dist(xp, xm, nullptr, si.D, lane);
            int64_t e0, e1;
            if (si.kdeg > 0) { e0 = p * si.kdeg; e1 = e0 + si.kdeg; }
            else { e0 = si.row_ptr[p]; e1 = si.row_ptr[p + 1]; }
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
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) atomicAdd(&energy[b], acc);
    }
}

// End of an outer iteration: count it for the instances that ran, add their
// z-updates, keep running the ones whose modes changed, reset the inner-loop
// words of the next outer iteration.
__global__ void seg_outer_update_kernel(int count, int* outer_active, const int* changed,
                                        int* iters, int* outer_done, int* inner_total,
                                        unsigned* delta, double* energy, double* energy_out,
                                        SegState* ss) {
    __shared__ int n_active;
    if (threadIdx.x == 0) n_active = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
        if (outer_active[b]) {
            outer_done[b] += 1;
            inner_total[b] += max(iters[b], 0);
            energy_out[b] = energy[b];
            if (!changed[b]) outer_active[b] = 0;
        }
        iters[b] = -1;
        energy[b] = 0.0;
        delta[3 * b] = delta[3 * b + 1] = delta[3 * b + 2] = 0u;
        if (outer_active[b]) atomicAdd(&n_active, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ss->active_outer = n_active;
        ss->active_inner = n_active;
        ss->arrive = 0;
    }
}

struct TuneKey {
    int count;
    int64_t rows;
    bool operator<(const TuneKey& o) const {
        return count != o.count ? count < o.count : rows < o.rows;
    }
};
struct TuneChoice {
    int threads, window;
};

std::map<const void*, std::map<TuneKey, TuneChoice>> g_tuned;  // per context

}  // namespace

// ------------------------------------------------------------------ host driver

namespace {

int pow2_at_least(int x) {
    int g = 1;
    while (g < x) g <<= 1;
    return g;
}

// Lanes per row of an instance in the segment-indexed kernels; the tile
// tables and the kernels' tile counts both come from it.
int seg_group(int L) { return std::min(32, pow2_at_least(L)); }

slk_status launch_seg_bound(slk_ctx* ctx, const TuneChoice& tc, const SegInfo* seg,
                            const SegTile* tiles, const int* tile0, int count, int64_t ntiles,
                            int max_iters, float tol, SegState* ss, unsigned* delta, int* iters,
                            const int* outer_active) {
    const void* kern = nullptr;
    if (tc.threads == 256 && tc.window == 8) kern = (const void*)seg_bound_kernel<256, 8>;
    else if (tc.threads == 256) kern = (const void*)seg_bound_kernel<256, 4>;
    else if (tc.window == 8) kern = (const void*)seg_bound_kernel<512, 8>;
    else kern = (const void*)seg_bound_kernel<512, 4>;
    const size_t smem = sizeof(int) * (count + 1);
    SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SLK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tc.threads, smem));
    if (per_sm < 1) return set_err(ctx, SLK_ERR_CUDA, "segmented bound kernel cannot be resident");
    int64_t grid = (int64_t)per_sm * ctx->num_sms;
    const int64_t need = (ntiles + tc.threads / 32 - 1) / (tc.threads / 32);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    void* args[] = {(void*)&seg, (void*)&tiles, (void*)&tile0, (void*)&count, (void*)&max_iters,
                    (void*)&tol, (void*)&ss, (void*)&delta, (void*)&iters, (void*)&outer_active};
    cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)grid), dim3(tc.threads), args,
                                                smem, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "seg_bound_kernel");
    SLK_COUNT_LAUNCH(ctx, 1);
    return SLK_OK;
}

}  // namespace

extern "C" slk_status slk_solve_batched(slk_ctx* ctx, const slk_instance* inst, int32_t count,
                                        const slk_params* params, slk_stats* stats) {
    if (!ctx) return SLK_ERR_INVALID_ARG;
    ctx->err.clear();
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
        return set_err(ctx, SLK_ERR_CUDA, "cannot select device %d", ctx->device);
    struct Restore {
        int d;
        ~Restore() { if (d >= 0) cudaSetDevice(d); }
    } restore{prev_dev};
    slk_params p;
    if (params) p = *params; else slk_default_params(&p);
    if (!inst || count < 1 || count > SLK_BATCH_MAX_COUNT)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "need 1 <= count <= %d instances", SLK_BATCH_MAX_COUNT);
    if (p.max_outer < 1 || p.max_inner < 1)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "max_outer and max_inner must be >= 1");
    if (p.symmetrize != 0)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "the batched form runs on the directed kNN graph only");
    for (int b = 0; b < count; ++b) {
        const slk_instance& q = inst[b];
        if (!q.X || !q.init_modes || !q.Z || !q.labels || !q.modes)
            return set_err(ctx, SLK_ERR_INVALID_ARG, "instance %d: required pointer is NULL", b);
        if (q.N < 2 || q.N >= (int64_t)0x7fffffff || q.D < 1 || q.L < 1 || q.L > SLK_BATCH_MAX_L ||
            q.L > q.N || q.k < 1 || q.k > SLK_MAX_K || q.k > q.N - 1)
            return set_err(ctx, SLK_ERR_INVALID_ARG, "instance %d: bad sizes (N=%lld D=%d L=%d k=%d)",
                           b, (long long)q.N, q.D, q.L, q.k);
    }
    // ---- workspace: per instance graph + A + Zs; shared kNN scratch; tables
    size_t knn_max = 0;
    int64_t rows_total = 0, z_total = 0, nnz_total = 0, L_total = 0, ntiles = 0, nutiles = 0;
    for (int b = 0; b < count; ++b) {
        const slk_instance& q = inst[b];
        knn_max = std::max(knn_max, knn_ws_bytes(ctx, q.N, q.D, q.k, p.knn_precision));
        rows_total += q.N;
        z_total += q.N * q.L;
        nnz_total += q.N * q.k;
        L_total += q.L;
        const int rows_per_tile = 32 / seg_group(q.L);
        ntiles += (q.N + rows_per_tile - 1) / rows_per_tile;
        nutiles += (q.N + 31) / 32;
    }
    constexpr int kAux = 8;   // graphs of different instances are built on kAux streams
    size_t need = kAux * (align_up(knn_max, 256) + align_up(sizeof(DevState), 256)) + 4096;
    need += count * (align_up(sizeof(int64_t) * 1, 256));  // slack
    need += align_up(sizeof(int64_t) * (rows_total + count), 256);
    need += 3 * align_up(sizeof(float) * nnz_total, 256) + align_up(sizeof(int32_t) * nnz_total, 256);
    need += 2 * align_up(sizeof(float) * z_total, 256);
    need += align_up(sizeof(SegInfo) * count, 256) + align_up(sizeof(SegTile) * (ntiles + nutiles), 256);
    need += align_up(sizeof(int) * (count + 1), 256);
    need += align_up(sizeof(unsigned long long) * L_total, 256) + align_up(sizeof(SegState), 256);
    need += align_up(sizeof(unsigned) * 3 * count, 256) + 6 * align_up(sizeof(int) * count, 256);
    need += 2 * align_up(sizeof(double) * count, 256) + align_up(sizeof(float) * count, 256);
    need += (size_t)count * 8 * 256 + 64 * 256;   // alignment of the per-instance slices
    slk_status r = ensure_ws(ctx, need);
    if (r != SLK_OK) return r;
    WsCarver wc(ctx->ws);
    void* knn_ws[kAux];
    DevState* aux_st[kAux];
    for (int i = 0; i < kAux; ++i) {
        knn_ws[i] = wc.take<unsigned char>(knn_max);
        aux_st[i] = wc.take<DevState>(1);
    }
    while ((int)ctx->aux.size() < kAux) {
        cudaStream_t a = nullptr;
        cudaEvent_t e = nullptr;
        SLK_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
        SLK_CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->aux.push_back(a);
        ctx->aux_ev.push_back(e);
    }
    SegInfo* d_seg = wc.take<SegInfo>(count);
    SegTile* d_tiles = wc.take<SegTile>(ntiles);
    SegTile* d_utiles = wc.take<SegTile>(nutiles);
    int* d_tile0 = wc.take<int>(count + 1);
    std::vector<int> tile0(count + 1, 0);
    unsigned long long* d_best = wc.take<unsigned long long>(L_total);
    SegState* d_ss = wc.take<SegState>(1);
    unsigned* d_delta = wc.take<unsigned>(3 * count);
    int* d_iters = wc.take<int>(count);
    int* d_active = wc.take<int>(count);
    int* d_changed = wc.take<int>(count);
    int* d_outer = wc.take<int>(count);
    int* d_inner = wc.take<int>(count);
    double* d_energy = wc.take<double>(count);
    double* d_energy_out = wc.take<double>(count);
    float* d_sigma = wc.take<float>(count);
    std::vector<SegInfo> seg(count);
    std::vector<SegTile> tiles, utiles;
    tiles.reserve(ntiles);
    utiles.reserve(nutiles);
    cudaStream_t s = ctx->stream;
    // the auxiliary streams start after everything already on the main stream
    SLK_CUDA_TRY(ctx, cudaEventRecord(ctx->aux_ev[0], s));
    for (int i = 0; i < kAux; ++i) SLK_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->aux[i], ctx->aux_ev[0], 0));
    int moff = 0;
    for (int b = 0; b < count; ++b) {
        const int lane_s = b % kAux;
        DevState* st = aux_st[lane_s];
        ctx->stream = ctx->aux[lane_s];   // the launchers below enqueue on ctx->stream
        const slk_instance& q = inst[b];
        SegInfo& si = seg[b];
        int64_t* row_ptr = wc.take<int64_t>(q.N + 1);
        int32_t* col = wc.take<int32_t>(q.N * q.k);
        float* dist2 = wc.take<float>(q.N * q.k);
        float* wts = (p.affinity == SLK_AFFINITY_HEAT) ? wc.take<float>(q.N * q.k) : nullptr;
        si.A = wc.take<float>(q.N * q.L);
        si.Zs = wc.take<float>(q.N * q.L);
        si.X = q.X;
        si.Z = q.Z;
        si.labels = q.labels;
        si.modes = q.modes;
        si.row_ptr = row_ptr;
        si.col = col;
        si.w = wts;
        si.sigma = d_sigma + b;
        si.N = q.N;
        si.L = q.L;
        si.D = q.D;
        si.G = seg_group(q.L);
        si.moff = moff;
        si.lambda = q.lambda;
        si.kdeg = q.k;
        moff += q.L;
        // the instance's graph and kernel width (same kernels as slk_solve)
        r = knn_graph_launch(ctx, q.X, q.N, q.D, q.k, p.knn_precision, row_ptr, col, dist2,
                             knn_ws[lane_s], st);
        if (r != SLK_OK) { ctx->stream = s; return r; }
        r = (q.sigma > 0.f) ? set_sigma_launch(ctx, q.sigma, st)
                            : sigma_launch(ctx, dist2, q.N * (int64_t)q.k, p.sigma_rule, st);
        if (r != SLK_OK) { ctx->stream = s; return r; }
        cudaError_t ce = cudaMemcpyAsync(d_sigma + b, &st->sigma, sizeof(float),
                                         cudaMemcpyDeviceToDevice, ctx->stream);
        if (ce == cudaSuccess && wts)
            r = weights_launch(ctx, dist2, q.N * (int64_t)q.k, SLK_AFFINITY_HEAT, d_sigma + b, wts);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(q.modes, q.init_modes, sizeof(int32_t) * q.L,
                                 cudaMemcpyDeviceToDevice, ctx->stream);
        ctx->stream = s;
        if (ce != cudaSuccess) return cuda_err(ctx, ce, "batched graph set-up");
        if (r != SLK_OK) return r;
        const int rpt = 32 / si.G;
        tile0[b] = (int)tiles.size();
        for (int64_t r0 = 0; r0 < q.N; r0 += rpt)
            tiles.push_back({b, (int32_t)r0, (int32_t)std::min<int64_t>(rpt, q.N - r0), 0});
        for (int64_t r0 = 0; r0 < q.N; r0 += 32)
            utiles.push_back({b, (int32_t)r0, (int32_t)std::min<int64_t>(32, q.N - r0), 0});
    }
    // join: the main stream continues once every auxiliary stream is done
    for (int i = 0; i < kAux; ++i) {
        SLK_CUDA_TRY(ctx, cudaEventRecord(ctx->aux_ev[i], ctx->aux[i]));
        SLK_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->aux_ev[i], 0));
    }
    // tables and per-instance state (pageable copies: staged by the driver)
    if ((int64_t)tiles.size() != ntiles || (int64_t)utiles.size() != nutiles)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "batched tile tables disagree with their counts");
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(d_seg, seg.data(), sizeof(SegInfo) * count, cudaMemcpyHostToDevice, s));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(SegTile) * ntiles, cudaMemcpyHostToDevice, s));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(d_utiles, utiles.data(), sizeof(SegTile) * nutiles, cudaMemcpyHostToDevice, s));
    tile0[count] = (int)tiles.size();
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(d_tile0, tile0.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_best, 0, sizeof(unsigned long long) * L_total, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_ss, 0, sizeof(SegState), s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_delta, 0, sizeof(unsigned) * 3 * count, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_iters, 0xff, sizeof(int) * count, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_outer, 0, sizeof(int) * count, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_inner, 0, sizeof(int) * count, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_energy, 0, sizeof(double) * count, s));
    SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_changed, 0, sizeof(int) * count, s));
    {
        std::vector<int> ones(count, 1);
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(d_active, ones.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
        const SegState init{0u, 0u, 0u, 0u, count, count};
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(d_ss, &init, sizeof(SegState), cudaMemcpyHostToDevice, s));
        SLK_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // host vectors go out of scope
    }
    // ---- autotune the z-update launch shape once per (count, rows)
    const TuneKey key{count, rows_total};
    auto& cache = g_tuned[ctx];
    TuneChoice tc{256, 8};
    auto hit = cache.find(key);
    if (hit != cache.end()) {
        tc = hit->second;
    } else {
        const TuneChoice cands[4] = {{256, 8}, {256, 4}, {512, 8}, {512, 4}};
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        SLK_CUDA_TRY(ctx, cudaEventCreate(&e0));
        SLK_CUDA_TRY(ctx, cudaEventCreate(&e1));
        seg_unary_kernel<<<(unsigned)nutiles, 256, 0, s>>>(d_seg, d_utiles, d_active);
        SLK_COUNT_LAUNCH(ctx, 1);
        for (const TuneChoice& c : cands) {
            const SegState init{0u, 0u, 0u, 0u, count, count};
            SLK_CUDA_TRY(ctx, cudaMemcpyAsync(d_ss, &init, sizeof(SegState), cudaMemcpyHostToDevice, s));
            SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_iters, 0xff, sizeof(int) * count, s));
            SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_delta, 0, sizeof(unsigned) * 3 * count, s));
            SLK_CUDA_TRY(ctx, cudaEventRecord(e0, s));
            r = launch_seg_bound(ctx, c, d_seg, d_tiles, d_tile0, count, ntiles, 4, -1.f, d_ss, d_delta,
                                 d_iters, d_active);
            if (r != SLK_OK) return r;
            SLK_CUDA_TRY(ctx, cudaEventRecord(e1, s));
            SLK_CUDA_TRY(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            SLK_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) { best_ms = ms; tc = c; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cache[key] = tc;
        const SegState init{0u, 0u, 0u, 0u, count, count};
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(d_ss, &init, sizeof(SegState), cudaMemcpyHostToDevice, s));
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_iters, 0xff, sizeof(int) * count, s));
        SLK_CUDA_TRY(ctx, cudaMemsetAsync(d_delta, 0, sizeof(unsigned) * 3 * count, s));
        SLK_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    // ---- one outer iteration of every active instance, captured once
    SegState* h_ss = static_cast<SegState*>(ctx->host_pin);
    auto enqueue_outer = [&]() -> slk_status {
        seg_unary_kernel<<<(unsigned)nutiles, 256, 0, s>>>(d_seg, d_utiles, d_active);
        slk_status rr = launch_seg_bound(ctx, tc, d_seg, d_tiles, d_tile0, count, ntiles, p.max_inner,
                                         p.tol_inner, d_ss, d_delta, d_iters, d_active);
        if (rr != SLK_OK) return rr;
        seg_finish_iters_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, p.max_inner, d_iters, d_active);
        seg_swap_kernel<<<(unsigned)nutiles, 256, 0, s>>>(d_seg, d_utiles, d_iters, d_active);
        int64_t mg = (ntiles + 7) / 8;
        if (mg > (int64_t)ctx->num_sms * 16) mg = (int64_t)ctx->num_sms * 16;
        seg_mode_kernel<8><<<(unsigned)mg, 256, 0, s>>>(d_seg, d_tiles, ntiles, d_iters, d_active, d_best);
        seg_mode_finish_kernel<<<count, 64, 0, s>>>(d_seg, count, d_active, d_best, d_changed);
        seg_energy_kernel<<<(unsigned)mg, 256, 0, s>>>(d_seg, d_tiles, ntiles, d_active, d_energy);
        seg_outer_update_kernel<<<1, 256, 0, s>>>(count, d_active, d_changed, d_iters, d_outer, d_inner,
                                                 d_delta, d_energy, d_energy_out, d_ss);
        SLK_CUDA_TRY(ctx, cudaMemcpyAsync(h_ss, d_ss, sizeof(SegState), cudaMemcpyDeviceToHost, s));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(ctx, e, "batched outer iteration");
        return SLK_OK;
    };
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = false;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const long long launches_before = ctx->launches;
        const slk_status rr = enqueue_outer();
        const cudaError_t ec = cudaStreamEndCapture(s, &graph);
        ctx->launches = launches_before;   // counted per replay below
        if (rr == SLK_OK && ec == cudaSuccess && graph &&
            cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess) {
            use_graph = true;
        } else {
            cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            graph = nullptr;
            ctx->launches = launches_before;
            ctx->err.clear();
        }
    } else {
        cudaGetLastError();
    }
    int outer = 0;
    PhaseScope loop_scope(ctx, SLK_PHASE_BOUND);
    for (outer = 0; outer < p.max_outer; ++outer) {
        if (use_graph) {
            SLK_CUDA_TRY(ctx, cudaGraphLaunch(gexec, s));
            SLK_COUNT_LAUNCH(ctx, 9);
        } else {
            r = enqueue_outer();
            if (r != SLK_OK) return r;
            SLK_COUNT_LAUNCH(ctx, 8);   // + the z-update launch counted inside
        }
        SLK_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (h_ss->error) {
            if (gexec) cudaGraphExecDestroy(gexec);
            if (graph) cudaGraphDestroy(graph);
            return set_err(ctx, SLK_ERR_TIMEOUT, "device-wide barrier of the batched kernel timed out");
        }
        if (h_ss->active_outer == 0) { ++outer; break; }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    // ---- per-instance results
    std::vector<int> h_outer(count), h_inner(count), h_active(count);
    std::vector<double> h_energy(count);
    std::vector<float> h_sigma(count);
    std::vector<long long> dummy;
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(h_outer.data(), d_outer, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(h_inner.data(), d_inner, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(h_active.data(), d_active, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(h_energy.data(), d_energy_out, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    SLK_CUDA_TRY(ctx, cudaMemcpyAsync(h_sigma.data(), d_sigma, sizeof(float) * count, cudaMemcpyDeviceToHost, s));
    SLK_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    bool all_conv = true;
    for (int b = 0; b < count; ++b) {
        const bool conv = h_active[b] == 0;
        all_conv = all_conv && conv;
        if (stats) {
            stats[b].outer_iters = h_outer[b];
            stats[b].inner_iters_total = h_inner[b];
            stats[b].converged = conv ? 1 : 0;
            stats[b].sigma = h_sigma[b];
            stats[b].energy = h_energy[b];
            stats[b].knn_fallback_rows = -1;
            stats[b].ms_iters_total = 0;
            stats[b].knn_float32_rows = -1;
            stats[b].knn_exact_rows = -1;
        }
    }
    (void)use_graph;
    return all_conv ? SLK_OK : SLK_NOT_CONVERGED;
}
