// bfloat16 tensor-core (tcgen05) distance tiles for the kNN candidates.
//
// Computes dt(p, q) = ||xt_p||^2 + ||xt_q||^2 - 2 xt_p . xt_q for 128 x 256
// tiles (p: a 128-row block, q: a 256-column tile) with the dot products on
// the 5th-generation tensor cores, and keeps per row the KC smallest
// (dt, q) of a column split -- the same contract as the float32 SIMT
// candidate kernel; the exact float32 rerank and its certificate follow.
// The epilogue forms w = fl(||xt_q||^2 - 2 dot) and compares it with the
// row's threshold less ||xt_p||^2 rounded upward, so that a rejected column
// has dt = fl(w + ||xt_p||^2) >= threshold; the survivors store that dt
// (two roundings, as fl(-2 dot + fl(||xt_p||^2 + ||xt_q||^2)) had).
//
// One persistent CTA per SM:
//   warp 0      TMA producer: 64-wide K slices of the A (128 rows) and B
//               (256 rows) tiles, 128-byte swizzle, into a 3-stage ring;
//   warp 1      TMEM owner (512 columns = two 128 x 256 fp32 accumulators)
//               and MMA issuer (one thread, tcgen05.mma kind::f16, M=128,
//               N=256, K=16 per instruction);
//   EW epilogue warps (4 or 8): warp w reads TMEM lanes 32 (w % 4) .. +31,
//               so each thread owns one row; with 8 warps two warps share a
//               lane quarter and take 128 columns each (one candidate list
//               per half, written as separate lists).  Each thread filters
//               its distances against its running threshold (the KC-th best
//               so far).  Survivors are appended to a per-row buffer in
//               shared memory; whenever a lane's buffer holds 16 or more, the
//               whole warp merges in step: each lane sorts 32 buffered
//               entries with a bitonic network in registers and
//               bitonic-merges them into its register-resident sorted
//               top-KC, with no divergence.
// The two accumulators let the epilogue of tile t overlap the MMAs of t+1.
// Every mbarrier wait is bounded in time; on a timeout the CTA raises an
// error bit, drains its own copies in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "slk_internal.cuh"

namespace {

// K slice of a stage: 64 bf16 = 128-byte rows (128-byte swizzle), or 32 bf16 =
// 64-byte rows (64-byte swizzle) for twice as many stages in the same bytes.
#ifndef SLK_TC_BK
#define SLK_TC_BK 64
#endif
constexpr int TC_M = 128, TC_N = 256, TC_BK = SLK_TC_BK;
static_assert(TC_BK == 64 || TC_BK == 32, "K slice of 64 or 32 bf16");
constexpr int TC_ROWB = TC_BK * 2;   // bytes per operand row of a stage (= the swizzle span)
#ifndef SLK_TC_STAGES
#define SLK_TC_STAGES 3
#endif
constexpr int TC_STAGES = SLK_TC_STAGES;
// Epilogue warps of the KC = 32 kernel (4 or 8) and its pipelined TMEM loads
// (the KC = 64 kernel keeps 4 warps and single loads: its lists fill the
// registers).
#ifndef SLK_TC_EW32
#define SLK_TC_EW32 4
#endif
#ifndef SLK_TC_PIPE
#define SLK_TC_PIPE 0
#endif
// Epilogue without block barriers per tile (column norms read by 16-byte
// loads from global memory, L1 hits after the first warp), for the KC = 32
// and the KC = 64 kernel; 0 stages the norms in shared memory behind a
// barrier of the epilogue warps per tile (measured faster for KC = 64 at
// D = 128: 552 ms against 797 ms at 1e6 x 128).
#ifndef SLK_TC_NOBAR
#define SLK_TC_NOBAR 1
#endif
#ifndef SLK_TC_NOBAR64
#define SLK_TC_NOBAR64 0
#endif
#ifndef SLK_TC_NOBAR8
#define SLK_TC_NOBAR8 0
#endif
// 8 epilogue warps: 1 keeps the TMEM load of the next 16 columns in flight
// while the current ones are filtered (measured slower at 1e6 x 128: 612
// against 428 ms; the second register set spills around the merges)
#ifndef SLK_TC_PIPE8
#define SLK_TC_PIPE8 0
#endif
// Epilogue warps of the KC = 64 kernel: 4, or 8 (two per SM sub-partition,
// each with half of a row's columns and its own list of 64, 16-column TMEM
// loads; the 10-warp CTA then has 168 registers a thread and spills).
#ifndef SLK_TC_EW64
#define SLK_TC_EW64 4
#endif

// CTA pairs (cta_group::2) for the KC = 32 kernel: the two CTAs of a cluster
// share one 256 x 256 MMA tile, each loading its own 128 A rows and half of
// the B tile, so that an SM takes 32 KiB instead of 48 KiB from L2 per K slice.
#ifndef SLK_TC_PAIR
#define SLK_TC_PAIR 0
#endif
// Folded-norm kernel with 8 epilogue warps: columns per TMEM load (16 or
// 32), pipelined loads (1: the next 16 columns in flight while the current
// ones are filtered, merges only between chunks, 16 entries at a time) and
// the columns per vote group of its narrowing (8 or 4).  Measured at
// 1e6 x 128: 16 columns pipelined 340 ms; unpipelined 357 (32 columns 387,
// vote groups of 4 360); pipelined with full 32-entry merges spilled (422)
#ifndef SLK_TC_AUG_C8
#define SLK_TC_AUG_C8 16
#endif
#ifndef SLK_TC_AUG_PIPE
#define SLK_TC_AUG_PIPE 1
#endif
#ifndef SLK_TC_AUG_G
#define SLK_TC_AUG_G 8
#endif
// Group maxima of the folded-norm epilogue by the three-input max.f32
#ifndef SLK_TC_MAX3
#define SLK_TC_MAX3 1
#endif
// Fraction of the SMs the point-tile kernels run on (1: all; a probe of how
// the operand feed scales: on half the SMs the 1e6 x 128 tiles take 578 ms
// against 293, so their limit is per SM)
#ifndef SLK_TC_GRID_DIV
#define SLK_TC_GRID_DIV 1
#endif
// Sleep between the producer's and the MMA warp's barrier polls (ns; 0:
// poll).  Measured at 1e6 x 128: 100 ns 334 ms, 400 ns 350 ms, polling 329 ms
#ifndef SLK_TC_SPIN_NS
#define SLK_TC_SPIN_NS 0
#endif
// Buffered entries (per lane) that trigger a merge after a tile (KC = 32).
#ifndef SLK_TC_MERGE_AT
#define SLK_TC_MERGE_AT 24
#endif
#ifndef SLK_TC_PAIR_STAGES
#define SLK_TC_PAIR_STAGES 4
#endif
constexpr uint32_t A_BYTES = TC_M * TC_BK * 2;  // 16 KiB (BK = 64)
constexpr uint32_t B_BYTES = TC_N * TC_BK * 2;  // 32 KiB (BK = 64)
// the folded-norm slice: 16 bf16 (32 bytes) per row
constexpr uint32_t AUG_A_BYTES = TC_M * 32;     // 4 KiB
constexpr uint32_t AUG_B_BYTES = TC_N * 32;     // 8 KiB
// the resident A block covers Dp <= 128
constexpr int RES_MAX_DP = 128;

// A vote checks VOTE columns at once and the survivors of APP columns are
// appended to a per-row buffer of BUF slots.  The buffer is merged into the
// sorted list once the tile's accumulator has been released, when some lane
// holds 16 or more; inside a tile only when it could otherwise overflow, so
// that merges rarely hold TMEM while the MMA waits for it.  A 4-stage ring of
// whole B tiles leaves room only for appends of 16 columns and 31 slots; with
// CTA pairs a stage holds half a B tile.
template <int EW, bool PAIR = false, int KC = 32> struct TcEpi {
    static constexpr int stages = PAIR ? SLK_TC_PAIR_STAGES : TC_STAGES;
    static constexpr uint32_t b_bytes = PAIR ? B_BYTES / 2 : B_BYTES;
    static constexpr int halves = EW / 4;             // column halves of a tile
    static constexpr int vote = (EW == 8) ? 16 : 32;  // columns per vote
    // more than 3 x 48 KiB of operand stages leaves room only for 31 slots
    static constexpr bool tight = !PAIR && TC_STAGES * (A_BYTES + B_BYTES) > 3u * 49152u;
    // KC = 64 (an epilogue-bound kernel at small D) merges right away instead,
    // and so do 8 epilogue warps (their two column halves' buffers of 47
    // slots would not fit beside 3 stages)
    static constexpr bool defer = (KC == 32) && !tight && EW == 4;
    static constexpr int app = tight ? 16 : vote;     // columns per append
    static constexpr int buf = defer ? 31 + app : 15 + app;   // buffer slots per row and half
    static constexpr int threads = 64 + 32 * EW;
    // columns per TMEM load: 16 with 8 epilogue warps (the registers of a
    // 10-warp CTA: 168 a thread), else 32
    static constexpr int chunk = (EW == 8) ? 16 : 32;
};
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s
constexpr int kNoIdx = 0x7fffffff;

template <int EW, bool PAIR = false, int KC = 32>
struct TcSmem {
    using E = TcEpi<EW, PAIR, KC>;
    static constexpr int stages = E::stages;
    static constexpr int buf = E::buf;
    uint8_t a[E::stages][A_BYTES];   // 1024-byte aligned stages (swizzle atoms)
    uint8_t b[E::stages][E::b_bytes];
    float buf_d[E::halves][E::buf][TC_M];   // per-row append buffer
    int buf_i[E::halves][E::buf][TC_M];
    float ncol[2][TC_N];             // column norms of the tile in each accumulator
    unsigned long long full[E::stages], empty[E::stages], tfull[2], tempty[2];
    uint32_t tmem_base;
    int abort;
};
template <int EW, bool PAIR = false, int KC = 32>
constexpr size_t tc_smem_bytes() { return sizeof(TcSmem<EW, PAIR, KC>) + 1024; }

// Resident A block for the folded-norm tiles at Dp <= 128 (1) and its ring
// of B slices: with the folded-norm B slices in a ring of their own
// (AUGRING), 8 epilogue warps get STAGES8 B stages and append buffers of BUF
// slots.  Measured at 1e6 x 128: 4 stages with 20 slots 414 ms against 294
// for 3 stages with 31 (the merges that a smaller buffer forces cost more
// than the deeper ring saves), so AUGRING is off by default
#ifndef SLK_TC_RES
#define SLK_TC_RES 1
#endif
#ifndef SLK_TC_RES_AUGRING
#define SLK_TC_RES_AUGRING 0
#endif
#ifndef SLK_TC_RES_STAGES8
#define SLK_TC_RES_STAGES8 4
#endif
#ifndef SLK_TC_RES_BUF
#define SLK_TC_RES_BUF 20
#endif
#ifndef SLK_TC_RES_STAGES
#define SLK_TC_RES_STAGES 3
#endif
// Shared memory of the resident-A form: the row block's A slices (Dp <= 128,
// two of 64 columns) and its folded-norm slice are loaded once per row block
// and stay; the ring carries only B slices, the last slice of a tile with the
// B side of the folded norms.  Per tile the TMA moves 72 KiB instead of 108.
template <int EW>
struct TcSmemRes {
    using E = TcEpi<EW, false, 32>;
    // the tile's folded-norm B slice in a ring of its own (2 slots), which
    // leaves room for a 4th B stage beside append buffers of 20 slots with 8
    // epilogue warps
    static constexpr bool augring = SLK_TC_RES_AUGRING != 0;
    static constexpr int stages = (EW == 8 && augring) ? SLK_TC_RES_STAGES8 : SLK_TC_RES_STAGES;
    static constexpr int buf = (EW == 8 && augring) ? SLK_TC_RES_BUF : E::buf;
    uint8_t a[RES_MAX_DP / TC_BK][A_BYTES];   // 1024-byte aligned (swizzle atoms)
    uint8_t a_aug[AUG_A_BYTES];      // 128 rows x 32 bytes
    uint8_t b[stages][B_BYTES];
    uint8_t b_aug[augring ? 2 : stages][AUG_B_BYTES];
    float buf_d[E::halves][buf][TC_M];
    int buf_i[E::halves][buf][TC_M];
    float ncol[2][TC_N];
    unsigned long long full[stages], empty[stages], tfull[2], tempty[2], afull, aempty;
    unsigned long long augfull[2], augempty[2];
    unsigned long long colbar[8];   // tile column handed from the producer to the epilogue
    int tcol[8];
    uint32_t tmem_base;
    int abort;
};
template <int EW>
constexpr size_t tc_smem_res_bytes() { return sizeof(TcSmemRes<EW>) + 1024; }

// Resident A block with CTA pairs: each CTA of a cluster keeps its own 128
// A rows and receives half of every B slice (128 of the 256 columns) and of
// its folded-norm slice; the pair's MMA (M = 256) reads both halves.  Half
// the B bytes per SM, so the ring holds twice the slices.  Measured at
// 1e6 x 128: 379 ms against 288 for single CTAs (each tile waits for the
// slower of the two epilogues), so it is compiled but off by default.
#ifndef SLK_TC_RESP
#define SLK_TC_RESP 0
#endif
#ifndef SLK_TC_RESP_STAGES
#define SLK_TC_RESP_STAGES 6
#endif
template <int EW>
struct TcSmemResPair {
    using E = TcEpi<EW, true, 32>;
    static constexpr int stages = SLK_TC_RESP_STAGES;
    static constexpr int buf = E::buf;
    uint8_t a[RES_MAX_DP / TC_BK][A_BYTES];
    uint8_t a_aug[AUG_A_BYTES];
    uint8_t b[stages][B_BYTES / 2];      // 128 B rows x 128 bytes
    uint8_t b_aug[stages][AUG_B_BYTES / 2];  // 128 B rows x 32 bytes
    float buf_d[E::halves][E::buf][TC_M];
    int buf_i[E::halves][E::buf][TC_M];
    float ncol[2][TC_N];
    unsigned long long full[stages], empty[stages], tfull[2], tempty[2], afull, aempty;
    unsigned long long colbar[8];
    int tcol[8];
    uint32_t tmem_base;
    int abort;
};
template <int EW>
constexpr size_t tc_smem_resp_bytes() { return sizeof(TcSmemResPair<EW>) + 1024; }

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// the same with cluster-scope acquire (arrivals from the peer CTA)
__device__ __forceinline__ bool mbar_test_cl(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of barrier b.  Gives up (false) after
// kWaitNs or once another role has raised abort.  SLEEP_NS > 0 sleeps
// between polls (the producer and MMA warps, which mostly wait: their polls
// would otherwise take issue slots from the epilogue warps on their SMSPs).
template <bool CL = false, int SLEEP_NS = 0>
__device__ __noinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, volatile int* abort) {
    if (CL ? mbar_test_cl(b, parity) : mbar_test(b, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        if constexpr (SLEEP_NS > 0) __nanosleep(SLEEP_NS);
        if (CL ? mbar_test_cl(b, parity) : mbar_test(b, parity)) return true;
        if (*abort) return false;
        if (globaltimer_ns() - t0 > kWaitNs) {
            *abort = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map,
                                            unsigned long long* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
    d |= (uint64_t)((8 * TC_ROWB) >> 4) << 32;   // SBO: 8-row atoms
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)(TC_ROWB == 128 ? 2 : 4) << 61;   // 128- or 64-byte swizzle
    return d;
}
// max(a, b, c) in one instruction (sm_100 and later)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
// The same for 32-byte swizzle rows (16 bf16): 8-row atoms 256 bytes apart.
__device__ __forceinline__ uint64_t sw32_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((8 * 32) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;   // 32-byte swizzle
    return d;
}
// Instruction descriptor: D fp32, A/B bf16, both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                            ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                     uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(bar))
        : "memory");
}
// CTA-pair forms.  The leader (rank 0 of the cluster) issues the M = 256
// MMAs over both CTAs' A rows and B halves (same shared-memory offsets);
// each CTA's TMEM receives its own 128 rows.  Commits arrive on the barrier
// at the same offset in both CTAs; the loads of both CTAs complete on the
// leader's stage barrier.
constexpr uint32_t kIdescPair = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                                ((uint32_t)((2 * TC_M) >> 4) << 24);
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t mapa_rank(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(su32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cl_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_addr)
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cl,
                                                 int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cl), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdescPair), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit_pair(unsigned long long* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(su32(bar)), "h"((unsigned short)3)
        : "memory");
}

// tcgen05.ld of 32 columns without the wait: the registers are valid only
// after tmem_wait_regs on the same array, which names them as in/out
// operands so that no use can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
template <int C>
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[C]) {
    static_assert(C == 16, "16-column load");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
template <int C>
__device__ __forceinline__ void tmem_wait_regs(uint32_t (&r)[C]) {
    static_assert(C == 16, "16-column wait");
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
          "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
          "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
        :
        : "memory");
}
template <int C>
__device__ __forceinline__ void tmem_ld_issue(uint32_t taddr, uint32_t (&r)[C]) {
    if constexpr (C == 32) tmem_ld32_issue(taddr, r);
    else tmem_ld16_issue<C>(taddr, r);
}
__device__ __forceinline__ void tmem_wait_regs(uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
          "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
          "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]),
          "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]),
          "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]),
          "+r"(r[31])
        :
        : "memory");
}

// Barrier 1 over the NT epilogue threads with an AND of `ok`: every
// epilogue warp gets the same answer, so they all leave their loops together.
template <int NT>
__device__ __forceinline__ bool epilogue_bar_and(bool ok) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r) : "r"(ok ? 1u : 0u), "n"(NT) : "memory");
    return r != 0;
}
template <int NT>
__device__ __forceinline__ void epilogue_bar() {
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// (ad, ai) <-> (bd, bi) so that the pair is ascending (up) or descending,
// ordered by (distance, index).
__device__ __forceinline__ void cas(float& ad, int& ai, float& bd, int& bi, bool up) {
    const bool gt = (ad > bd) || (ad == bd && ai > bi);
    const bool sw = up ? gt : !gt;
    const float td = sw ? bd : ad;
    const int ti = sw ? bi : ai;
    bd = sw ? ad : bd;
    bi = sw ? ai : bi;
    ad = td;
    ai = ti;
}

// Bitonic sort of 32 (distance, index) pairs held in registers, ascending.
__device__ __forceinline__ void bitonic_sort32(float (&d)[32], int (&i)[32]) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int x = 0; x < 32; ++x) {
                const int l = x ^ j;
                if (l > x) cas(d[x], i[x], d[l], i[l], (x & k) == 0);
            }
}

// list (KC entries, sorted ascending) <- the KC smallest of list and b (32
// entries sorted ascending, padded with +inf to KC): the element-wise
// minimum of list and reversed b is bitonic and holds exactly those KC; a
// bitonic merge sorts it.  Only the last 32 slots can take an entry of b.
template <int KC>
__device__ __forceinline__ void merge_topk(float (&ld)[KC], int (&li)[KC], const float (&bd)[32],
                                           const int (&bi)[32]) {
#pragma unroll
    for (int x = KC - 32; x < KC; ++x) {
        const float od = bd[KC - 1 - x];
        const int oi = bi[KC - 1 - x];
        if (od < ld[x] || (od == ld[x] && oi < li[x])) { ld[x] = od; li[x] = oi; }
    }
#pragma unroll
    for (int j = KC / 2; j > 0; j >>= 1)
#pragma unroll
        for (int x = 0; x < KC; ++x) {
            const int l = x ^ j;
            if (l > x) cas(ld[x], li[x], ld[l], li[l], true);
        }
}

// NB (16) entries sorted ascending (bitonic network in registers).
template <int NB>
__device__ __forceinline__ void bitonic_sort_n(float (&d)[NB], int (&i)[NB]) {
#pragma unroll
    for (int k = 2; k <= NB; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int x = 0; x < NB; ++x) {
                const int l = x ^ j;
                if (l > x) cas(d[x], i[x], d[l], i[l], (x & k) == 0);
            }
}

// merge_topk for 16 sorted entries (padded with +inf to KC): only the last 16
// slots of the list can take one of them.
template <int KC>
__device__ __forceinline__ void merge_topk16(float (&ld)[KC], int (&li)[KC], const float (&bd)[16],
                                             const int (&bi)[16]) {
#pragma unroll
    for (int x = KC - 16; x < KC; ++x) {
        const float od = bd[KC - 1 - x];
        const int oi = bi[KC - 1 - x];
        if (od < ld[x] || (od == ld[x] && oi < li[x])) { ld[x] = od; li[x] = oi; }
    }
#pragma unroll
    for (int j = KC / 2; j > 0; j >>= 1)
#pragma unroll
        for (int x = 0; x < KC; ++x) {
            const int l = x ^ j;
            if (l > x) cas(ld[x], li[x], ld[l], li[l], true);
        }
}

// flush_buffer in rounds of 16 entries: half the registers of a 32-entry sort.
template <int KC, class S>
__device__ __forceinline__ void flush_buffer16(S& s, int h, int r, int& cnt,
                                               float (&ld)[KC], int (&li)[KC]) {
    for (int base = 0; __any_sync(0xffffffffu, cnt > base); base += 16) {
        float bd[16];
        int bi[16];
#pragma unroll
        for (int x = 0; x < 16; ++x) {
            const bool have = base + x < cnt;
            bd[x] = have ? s.buf_d[h][base + x][r] : __int_as_float(0x7f800000);
            bi[x] = have ? s.buf_i[h][base + x][r] : kNoIdx;
        }
        bitonic_sort_n<16>(bd, bi);
        merge_topk16<KC>(ld, li, bd, bi);
    }
    cnt = 0;
}

// Warp-synchronous: fold every lane's buffered entries into its top-KC.
template <int KC, class S>
__device__ __forceinline__ void flush_buffer(S& s, int h, int r, int& cnt,
                                             float (&ld)[KC], int (&li)[KC]) {
    for (int base = 0; __any_sync(0xffffffffu, cnt > base); base += 32) {
        float bd[32];
        int bi[32];
#pragma unroll
        for (int x = 0; x < 32; ++x) {
            const bool have = base + x < cnt;
            bd[x] = have ? s.buf_d[h][base + x][r] : __int_as_float(0x7f800000);
            bi[x] = have ? s.buf_i[h][base + x][r] : kNoIdx;
        }
        bitonic_sort32(bd, bi);
        merge_topk<KC>(ld, li, bd, bi);
    }
    cnt = 0;
}

__device__ __forceinline__ void item_range(int item, int splits, int n_tiles, int& rb, int& t0,
                                           int& t1, int& sp) {
    rb = item / splits;
    sp = item % splits;
    t0 = (int)((int64_t)sp * n_tiles / splits);
    t1 = (int)((int64_t)(sp + 1) * n_tiles / splits);
}

// PAIR: launched in clusters of two; an item's row block is a pair of
// 128-row blocks (rank r of the cluster takes block 2 rb + r), both CTAs walk
// the same items, and only the leader's MMA warp issues.
// AUG: one more K slice of 16 columns (32-byte swizzle, one K = 16 MMA)
// from the aug matrix (tmA2 reads its columns 0..15 for the A rows, tmB2 its
// columns 16..31 for the B rows): [1, 1, 1, a_p] against [a_q, 1, 1, 1], a
// the three bfloat16 terms of -||xt||^2 / 2, so that the accumulator holds
// -dt / 2 and the epilogue needs no norms (padding rows and columns carry
// -inf there).
// SPLIT: the two-term operands s = h + l of listed query rows against every
// point.  The accumulator sums three passes over the K slices, h_p . h_q
// (tmA, tmB), h_p . l_q (tmA, tmB2) and l_p . h_q (tmA2, tmB); the rows are
// the first min(*rows_dev, 128 row_blocks) query rows, their norms in
// row_norms (+inf for padding rows); lists go to ((list Np + f) KC), Np
// being the list stride.  Otherwise tmA2 / tmB2 / row_norms / rows_dev are
// unused and the rows are the points themselves.
template <int TC_KC, int EW, bool PIPE, bool NOBAR, bool PAIR = false, bool SPLIT = false,
          bool AUG = false, bool RES = false>
__global__ void __launch_bounds__(TcEpi<EW, PAIR, TC_KC>::threads, 1)
knn_cand_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
                   const float* __restrict__ norms, const float* __restrict__ row_norms,
                   const long long* __restrict__ rows_dev, int64_t N, int64_t Np, int Dp,
                   int n_tiles, int splits, int row_blocks, float* __restrict__ cand_d,
                   int32_t* __restrict__ cand_i, unsigned int* __restrict__ err_flag,
                   unsigned long long* __restrict__ sweep) {
    static_assert(!(SPLIT && PAIR), "split query rows run on single CTAs");
    static_assert(!(AUG && (SPLIT || (PAIR && !RES))), "folded norms: single CTAs, or pairs with a resident A");
    static_assert(!RES || (AUG && TC_KC == 32), "a resident A block goes with the folded norms");
    using E = TcEpi<EW, PAIR, TC_KC>;
    using SMT = std::conditional_t<RES, std::conditional_t<PAIR, TcSmemResPair<EW>, TcSmemRes<EW>>,
                                   TcSmem<EW, PAIR, TC_KC>>;
    constexpr int STAGES = RES ? SMT::stages : E::stages;
    constexpr int BUF = SMT::buf;   // append-buffer slots per row and half
    constexpr bool AUGR = RES && !PAIR && (SLK_TC_RES_AUGRING != 0);   // folded-norm B slices in their own ring
    // bytes of one CTA's B slice (a half with CTA pairs) and of its folded-norm part
    constexpr uint32_t B_SLICE = E::b_bytes;
    constexpr uint32_t B_AUG = PAIR ? AUG_B_BYTES / 2 : AUG_B_BYTES;
    constexpr int H = E::halves, VOTE = E::vote, APP = E::app, NT = 32 * EW;
    // columns per TMEM load (the folded-norm epilogue of 8 warps keeps no
    // second value array, so it has the registers for 32)
    constexpr int C = (AUG && EW == 8) ? SLK_TC_AUG_C8 : E::chunk;
    constexpr int CH_PER_HALF = TC_N / C / H;    // TMEM loads per thread and tile
    extern __shared__ uint8_t smem_raw[];
    SMT& s = *reinterpret_cast<SMT*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb0 = Dp / TC_BK;                   // K slices of one operand pass
    const int nkb = SPLIT ? 3 * nkb0 : (AUG ? nkb0 + 1 : nkb0);   // K slices per tile
    if constexpr (SPLIT) {
        // query rows counted on the device (every thread reads the same value)
        long long rows = *rows_dev;
        const long long cap = (long long)row_blocks * TC_M;
        if (rows > cap) rows = cap;
        if (rows < 0) rows = 0;
        row_blocks = (int)((rows + TC_M - 1) / TC_M);
    }
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;      // CTA or cluster
    const int n_units = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int n_items = (PAIR ? row_blocks / 2 : row_blocks) * splits;
    // each unit takes a contiguous range of items, so consecutive items mostly
    // continue the same row block (the epilogue then keeps its lists going)
    const int item_begin = (int)((int64_t)unit * n_items / n_units);
    const int item_end = (int)((int64_t)(unit + 1) * n_items / n_units);
    volatile int* abort = &s.abort;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&s.full[i], 1);
            mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&s.tfull[i], 1);
            mbar_init(&s.tempty[i], PAIR ? 2 * EW : EW);
        }
        if constexpr (RES) {
            mbar_init(&s.afull, 1);
            mbar_init(&s.aempty, 1);
            for (int i = 0; i < 8; ++i) mbar_init(&s.colbar[i], 1);
        }
        if constexpr (AUGR) {
            for (int i = 0; i < 2; ++i) {
                mbar_init(&s.augfull[i], 1);
                mbar_init(&s.augempty[i], 1);
            }
        }
        s.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             su32(&s.tmem_base)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             su32(&s.tmem_base)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    if constexpr (PAIR) cluster_sync_all();   // barriers and TMEM of both CTAs are ready
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            if constexpr (SPLIT || AUG) {
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA2)) : "memory");
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB2)) : "memory");
            }
            if constexpr (RES) {
                // A slices (and their folded-norm slice) once per row block,
                // after the MMA warp has released the previous block; the ring
                // carries B slices only
                uint32_t iter = 0, aload = 0, tseq = 0;
                bool ok = true;
                int cur_rb = -1;
                for (int item = item_begin; item < item_end && ok; ++item) {
                    int rb, t0, t1, sp;
                    item_range(item, splits, n_tiles, rb, t0, t1, sp);
                    // single CTAs sweep a row block's columns starting where the
                    // other CTAs are (the global count of tiles issued, per CTA,
                    // modulo the range) and wrap around, so that CTAs that drift
                    // apart still read the same B tiles from L2; the candidate
                    // lists do not depend on the order
                    const int nt = t1 - t0;
                    int off = 0;
                    if (!PAIR && sweep != nullptr && nt > 0)
                        off = (int)((*(volatile unsigned long long*)sweep / (unsigned long long)n_units) %
                                    (unsigned long long)nt);
                    if (rb != cur_rb) {
                        if (aload > 0 &&
                            !(ok = mbar_wait<false, SLK_TC_SPIN_NS>(&s.aempty, (aload - 1) & 1, abort)))
                            break;
                        const int arow = (PAIR ? 2 * rb + (int)rank : rb) * TC_M;
                        const uint32_t abytes = (uint32_t)nkb0 * A_BYTES + AUG_A_BYTES;
                        if constexpr (PAIR) {
                            // both CTAs' A loads complete on the leader's barrier
                            const uint32_t abar = mapa_rank(&s.afull, 0);
                            if (rank == 0) mbar_expect_tx(&s.afull, 2 * abytes);
                            for (int kb = 0; kb < nkb0; ++kb)
                                tma_load_2d_pair(s.a[kb], &tmA, abar, kb * TC_BK, arow);
                            tma_load_2d_pair(s.a_aug, &tmA2, abar, 0, arow);
                        } else {
                            mbar_expect_tx(&s.afull, abytes);
                            for (int kb = 0; kb < nkb0; ++kb)
                                tma_load_2d(s.a[kb], &tmA, &s.afull, kb * TC_BK, arow);
                            tma_load_2d(s.a_aug, &tmA2, &s.afull, 0, arow);
                        }
                        ++aload;
                        cur_rb = rb;
                    }
                    for (int i = 0; i < nt && ok; ++i) {
                        const int t = t0 + (off + i) % nt;
                        // the tile's column block for the epilogue (released by the arrival)
                        const uint32_t slot = tseq & 7u;
                        s.tcol[slot] = t;
                        mbar_arrive(&s.colbar[slot]);
                        ++tseq;
                        if (!PAIR && sweep != nullptr && (tseq & 15u) == 0u) atomicAdd(sweep, 16ull);
                        const int bcol = t * TC_N + (int)rank * (TC_N / 2);   // rank 0 unless PAIR
                        if constexpr (AUGR) {
                            // the tile's folded-norm B slice into its own 2-slot ring
                            const uint32_t tix = tseq - 1, as = tix & 1u, ause = tix >> 1;
                            if (ause > 0 &&
                                !(ok = mbar_wait<false, SLK_TC_SPIN_NS>(&s.augempty[as], (ause - 1) & 1, abort)))
                                break;
                            mbar_expect_tx(&s.augfull[as], AUG_B_BYTES);
                            tma_load_2d(s.b_aug[as], &tmB2, &s.augfull[as], 16, bcol);
                        }
                        for (int kb = 0; kb < nkb0; ++kb) {
                            const uint32_t st = iter % STAGES, use = iter / STAGES;
                            if (use > 0 &&
                                !(ok = mbar_wait<false, SLK_TC_SPIN_NS>(&s.empty[st], (use - 1) & 1, abort)))
                                break;
                            const bool last = kb == nkb0 - 1 && !AUGR;
                            const uint32_t bytes = B_SLICE + (last ? B_AUG : 0u);
                            if constexpr (PAIR) {
                                const uint32_t bar = mapa_rank(&s.full[st], 0);
                                if (rank == 0) mbar_expect_tx(&s.full[st], 2 * bytes);
                                tma_load_2d_pair(s.b[st], &tmB, bar, kb * TC_BK, bcol);
                                if (last) tma_load_2d_pair(s.b_aug[st], &tmB2, bar, 16, bcol);
                            } else {
                                mbar_expect_tx(&s.full[st], bytes);
                                tma_load_2d(s.b[st], &tmB, &s.full[st], kb * TC_BK, bcol);
                                if (last) tma_load_2d(s.b_aug[st], &tmB2, &s.full[st], 16, bcol);
                            }
                            ++iter;
                        }
                    }
                }
                // drain: every issued load must have landed before the CTA leaves
                if (!ok || *abort) {
                    if (!PAIR || rank == 0) {
                        const uint32_t first = iter > STAGES ? iter - STAGES : 0;
                        for (uint32_t i = first; i < iter; ++i) {
                            const unsigned long long t0 = globaltimer_ns();
                            while (!mbar_test(&s.full[i % STAGES], (i / STAGES) & 1) &&
                                   globaltimer_ns() - t0 < kWaitNs) {
                            }
                        }
                        if (aload > 0) {
                            const unsigned long long t0 = globaltimer_ns();
                            while (!mbar_test(&s.afull, (aload - 1) & 1) && globaltimer_ns() - t0 < kWaitNs) {
                            }
                        }
                        if constexpr (AUGR) {
                            // the last two folded-norm loads
                            for (uint32_t i = tseq > 2 ? tseq - 2 : 0; i < tseq; ++i) {
                                const unsigned long long t0 = globaltimer_ns();
                                while (!mbar_test(&s.augfull[i & 1u], (i >> 1) & 1u) &&
                                       globaltimer_ns() - t0 < kWaitNs) {
                                }
                            }
                        }
                    } else {
                        // the peer's loads complete on the leader's barriers: give
                        // them time to land (a load takes microseconds)
                        const unsigned long long t0 = globaltimer_ns();
                        while (globaltimer_ns() - t0 < 1000000ull) {
                        }
                    }
                }
            } else {
            uint32_t iter = 0;
            bool ok = true;
            for (int item = item_begin; item < item_end && ok; ++item) {
                int rb, t0, t1, sp;
                item_range(item, splits, n_tiles, rb, t0, t1, sp);
                const int arow = (PAIR ? 2 * rb + (int)rank : rb) * TC_M;
                for (int t = t0; t < t1 && ok; ++t) {
                    const int bcol = t * TC_N + (int)rank * (TC_N / 2);   // rank 0 unless PAIR
                    for (int kb = 0; kb < nkb; ++kb) {
                        const uint32_t st = iter % STAGES, use = iter / STAGES;
                        if (use > 0 && !(ok = mbar_wait<false, SLK_TC_SPIN_NS>(&s.empty[st], (use - 1) & 1, abort))) break;
                        if constexpr (PAIR) {
                            // both CTAs' loads complete on the leader's barrier, whose
                            // one arrival (the leader's) expects the bytes of both
                            const uint32_t bar = mapa_rank(&s.full[st], 0);
                            if (rank == 0) mbar_expect_tx(&s.full[st], 2 * (A_BYTES + E::b_bytes));
                            tma_load_2d_pair(s.a[st], &tmA, bar, kb * TC_BK, arow);
                            tma_load_2d_pair(s.b[st], &tmB, bar, kb * TC_BK, bcol);
                        } else {
                            const CUtensorMap* ma = &tmA;
                            const CUtensorMap* mb = &tmB;
                            int kx = kb;
                            if constexpr (AUG) {
                                if (kb == nkb0) {
                                    // the folded norms: 16 columns of A (x = 0) and B (x = 16)
                                    mbar_expect_tx(&s.full[st], AUG_A_BYTES + AUG_B_BYTES);
                                    tma_load_2d(s.a[st], &tmA2, &s.full[st], 0, arow);
                                    tma_load_2d(s.b[st], &tmB2, &s.full[st], 16, bcol);
                                    ++iter;
                                    continue;
                                }
                            }
                            if constexpr (SPLIT) {
                                // passes h . h, h . l, l . h
                                const int part = kb / nkb0;
                                kx = kb - part * nkb0;
                                if (part == 2) ma = &tmA2;
                                if (part == 1) mb = &tmB2;
                            }
                            mbar_expect_tx(&s.full[st], A_BYTES + B_BYTES);
                            tma_load_2d(s.a[st], ma, &s.full[st], kx * TC_BK, arow);
                            tma_load_2d(s.b[st], mb, &s.full[st], kx * TC_BK, bcol);
                        }
                        ++iter;
                    }
                }
            }
            // drain: every issued load must have landed before the CTA leaves
            if (!ok || *abort) {
                if (!PAIR || rank == 0) {
                    const uint32_t first = iter > STAGES ? iter - STAGES : 0;
                    for (uint32_t i = first; i < iter; ++i) {
                        const unsigned long long t0 = globaltimer_ns();
                        while (!mbar_test(&s.full[i % STAGES], (i / STAGES) & 1) &&
                               globaltimer_ns() - t0 < kWaitNs) {
                        }
                    }
                } else {
                    // the peer's loads complete on the leader's barriers: give
                    // them time to land (a load takes microseconds)
                    const unsigned long long t0 = globaltimer_ns();
                    while (globaltimer_ns() - t0 < 1000000ull) {
                    }
                }
            }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if constexpr (RES) {
            if (lane == 0 && rank == 0) {
                uint32_t iter = 0, tcount = 0, aload = 0;
                bool ok = true;
                int cur_rb = -1;
                for (int item = item_begin; item < item_end && ok; ++item) {
                    int rb, t0, t1, sp;
                    item_range(item, splits, n_tiles, rb, t0, t1, sp);
                    if (rb != cur_rb) {
                        // release the previous block once its MMAs complete, then
                        // wait for the new one
                        if (cur_rb >= 0) {
                            if constexpr (PAIR) umma_commit_pair(&s.aempty);
                            else umma_commit(&s.aempty);
                        }
                        if (!(ok = mbar_wait<false, SLK_TC_SPIN_NS>(&s.afull, aload & 1, abort))) break;
                        tc_fence_after();
                        ++aload;
                        cur_rb = rb;
                    }
                    for (int t = t0; t < t1 && ok; ++t) {
                        const uint32_t acc = tcount & 1, use = tcount >> 1;
                        // with CTA pairs the epilogues of both CTAs release the accumulator
                        if (use > 0 &&
                            !(ok = mbar_wait<PAIR, SLK_TC_SPIN_NS>(&s.tempty[acc], (use - 1) & 1, abort)))
                            break;
                        tc_fence_after();
                        const uint32_t d_tmem = tmem + acc * TC_N;
                        for (int kb = 0; kb < nkb0; ++kb) {
                            const uint32_t st = iter % STAGES;
                            if (!(ok = mbar_wait<false, SLK_TC_SPIN_NS>(&s.full[st], (iter / STAGES) & 1, abort)))
                                break;
                            tc_fence_after();
                            const uint64_t da = sw128_desc(su32(s.a[kb]));
                            const uint64_t db = sw128_desc(su32(s.b[st]));
#pragma unroll
                            for (int k = 0; k < TC_BK / 16; ++k) {
                                if constexpr (PAIR)
                                    umma_pair(d_tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k),
                                              (kb | k) != 0 ? 1u : 0u);
                                else
                                    umma(d_tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k),
                                         (kb | k) != 0 ? 1u : 0u);
                            }
                            if (kb == nkb0 - 1) {   // folded norms: one K = 16 step, 32-byte swizzle
                                if constexpr (AUGR) {
                                    const uint32_t as = tcount & 1u;
                                    if (!(ok = mbar_wait<false, SLK_TC_SPIN_NS>(&s.augfull[as], (tcount >> 1) & 1u,
                                                                                abort)))
                                        break;
                                    tc_fence_after();
                                    umma(d_tmem, sw32_desc(su32(s.a_aug)), sw32_desc(su32(s.b_aug[as])), 1u);
                                    umma_commit(&s.augempty[as]);
                                } else if constexpr (PAIR) {
                                    umma_pair(d_tmem, sw32_desc(su32(s.a_aug)), sw32_desc(su32(s.b_aug[st])), 1u);
                                } else {
                                    umma(d_tmem, sw32_desc(su32(s.a_aug)), sw32_desc(su32(s.b_aug[st])), 1u);
                                }
                            }
                            if constexpr (PAIR) umma_commit_pair(&s.empty[st]);
                            else umma_commit(&s.empty[st]);
                            ++iter;
                        }
                        if (!ok) break;
                        if constexpr (PAIR) umma_commit_pair(&s.tfull[acc]);
                        else umma_commit(&s.tfull[acc]);
                        ++tcount;
                    }
                }
                if (!ok || *abort) {
                    // let the MMAs already issued finish before TMEM is released
                    if (iter > 0) {
                        const uint32_t i = iter - 1;
                        const unsigned long long t0 = globaltimer_ns();
                        while (!mbar_test(&s.empty[i % STAGES], (i / STAGES) & 1) &&
                               globaltimer_ns() - t0 < kWaitNs) {
                        }
                    }
                }
            }
        } else if (lane == 0 && rank == 0) {
            uint32_t iter = 0, tcount = 0;
            bool ok = true;
            for (int item = item_begin; item < item_end && ok; ++item) {
                int rb, t0, t1, sp;
                item_range(item, splits, n_tiles, rb, t0, t1, sp);
                for (int t = t0; t < t1 && ok; ++t) {
                    const uint32_t acc = tcount & 1, use = tcount >> 1;
                    // with CTA pairs the epilogues of both CTAs release the accumulator
                    if (use > 0 && !(ok = mbar_wait<PAIR, SLK_TC_SPIN_NS>(&s.tempty[acc], (use - 1) & 1, abort))) break;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + acc * TC_N;
                    for (int kb = 0; kb < nkb; ++kb) {
                        const uint32_t st = iter % STAGES;
                        if (!(ok = mbar_wait<false, SLK_TC_SPIN_NS>(&s.full[st], (iter / STAGES) & 1, abort))) break;
                        tc_fence_after();
                        if (AUG && kb == nkb0) {
                            // folded norms: one K = 16 step in 32-byte swizzle rows
                            const uint64_t da = sw32_desc(su32(s.a[st]));
                            const uint64_t db = sw32_desc(su32(s.b[st]));
                            umma(d_tmem, da, db, 1u);
                            umma_commit(&s.empty[st]);
                            ++iter;
                            continue;
                        }
                        const uint64_t da = sw128_desc(su32(s.a[st]));
                        const uint64_t db = sw128_desc(su32(s.b[st]));
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k) {   // 32-byte steps inside the swizzle row
                            if constexpr (PAIR)
                                umma_pair(d_tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k),
                                          (kb | k) != 0 ? 1u : 0u);
                            else
                                umma(d_tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k),
                                     (kb | k) != 0 ? 1u : 0u);
                        }
                        if constexpr (PAIR) umma_commit_pair(&s.empty[st]);
                        else umma_commit(&s.empty[st]);
                        ++iter;
                    }
                    if (!ok) break;
                    if constexpr (PAIR) umma_commit_pair(&s.tfull[acc]);
                    else umma_commit(&s.tfull[acc]);
                    ++tcount;
                }
            }
            if (!ok || *abort) {
                // let the MMAs already issued finish before TMEM is released
                if (iter > 0) {
                    const uint32_t i = iter - 1;
                    const unsigned long long t0 = globaltimer_ns();
                    while (!mbar_test(&s.empty[i % STAGES], (i / STAGES) & 1) &&
                           globaltimer_ns() - t0 < kWaitNs) {
                    }
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int sub = warp & 3;
        const int r = sub * 32 + lane;
        const int et = threadIdx.x - 64;  // 0..NT-1 among the epilogue threads
        const int h = et / 128;           // column half of this thread (EW == 8)
        uint32_t tcount = 0;
        bool ok = true;
        float ld[TC_KC];
        int li[TC_KC];
        int cnt = 0;
        int run_rb = -1, run_sp = 0;   // the row block whose list is being built
        bool hit = false;              // a chunk appended since the last room check (warp-uniform)
        for (int item = item_begin; item < item_end && ok; ++item) {
            int rb, t0, t1, sp;
            item_range(item, splits, n_tiles, rb, t0, t1, sp);
            const int64_t p = (int64_t)(PAIR ? 2 * rb + (int)rank : rb) * TC_M + r;
            if (rb != run_rb) {
                // a new row block: the list restarts (the previous one was written)
#pragma unroll
                for (int x = 0; x < TC_KC; ++x) {
                    ld[x] = __int_as_float(0x7f800000);
                    li[x] = kNoIdx;
                }
                cnt = 0;
                run_rb = rb;
                run_sp = sp;
            } else {
                // this split continues the run: its own slot stays empty
                const int64_t o = ((int64_t)(sp * H + h) * Np + p) * TC_KC;
#pragma unroll
                for (int x = 0; x < TC_KC; ++x) {
                    cand_d[o + x] = __int_as_float(0x7f800000);
                    cand_i[o + x] = -1;
                }
            }
            // padding rows / columns get an infinite norm: their distances never pass
            const float np_ = SPLIT ? row_norms[p] : ((p < N) ? norms[p] : __int_as_float(0x7f800000));
            for (int t = t0; t < t1; ++t) {
                const uint32_t acc = tcount & 1, use = tcount >> 1;
                int tc = t;
                if constexpr (RES) {
                    // the producer's sweep order: the tile's column block from its ring
                    const uint32_t slot = tcount & 7u;
                    ok = mbar_wait(&s.colbar[slot], (tcount >> 3) & 1u, abort);
                    if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                    tc = s.tcol[slot];
                }
                const int64_t col0 = (int64_t)tc * TC_N;
                // NOBAR: column norms straight from global memory (uniform
                // addresses, L1 hits after the first warp; padding rows hold an
                // infinite norm), each warp waits for the accumulator on its own
                const float* ncol_g = norms + col0;
                if constexpr (NOBAR || AUG) {
                    ok = mbar_wait(&s.tfull[acc], use & 1, abort);
                    if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                } else {
                    for (int c = et; c < TC_N; c += NT)
                        s.ncol[acc][c] = (col0 + c < N) ? norms[col0 + c] : __int_as_float(0x7f800000);
                    epilogue_bar<NT>();
                    ok = epilogue_bar_and<NT>(mbar_wait(&s.tfull[acc], use & 1, abort));
                    if (!ok) break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(sub * 32) << 16) + acc * TC_N;
                // distances of one 32-column chunk, filtered in votes of VOTE
                // columns against the row's threshold (the row's own column,
                // distance ~0, is kept here and dropped by the rerank)
                // AUG, pipelined loads: appends only (the caller flushes at
                // chunk boundaries, keeping room for C appends, and only after a
                // chunk with a hit: `hit` is set by the warp-uniform vote)
                constexpr bool AUG_PIPE = AUG && (SLK_TC_AUG_PIPE != 0);
                auto process_aug = [&](const uint32_t (&rv)[C], int ch) {
                    // the accumulator holds -dt / 2: a column passes when it
                    // exceeds -thr / 2 (dt < thr; both scalings exact); padding
                    // rows and columns hold -inf and never pass.  Votes narrow
                    // down by groups of G columns, each group's maximum by a tree.
                    constexpr int G = SLK_TC_AUG_G;
#pragma unroll
                    for (int g0 = 0; g0 < C; g0 += VOTE) {
                        const float hthr = -0.5f * ld[TC_KC - 1];
                        float mg[VOTE / G];
#pragma unroll
                        for (int q = 0; q < VOTE / G; ++q) {
                            float t[G];
#pragma unroll
                            for (int j = 0; j < G; ++j) t[j] = __uint_as_float(rv[g0 + G * q + j]);
                            if constexpr (G == 8 && SLK_TC_MAX3) {
                                // three-input maximum: 4 instructions, depth 2
                                const float u0 = fmax3(t[0], t[1], t[2]);
                                const float u1 = fmax3(t[3], t[4], t[5]);
                                mg[q] = fmax3(u0, u1, fmaxf(t[6], t[7]));
                            } else {
#pragma unroll
                                for (int w = G / 2; w > 0; w >>= 1)
#pragma unroll
                                    for (int j = 0; j < w; ++j) t[j] = fmaxf(t[j], t[j + w]);
                                mg[q] = t[0];
                            }
                        }
                        float mx = mg[0];
#pragma unroll
                        for (int q = 1; q < VOTE / G; ++q) mx = fmaxf(mx, mg[q]);
                        if (__any_sync(0xffffffffu, mx > hthr)) {
                            hit = true;
#pragma unroll
                            for (int a0 = 0; a0 < VOTE; a0 += APP) {
                                if constexpr (E::defer && !AUG_PIPE) {
                                    if (__any_sync(0xffffffffu, cnt > E::buf - APP))
                                        flush_buffer<TC_KC>(s, h, r, cnt, ld, li);
                                }
#pragma unroll
                                for (int q = a0 / G; q < (a0 + APP) / G; ++q) {
                                    if (!__any_sync(0xffffffffu, mg[q] > hthr)) continue;
#pragma unroll
                                    for (int j = g0 + G * q; j < g0 + G * q + G; ++j) {
                                        const float a = __uint_as_float(rv[j]);
                                        if (a > hthr) {
                                            s.buf_d[h][cnt][r] = -2.f * a;
                                            s.buf_i[h][cnt][r] = (int)(col0 + ch * C + j);
                                            ++cnt;
                                        }
                                    }
                                }
                                if constexpr (!E::defer && !AUG_PIPE) {
                                    if (__any_sync(0xffffffffu, cnt >= 16))
                                        flush_buffer<TC_KC>(s, h, r, cnt, ld, li);
                                }
                            }
                        }
                    }
                };
                auto process = [&](const uint32_t (&rv)[C], int ch) {
                    if constexpr (AUG) {
                        process_aug(rv, ch);
                        return;
                    }
                    float v[C];   // w = fl(||xt_q||^2 - 2 dot)
                    if constexpr (NOBAR) {
                        const float4* n4 = reinterpret_cast<const float4*>(ncol_g + ch * C);
#pragma unroll
                        for (int q = 0; q < C / 4; ++q) {
                            const float4 c4 = __ldg(n4 + q);
                            v[4 * q + 0] = fmaf(-2.f, __uint_as_float(rv[4 * q + 0]), c4.x);
                            v[4 * q + 1] = fmaf(-2.f, __uint_as_float(rv[4 * q + 1]), c4.y);
                            v[4 * q + 2] = fmaf(-2.f, __uint_as_float(rv[4 * q + 2]), c4.z);
                            v[4 * q + 3] = fmaf(-2.f, __uint_as_float(rv[4 * q + 3]), c4.w);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < C; ++j)
                            v[j] = fmaf(-2.f, __uint_as_float(rv[j]), s.ncol[acc][ch * C + j]);
                    }
#pragma unroll
                    for (int g0 = 0; g0 < C; g0 += VOTE) {
                        // w < thr - ||xt_p||^2 (rounded up) whenever dt < thr; a
                        // padding row (infinite norm) gets NaN and never passes
                        const float thr_w = __fsub_ru(ld[TC_KC - 1], np_);
                        float m8[VOTE / 8];
#pragma unroll
                        for (int q = 0; q < VOTE / 8; ++q) {
                            m8[q] = v[g0 + 8 * q];
#pragma unroll
                            for (int j = 1; j < 8; ++j) m8[q] = fminf(m8[q], v[g0 + 8 * q + j]);
                        }
                        float mn = m8[0];
#pragma unroll
                        for (int q = 1; q < VOTE / 8; ++q) mn = fminf(mn, m8[q]);
                        // some row of the warp may have a distance below its threshold:
                        // narrow down by groups of 8 columns (warp-uniform branches),
                        // then append per lane
                        if (__any_sync(0xffffffffu, mn < thr_w)) {
#pragma unroll
                            for (int a0 = 0; a0 < VOTE; a0 += APP) {
                                // room for APP more entries
                                if constexpr (E::defer) {
                                    if (__any_sync(0xffffffffu, cnt > E::buf - APP))
                                        flush_buffer<TC_KC>(s, h, r, cnt, ld, li);
                                }
#pragma unroll
                                for (int q = a0 / 8; q < (a0 + APP) / 8; ++q) {
                                    if (!__any_sync(0xffffffffu, m8[q] < thr_w)) continue;
#pragma unroll
                                    for (int j = g0 + 8 * q; j < g0 + 8 * q + 8; ++j) {
                                        if (v[j] < thr_w) {
                                            s.buf_d[h][cnt][r] = __fadd_rn(v[j], np_);
                                            s.buf_i[h][cnt][r] = (int)(col0 + ch * C + j);
                                            ++cnt;
                                        }
                                    }
                                }
                                if constexpr (!E::defer) {
                                    // merge right away (the threshold only drops: the stale
                                    // one lets through entries the next merge discards)
                                    if (__any_sync(0xffffffffu, cnt >= 16))
                                        flush_buffer<TC_KC>(s, h, r, cnt, ld, li);
                                }
                            }
                        }
                    }
                };
                auto release = [&]() {   // this warp's last TMEM read of the tile is done
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if constexpr (PAIR) mbar_arrive_remote(mapa_rank(&s.tempty[acc], 0));
                        else mbar_arrive(&s.tempty[acc]);
                    }
                };
                const int ch0 = h * CH_PER_HALF;
                if constexpr (AUG_PIPE) {
                    // the load of the next chunk is in flight while one is
                    // filtered; merges happen only at chunk boundaries, with one
                    // chunk's values live, keeping room for C appends
                    static_assert(BUF >= C, "room for a chunk's appends");
                    uint32_t ra[C], rb2[C];
                    tmem_ld_issue<C>(tbase + ch0 * C, ra);
#pragma unroll 1
                    for (int cc = 0; cc < CH_PER_HALF; cc += 2) {
                        tmem_wait_regs(ra);
                        if (hit) {
                            hit = false;
                            if (__any_sync(0xffffffffu, cnt > BUF - C)) flush_buffer16<TC_KC>(s, h, r, cnt, ld, li);
                        }
                        tmem_ld_issue<C>(tbase + (ch0 + cc + 1) * C, rb2);
                        process(ra, ch0 + cc);
                        tmem_wait_regs(rb2);
                        if (cc + 2 >= CH_PER_HALF) release();
                        if (hit) {
                            hit = false;
                            if (__any_sync(0xffffffffu, cnt > BUF - C)) flush_buffer16<TC_KC>(s, h, r, cnt, ld, li);
                        }
                        if (cc + 2 < CH_PER_HALF) tmem_ld_issue<C>(tbase + (ch0 + cc + 2) * C, ra);
                        process(rb2, ch0 + cc + 1);
                    }
                } else if constexpr (PIPE) {
                // two register sets: the load of chunk c + 1 is in flight while
                // chunk c is filtered
                uint32_t ra[C], rb2[C];
                tmem_ld_issue<C>(tbase + ch0 * C, ra);
                tmem_wait_regs(ra);
#pragma unroll 1
                for (int cc = 0; cc < CH_PER_HALF; cc += 2) {
                    tmem_ld_issue<C>(tbase + (ch0 + cc + 1) * C, rb2);
                    process(ra, ch0 + cc);
                    tmem_wait_regs(rb2);
                    if (cc + 2 < CH_PER_HALF) tmem_ld_issue<C>(tbase + (ch0 + cc + 2) * C, ra);
                    else release();
                    process(rb2, ch0 + cc + 1);
                    if (cc + 2 < CH_PER_HALF) tmem_wait_regs(ra);
                }
                } else {
#pragma unroll 1
                for (int cc = 0; cc < CH_PER_HALF; ++cc) {
                    uint32_t rv[C];
                    tmem_ld_issue(tbase + (ch0 + cc) * C, rv);
                    tmem_wait_regs(rv);
                    if (cc == CH_PER_HALF - 1) release();
                    process(rv, ch0 + cc);
                }
                }
                // merge with the accumulator released (the threshold only drops,
                // so the stale one let through entries the merge discards)
                if constexpr (E::defer) {
                    if (__any_sync(0xffffffffu, cnt >= SLK_TC_MERGE_AT)) flush_buffer<TC_KC>(s, h, r, cnt, ld, li);
                }
                ++tcount;
            }
            if (!ok) break;
            // write the run's list when the next item starts another row block
            int next_rb = -1;
            if (item + 1 < item_end) {
                int t0n, t1n, spn;
                item_range(item + 1, splits, n_tiles, next_rb, t0n, t1n, spn);
            }
            if (next_rb != rb) {
                flush_buffer<TC_KC>(s, h, r, cnt, ld, li);
                const int64_t o = ((int64_t)(run_sp * H + h) * Np + p) * TC_KC;
#pragma unroll
                for (int x = 0; x < TC_KC; ++x) {
                    cand_d[o + x] = ld[x];
                    cand_i[o + x] = (li[x] == kNoIdx) ? -1 : li[x];
                }
            }
        }
    }

    tc_fence_before();
    // with CTA pairs neither CTA leaves while the other may still reach its
    // shared memory (remote arrivals, commits, loads) or TMEM
    if constexpr (PAIR) cluster_sync_all();
    else __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(TMEM_COLS)
                         : "memory");
    }
    if (threadIdx.x == 0 && s.abort) atomicOr(err_flag, 2u);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

constexpr CUtensorMapSwizzle kTcSwizzle =
    TC_ROWB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

}  // namespace

int knn_tc_tile_cols() { return TC_N; }

// Candidate lists one split of the tensor-core kernel writes per row: two
// column halves with 8 epilogue warps (KC = 32), one with 4 (KC = 64, whose
// lists need the registers of a 6-warp CTA).
int knn_tc_lists_per_split(int kc, int ew) {
    (void)kc;
    return ew / 4;
}

slk_status knn_cand_bf16_launch(slk_ctx* ctx, const __nv_bfloat16* xt, const float* norms,
                                const __nv_bfloat16* aug, int64_t N, int Dp, int64_t Np, int kc,
                                int ew, int splits, float* cand_d, int32_t* cand_i,
                                unsigned int* err_flag, unsigned long long* sweep) {
    if (kc != 32 && kc != 64) return set_err(ctx, SLK_ERR_INVALID_ARG, "bf16 candidates need KC=32 or 64");
    if (ew != 4 && ew != 8) return set_err(ctx, SLK_ERR_INVALID_ARG, "4 or 8 epilogue warps");
    if (Dp % TC_BK != 0 || Np % TC_M != 0)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "bad padded shape %lld x %d", (long long)Np, Dp);
    if ((reinterpret_cast<uintptr_t>(xt) & 15) != 0)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "bf16 operand not 16-byte aligned");
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_err(ctx, SLK_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    CUtensorMap ta, tb;
    const cuuint64_t dims[2] = {(cuuint64_t)Dp, (cuuint64_t)Np};
    const cuuint64_t strides[1] = {(cuuint64_t)Dp * 2};
    const cuuint32_t box_a[2] = {TC_BK, TC_M};
    const cuuint32_t box_b[2] = {TC_BK, TC_N};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r1 = enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)xt, dims, strides, box_a, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, kTcSwizzle,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)xt, dims, strides, box_b, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, kTcSwizzle,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
        return set_err(ctx, SLK_ERR_CUDA, "tensor map encoding failed (%d, %d)", (int)r1, (int)r2);
    // folded norms: the aug matrix (Np x 32 bf16), 16-column boxes in 32-byte swizzle
    CUtensorMap ta2 = ta, tb2a = tb;
    const bool use_aug = aug != nullptr && kc == 32 && !(SLK_TC_PAIR != 0 && (Np / TC_M) % 2 == 0);
    if (use_aug) {
        if ((reinterpret_cast<uintptr_t>(aug) & 15) != 0)
            return set_err(ctx, SLK_ERR_INVALID_ARG, "aug operand not 16-byte aligned");
        const cuuint64_t adims[2] = {32, (cuuint64_t)Np};
        const cuuint64_t astr[1] = {64};
        const cuuint32_t abox_a[2] = {16, TC_M};
        const cuuint32_t abox_b[2] = {16, TC_N};
        CUresult r3 = enc(&ta2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)aug, adims, astr, abox_a,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        CUresult r4 = enc(&tb2a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)aug, adims, astr, abox_b,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r3 != CUDA_SUCCESS || r4 != CUDA_SUCCESS)
            return set_err(ctx, SLK_ERR_CUDA, "tensor map encoding failed (%d, %d)", (int)r3, (int)r4);
    }
    const int row_blocks = (int)(Np / TC_M);
    const int n_tiles = (int)((Np + TC_N - 1) / TC_N);
    const int n_items = row_blocks * splits;
    // a resident A block pays a pipeline drain per row block: only for long
    // sweeps (the batched form's small graphs have items of a few tiles)
    const bool res_ok = SLK_TC_RES != 0 && Dp <= RES_MAX_DP && n_tiles / splits >= 64;
    int grid = ctx->num_sms / SLK_TC_GRID_DIV;
    if (grid > n_items) grid = n_items;
    if (kc == 32 && SLK_TC_PAIR != 0 && row_blocks % 2 == 0) {
        // CTA pairs: clusters of two over 256-row blocks, B tiles in halves
        CUtensorMap tb2;
        const cuuint32_t box_b2[2] = {TC_BK, TC_N / 2};
        CUresult r3 = enc(&tb2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)xt, dims, strides, box_b2,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, kTcSwizzle,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r3 != CUDA_SUCCESS)
            return set_err(ctx, SLK_ERR_CUDA, "tensor map encoding failed (%d)", (int)r3);
        auto kern = knn_cand_tc_kernel<32, 4, false, true, true>;
        const size_t smem = tc_smem_bytes<4, true>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        const int pair_items = (row_blocks / 2) * splits;
        int clusters = ctx->num_sms / 2;
        if (clusters > pair_items) clusters = pair_items;
        if (clusters < 1) clusters = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * clusters));
        cfg.blockDim = dim3(TcEpi<4, true>::threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = ctx->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        SLK_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, kern, ta, tb2, ta, tb2, norms, norms,
                                             (const long long*)nullptr, N, Np, Dp, n_tiles, splits,
                                             row_blocks, cand_d, cand_i, err_flag,
                                             (unsigned long long*)nullptr));
    } else if (use_aug && res_ok && SLK_TC_RESP != 0 && ew == 8 &&
               row_blocks % 2 == 0) {
        // resident A block with CTA pairs: clusters of two over 256-row blocks,
        // B slices and their folded-norm part in halves
        CUtensorMap tbh, tb2h;
        const cuuint32_t box_bh[2] = {TC_BK, TC_N / 2};
        CUresult r5 = enc(&tbh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)xt, dims, strides, box_bh,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, kTcSwizzle,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        const cuuint64_t adims[2] = {32, (cuuint64_t)Np};
        const cuuint64_t astr[1] = {64};
        const cuuint32_t abox_bh[2] = {16, TC_N / 2};
        CUresult r6 = enc(&tb2h, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)aug, adims, astr, abox_bh,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r5 != CUDA_SUCCESS || r6 != CUDA_SUCCESS)
            return set_err(ctx, SLK_ERR_CUDA, "tensor map encoding failed (%d, %d)", (int)r5, (int)r6);
        auto kern = knn_cand_tc_kernel<32, 8, false, false, true, false, true, true>;
        const size_t smem = tc_smem_resp_bytes<8>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        const int pair_items = (row_blocks / 2) * splits;
        int clusters = ctx->num_sms / 2;
        if (clusters > pair_items) clusters = pair_items;
        if (clusters < 1) clusters = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * clusters));
        cfg.blockDim = dim3(TcEpi<8, true>::threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = ctx->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        SLK_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, kern, ta, tbh, ta2, tb2h, norms, norms,
                                             (const long long*)nullptr, N, Np, Dp, n_tiles, splits,
                                             row_blocks, cand_d, cand_i, err_flag,
                                             (unsigned long long*)nullptr));
    } else if (use_aug && res_ok) {
        // resident A block (Dp <= 128)
        if (ew == 4) {
            auto kern = knn_cand_tc_kernel<32, 4, false, false, false, false, true, true>;
            const size_t smem = tc_smem_res_bytes<4>();
            SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem));
            kern<<<grid, TcEpi<4>::threads, smem, ctx->stream>>>(
                ta, tb, ta2, tb2a, norms, norms, nullptr, N, Np, Dp, n_tiles, splits, row_blocks,
                cand_d, cand_i, err_flag, sweep);
        } else {
            auto kern = knn_cand_tc_kernel<32, 8, false, false, false, false, true, true>;
            const size_t smem = tc_smem_res_bytes<8>();
            SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem));
            kern<<<grid, TcEpi<8>::threads, smem, ctx->stream>>>(
                ta, tb, ta2, tb2a, norms, norms, nullptr, N, Np, Dp, n_tiles, splits, row_blocks,
                cand_d, cand_i, err_flag, sweep);
        }
    } else if (use_aug && ew == 4) {
        auto kern = knn_cand_tc_kernel<32, 4, false, false, false, false, true>;
        const size_t smem = tc_smem_bytes<4>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        kern<<<grid, TcEpi<4>::threads, smem, ctx->stream>>>(
            ta, tb, ta2, tb2a, norms, norms, nullptr, N, Np, Dp, n_tiles, splits, row_blocks, cand_d,
            cand_i, err_flag, nullptr);
    } else if (use_aug) {
        auto kern = knn_cand_tc_kernel<32, 8, false, false, false, false, true>;
        const size_t smem = tc_smem_bytes<8>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        kern<<<grid, TcEpi<8>::threads, smem, ctx->stream>>>(
            ta, tb, ta2, tb2a, norms, norms, nullptr, N, Np, Dp, n_tiles, splits, row_blocks, cand_d,
            cand_i, err_flag, nullptr);
    } else if (kc == 32 && ew == 4) {
        auto kern = knn_cand_tc_kernel<32, 4, SLK_TC_PIPE != 0, SLK_TC_NOBAR != 0>;
        const size_t smem = tc_smem_bytes<4>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        kern<<<grid, TcEpi<4>::threads, smem, ctx->stream>>>(
            ta, tb, ta, tb, norms, norms, nullptr, N, Np, Dp, n_tiles, splits, row_blocks, cand_d,
            cand_i, err_flag, nullptr);
    } else if (kc == 32) {
        // 8 epilogue warps: the column norms staged in shared memory (measured
        // faster here than per-warp global loads: 426 against 469 ms at 1e6 x 128)
        auto kern = knn_cand_tc_kernel<32, 8, SLK_TC_PIPE8 != 0, SLK_TC_NOBAR8 != 0>;
        const size_t smem = tc_smem_bytes<8>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        kern<<<grid, TcEpi<8>::threads, smem, ctx->stream>>>(
            ta, tb, ta, tb, norms, norms, nullptr, N, Np, Dp, n_tiles, splits, row_blocks, cand_d,
            cand_i, err_flag, nullptr);
    } else {
        constexpr int EW = SLK_TC_EW64;
        auto kern = knn_cand_tc_kernel<64, EW, false, SLK_TC_NOBAR64 != 0>;
        const size_t smem = tc_smem_bytes<EW, false, 64>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        kern<<<grid, TcEpi<EW, false, 64>::threads, smem, ctx->stream>>>(
            ta, tb, ta, tb, norms, norms, nullptr, N, Np, Dp, n_tiles, splits, row_blocks, cand_d,
            cand_i, err_flag, nullptr);
    }
    SLK_LAUNCH_CHECK(ctx, "knn_cand_tc_kernel");
    return SLK_OK;
}

// Two-term bfloat16 tiles of listed query rows (see the SPLIT form of the
// kernel): A operands qh / ql (Fcap rows, Fcap a multiple of 128), B operands
// xh / xl (Np rows, a multiple of 256), both Dp columns; the number of
// query rows is read on the device from *rows_dev (at most Fcap are taken),
// so the launch does not wait for the stage before it.  Lists of KC = 32,
// ew / 4 per split, at ((list Fcap + f) 32).
slk_status knn_cand_split_launch(slk_ctx* ctx, const __nv_bfloat16* qh, const __nv_bfloat16* ql,
                                 const float* qnorm, int64_t Fcap, const long long* rows_dev,
                                 const __nv_bfloat16* xh, const __nv_bfloat16* xl,
                                 const float* norms, int64_t N, int Dp, int64_t Np, int ew,
                                 int splits, float* cand_d, int32_t* cand_i,
                                 unsigned int* err_flag) {
    if (ew != 4 && ew != 8) return set_err(ctx, SLK_ERR_INVALID_ARG, "4 or 8 epilogue warps");
    if (Dp % TC_BK != 0 || Np % TC_N != 0 || Fcap % TC_M != 0 || Fcap <= 0)
        return set_err(ctx, SLK_ERR_INVALID_ARG, "bad padded shape %lld / %lld x %d", (long long)Fcap,
                       (long long)Np, Dp);
    const void* ptrs[4] = {qh, ql, xh, xl};
    for (const void* q : ptrs)
        if ((reinterpret_cast<uintptr_t>(q) & 15) != 0)
            return set_err(ctx, SLK_ERR_INVALID_ARG, "bf16 operand not 16-byte aligned");
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_err(ctx, SLK_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    CUtensorMap maps[4];
    const cuuint64_t strides[1] = {(cuuint64_t)Dp * 2};
    const cuuint32_t estr[2] = {1, 1};
    for (int m = 0; m < 4; ++m) {
        const bool a = m < 2;
        const cuuint64_t dims[2] = {(cuuint64_t)Dp, (cuuint64_t)(a ? Fcap : Np)};
        const cuuint32_t box[2] = {TC_BK, (cuuint32_t)(a ? TC_M : TC_N)};
        const CUresult r = enc(&maps[m], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptrs[m]),
                               dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, kTcSwizzle,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return set_err(ctx, SLK_ERR_CUDA, "tensor map encoding failed (%d)", (int)r);
    }
    const int row_cap_blocks = (int)(Fcap / TC_M);
    const int n_tiles = (int)(Np / TC_N);
    const int grid = ctx->num_sms > 0 ? ctx->num_sms : 148;   // persistent: items are counted on the device
    if (ew == 4) {
        auto kern = knn_cand_tc_kernel<32, 4, SLK_TC_PIPE != 0, SLK_TC_NOBAR != 0, false, true>;
        const size_t smem = tc_smem_bytes<4>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        kern<<<grid, TcEpi<4>::threads, smem, ctx->stream>>>(
            maps[0], maps[2], maps[1], maps[3], norms, qnorm, rows_dev, N, Fcap, Dp, n_tiles, splits,
            row_cap_blocks, cand_d, cand_i, err_flag, nullptr);
    } else {
        auto kern = knn_cand_tc_kernel<32, 8, SLK_TC_PIPE8 != 0, SLK_TC_NOBAR8 != 0, false, true>;
        const size_t smem = tc_smem_bytes<8>();
        SLK_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        kern<<<grid, TcEpi<8>::threads, smem, ctx->stream>>>(
            maps[0], maps[2], maps[1], maps[3], norms, qnorm, rows_dev, N, Fcap, Dp, n_tiles, splits,
            row_cap_blocks, cand_d, cand_i, err_flag, nullptr);
    }
    SLK_LAUNCH_CHECK(ctx, "knn_cand_tc_kernel (split query rows)");
    return SLK_OK;
}
