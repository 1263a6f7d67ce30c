// Share matrix x table mod 2^32 on the fifth-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), exactly: the product of the
// unfused baseline (paper Sec. 3.1: the B x L share matrix times the L x W
// table as one matrix-matrix product; Sec. 3.2.2) for batches that make it a dense contraction.
//
//   out[b][w] += sum_{k < K} S[b][k] * T[k][w]   (mod 2^32)
//
// Exactness.  Every u32 x is split into four signed 8-bit limbs,
// x = sum_i s_i 2^{8i} (mod 2^32) with s_i in [-128, 127]: the bytes y_i of
// y = x + 0x80808080 (mod 2^32) give s_i = y_i - 128.  These limbs are exact
// in fp16, and so is every limb product (|s_i t_j| <= 2^14).  Mod 2^32 the
// product keeps the ten limb products with i + j <= 3, in four shift classes
// d = i + j; class d accumulates in fp32 in tensor memory, where every partial
// sum is an integer of magnitude at most (d + 1) * 2^14 * 256 <= 2^24 over 256
// values of k, so no partial sum is rounded.  After every 256 values of k the
// classes are drained into u32 totals (sum_d class_d << 8d) and restart from
// zero.  (sm_103a has no integer kind of tcgen05.mma, hence fp16 limbs.)
//
// One CTA per (128-query x TN-word output tile, k slice), 13 warps:
//  - warps 5-12 load 64 values of k of the S tile (128 x 64 u32) and the T
//    tile (64 x TN u32), split them into fp16 limb planes and store the
//    planes in shared memory in the 128-byte-swizzled K-major layout the
//    tensor core reads; two stages with full/empty mbarriers;
//  - one lane of warp 4 issues a stage's 16 tcgen05.mma (M = 128, K = 16;
//    A = limb plane i of S, B = limb planes 0..3-i of T side by side, N =
//    (4 - i) TN, into classes i..3) and frees the stage with tcgen05.commit;
//  - warps 0-3 (TMEM lanes 0-127, one per query row of the tile) drain one
//    accumulator set with tcgen05.ld while the MMAs fill the other.
// Split-k partial tiles meet in out with u32 atomics (order-independent, so
// bit-exact).  Every wait is bounded: one that gives up records
// PIR_FAULT_WAIT_TIMEOUT and the CTA winds down (it waits, bounded, for its
// own MMAs, then frees its tensor memory).
//
// That is the kernel for operands of any alignment.  For 16-byte-aligned ones
// (S and T on 16-byte boundaries, ld and stride multiples of 4) a second
// kernel, further down, has one more warp bring the raw tiles in by
// tensor-map copies and the conversion warps read them from shared memory;
// it is the one launched unless PIR_TC_TENSOR_MAPS=0 is in the environment.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "internal.h"

namespace pir {
namespace dev {
namespace {

constexpr uint32_t kTcM = 128;              // queries per tile = TMEM lanes = MMA M
constexpr uint32_t kTcStageK = 64;          // k per stage: one 128-byte row of fp16 per operand row
constexpr uint32_t kTcStages = 2;
constexpr uint32_t kTcStagesPerChunk = 4;   // 256 k between drains (the exactness bound above)
constexpr uint32_t kTcChunkK = kTcStageK * kTcStagesPerChunk;
constexpr uint32_t kTcDrainWarps = 4;       // warps 0-3
constexpr uint32_t kTcMmaWarp = 4;          // allocates TMEM; its lane 0 issues the MMAs
constexpr uint32_t kTcConvWarps = 8;        // warps 5-12
constexpr uint32_t kTcConvThreads = 32 * kTcConvWarps;
constexpr uint32_t kTcThreads = 32 * (kTcDrainWarps + 1 + kTcConvWarps);
constexpr uint32_t kTcPlaneA = kTcM * 128;  // bytes of one limb plane of the S tile
constexpr uint32_t kTcHeader = 1024;        // mbarriers, TMEM address, abort flag
constexpr uint32_t kTcSpinLimit = 1u << 22; // polls per bounded wait (each try_wait may also suspend)


// header offsets (bytes from the 1024-aligned base)
constexpr uint32_t kTcFull = 0, kTcEmpty = kTcFull + 8 * kTcStages, kTcAccFull = kTcEmpty + 8 * kTcStages,
                   kTcAccEmpty = kTcAccFull + 16, kTcDone = kTcAccEmpty + 16;
constexpr uint32_t kTcTmemSlot = kTcDone + 8, kTcAbort = kTcTmemSlot + 4;
static_assert(kTcAbort + 4 <= kTcHeader, "header");

template <int TN>
struct TcShape {
    static_assert(TN == 32 || TN == 64, "tile width");
    static constexpr uint32_t kPlaneB = TN * 128;  // bytes of one limb plane of the T tile
    static constexpr uint32_t kStageBytes = 4 * kTcPlaneA + 4 * kPlaneB;
    static constexpr uint32_t kSmem = 1024 /* alignment slack */ + kTcHeader + kTcStages * kStageBytes;
    static constexpr uint32_t kTmemCols = 2 * 4 * TN;  // two accumulator sets of four classes
    // instruction descriptor of kind::f16 for an MMA of N = nplanes * TN: D f32
    // (bits 4-5 = 1), A and B f16 (bits 7-9, 10-12 = 0), both K-major (bits 15,
    // 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
    __host__ __device__ static constexpr uint32_t idesc(uint32_t nplanes) {
        return (1u << 4) | ((nplanes * (uint32_t)TN >> 3) << 17) | ((kTcM >> 4) << 24);
    }
    static_assert(kSmem <= 227u * 1024u, "shared memory");
    static_assert(kTmemCols >= 32 && kTmemCols <= 512 && (kTmemCols & (kTmemCols - 1)) == 0, "TMEM columns");
    static_assert(kPlaneB % 1024 == 0 && kTcPlaneA % 1024 == 0 && kTcHeader % 1024 == 0, "swizzle atoms");
};

struct TcParams {
    const uint32_t* S;
    uint64_t ld;
    const uint32_t* T;
    uint64_t stride;
    uint64_t K;
    uint64_t nchunks;  // 256-value accumulator chunks of k in all: ceil(K / 256)
    uint32_t cpc;      // chunks per CTA: CTA x takes chunks x * cpc .. x * cpc + cpc - 1
    uint32_t* out;
    uint32_t* faults;  // the library's device fault word
    uint32_t B, W;
    uint32_t vec;  // S and T 16-byte aligned, ld and stride multiples of 4
};

extern __shared__ char tc_sm[];

__device__ __forceinline__ uint32_t sm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `bar` with the given parity.  Gives up when
// another role of the CTA has given up (abort flag), or after kTcSpinLimit
// polls, recording the fault and raising the flag.
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, volatile uint32_t* abort_flag,
                                          uint32_t* faults) {
    for (uint32_t i = 0; i < kTcSpinLimit; ++i) {
        if (try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    atomicOr(faults, PIR_FAULT_WAIT_TIMEOUT);
    *abort_flag = 1u;
    return false;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// ---- tcgen05 -----------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand in 128-byte swizzle atoms
// (8 rows x 128 bytes, 1024-byte aligned): start address >> 4 at bits 0-13,
// leading byte offset (unused with this swizzle) 16 >> 4 at bits 16-29,
// stride byte offset between 8-row groups 1024 >> 4 at bits 32-45, descriptor
// version 1 at bits 46-47, swizzle mode 128B (2) at bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on `bar` once every tcgen05 operation this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- limb planes -------------------------------------------------------------
__device__ __forceinline__ uint32_t sub1152(uint32_t h) {  // (1024 + y) - 1152 = y - 128, per fp16 half, exact
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(h), "r"(0x64806480u));
    return r;
}

// Four consecutive values of k of one operand row -> for each limb plane p,
// the four fp16 limbs s_p of those values (8 bytes, lowest k first).  A
// half with bits 0x64yy is 1024 + yy.
__device__ __forceinline__ void limbs4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, uint2 (&pl)[4]) {
    const uint32_t y0 = x0 + 0x80808080u, y1 = x1 + 0x80808080u, y2 = x2 + 0x80808080u, y3 = x3 + 0x80808080u;
    const uint32_t a_lo = __byte_perm(y0, y1, 0x5140u), a_hi = __byte_perm(y0, y1, 0x7362u);
    const uint32_t b_lo = __byte_perm(y2, y3, 0x5140u), b_hi = __byte_perm(y2, y3, 0x7362u);
    constexpr uint32_t C = 0x64646464u;
    pl[0] = make_uint2(sub1152(__byte_perm(a_lo, C, 0x4140u)), sub1152(__byte_perm(b_lo, C, 0x4140u)));
    pl[1] = make_uint2(sub1152(__byte_perm(a_lo, C, 0x4342u)), sub1152(__byte_perm(b_lo, C, 0x4342u)));
    pl[2] = make_uint2(sub1152(__byte_perm(a_hi, C, 0x4140u)), sub1152(__byte_perm(b_hi, C, 0x4140u)));
    pl[3] = make_uint2(sub1152(__byte_perm(a_hi, C, 0x4342u)), sub1152(__byte_perm(b_hi, C, 0x4342u)));
}

// byte offset of (row r, k quad q) in a 128-byte-swizzled K-major plane: the
// 16-byte chunk q / 2 of row r moves to chunk (q / 2) ^ (r % 8)
__device__ __forceinline__ uint32_t sw128_off(uint32_t r, uint32_t q) {
    return r * 128u + ((((q >> 1) ^ (r & 7u)) << 4) | ((q & 1u) << 3));
}

__device__ __forceinline__ void sts64(uint32_t addr, uint2 v) {
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(v.x), "r"(v.y) : "memory");
}

// Four consecutive words from p, of which the first `nvalid` exist (the rest
// read as 0).  kStream: evict-first loads (the share matrix is read once).
template <bool kStream>
__device__ __forceinline__ uint4 load4(const uint32_t* p, uint32_t nvalid, uint32_t vec) {
    if (vec && nvalid >= 4)
        return kStream ? __ldcs(reinterpret_cast<const uint4*>(p)) : __ldg(reinterpret_cast<const uint4*>(p));
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (nvalid > 0) v.x = __ldg(p);
    if (nvalid > 1) v.y = __ldg(p + 1);
    if (nvalid > 2) v.z = __ldg(p + 2);
    if (nvalid > 3) v.w = __ldg(p + 3);
    return v;
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int w) {
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

template <int TN>
__global__ void __launch_bounds__(kTcThreads, 1) contract_tc_kernel(const TcParams p) {
    using Sh = TcShape<TN>;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t raw = sm_u32(tc_sm);
    const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms are 1024-byte aligned
    char* const gbase = tc_sm + (base - raw);
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(gbase + kTcAbort);
    const uint32_t m0 = blockIdx.y * kTcM, n0 = blockIdx.z * (uint32_t)TN;
    // this CTA's chunks of k: a run of at most cpc from cfirst; only the last
    // chunk of all (k up to K) can be partial
    const uint64_t cfirst = (uint64_t)blockIdx.x * p.cpc;
    const uint32_t nch = (uint32_t)(p.nchunks - cfirst < p.cpc ? p.nchunks - cfirst : p.cpc);
    const uint64_t klast = p.K - (cfirst + nch - 1) * kTcChunkK;
    const uint32_t nst = (nch - 1) * kTcStagesPerChunk +
                         (klast >= kTcChunkK ? kTcStagesPerChunk : (uint32_t)((klast + kTcStageK - 1) / kTcStageK));
    const uint64_t kend = p.K;
    // first k of local stage g
    auto stage_k = [&](uint32_t g) -> uint64_t { return cfirst * kTcChunkK + (uint64_t)g * kTcStageK; };

    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < kTcStages; ++s) {
            mbar_init(base + kTcFull + 8u * s, kTcConvThreads);
            mbar_init(base + kTcEmpty + 8u * s, 1u);
        }
        for (uint32_t b = 0; b < 2; ++b) {
            mbar_init(base + kTcAccFull + 8u * b, 1u);
            mbar_init(base + kTcAccEmpty + 8u * b, 32u * kTcDrainWarps);
        }
        mbar_init(base + kTcDone, 1u);
        *abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTcMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + kTcTmemSlot),
                     "r"(Sh::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + kTcTmemSlot);

    if (warp > kTcMmaWarp) {
        // ---- conversion warps: u32 tiles -> fp16 limb planes -------------------
        // S tile: thread -> k quad q of rows it*16 + cw*2 + lane/16 (it < 8).
        // Half a warp covers one 128-byte plane row: conflict-free 8-byte stores.
        // T tile: thread -> k quad qt (rows 4 qt .. 4 qt + 3) of words 4 n4 ..
        // 4 n4 + 3; a warp takes 8 word quads x 4 k quads, so each load
        // instruction reads four whole 128-byte lines.  Its plane rows n = 4 n4 +
        // w are written in the order w = (j + rot) % 4, rot = (n4 / 2) % 4: the
        // eight n4 of a warp then land on eight different 16-byte chunks of the
        // swizzle, and each 8-byte store takes the minimum two wavefronts.
        const uint32_t ct = threadIdx.x - 32u * (kTcMmaWarp + 1), cw = ct >> 5;
        const uint32_t q = lane & 15u;
        constexpr uint32_t kN8 = (uint32_t)TN / 32u;  // blocks of 8 word quads across the tile
        const uint32_t n4 = (cw % kN8) * 8u + (lane & 7u), qt = (cw / kN8) * 4u + (lane >> 3);
        const bool has_b = qt < kTcStageK / 4u;
        const uint32_t rot = (n4 >> 1) & 3u;
        const uint32_t nw = n0 + 4u * n4;
        const uint32_t wval = has_b && nw < p.W ? min(4u, p.W - nw) : 0u;
        // stage g's share words (S tile) and table words (T tile), into registers
        auto load_a = [&](uint32_t g, uint4 (&a)[8]) {
            const uint64_t kq = stage_k(g) + 4u * q;
            const uint32_t kval = kq < kend ? (uint32_t)(kend - kq < 4u ? kend - kq : 4u) : 0u;
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const uint32_t m = m0 + it * 16u + cw * 2u + (lane >> 4);
                a[it] = load4<true>(p.S + (uint64_t)m * p.ld + kq, m < p.B ? kval : 0u, p.vec);
            }
        };
        auto load_t = [&](uint32_t g, uint4 (&t)[4]) {
            const uint64_t kq = stage_k(g) + 4u * qt;
            const uint32_t kval = kq < kend ? (uint32_t)(kend - kq < 4u ? kend - kq : 4u) : 0u;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                t[e] = load4<false>(p.T + (kq + e) * p.stride + nw, e < (int)kval ? wval : 0u, p.vec);
        };
        // stage g's words -> limb planes in shared-memory stage g % 2
        auto convert_stage = [&](uint32_t g, const uint4 (&a)[8], const uint4 (&t)[4]) -> bool {
            const uint32_t s = g & 1u;
            if (!wait_bounded(base + kTcEmpty + 8u * s, ((g >> 1) & 1u) ^ 1u, abort_flag, p.faults)) return false;
            const uint32_t stage = base + kTcHeader + s * Sh::kStageBytes;
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                uint2 pl[4];
                limbs4(a[it].x, a[it].y, a[it].z, a[it].w, pl);
                const uint32_t off = sw128_off(it * 16u + cw * 2u + (lane >> 4), q);
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) sts64(stage + pp * kTcPlaneA + off, pl[pp]);
            }
            if (has_b) {
                uint4 u[4];  // u[e] word j = t[e] word (j + rot) % 4
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    u[e] = t[e];
                    if (rot & 1u) u[e] = make_uint4(u[e].y, u[e].z, u[e].w, u[e].x);
                    if (rot & 2u) u[e] = make_uint4(u[e].z, u[e].w, u[e].x, u[e].y);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint2 pl[4];
                    limbs4(word_of(u[0], j), word_of(u[1], j), word_of(u[2], j), word_of(u[3], j), pl);
                    const uint32_t off = sw128_off(4u * n4 + ((j + rot) & 3u), qt);
#pragma unroll
                    for (int pp = 0; pp < 4; ++pp) sts64(stage + 4u * kTcPlaneA + pp * Sh::kPlaneB + off, pl[pp]);
                }
            }
            // the tensor core reads the planes through the async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(base + kTcFull + 8u * s);
            return true;
        };
        if constexpr (TN == 64) {
            // Two stages' loads in flight: stage g + 1's are issued before stage
            // g is converted (and before the wait for a free shared-memory
            // stage, the MMAs of two stages back).  (Measured: 0.414 -> 0.403 ms
            // at 256 x 2^20 x 64; slower with 32-word tiles, which keep one.)
            uint4 a[8], t[4];
            if (nst) {
                load_a(0, a);
                load_t(0, t);
            }
            for (uint32_t g = 0; g < nst; ++g) {
                uint4 an[8], tn[4];
                if (g + 1 < nst) {
                    load_a(g + 1, an);
                    load_t(g + 1, tn);
                }
                if (!convert_stage(g, a, t)) break;
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = an[i];
#pragma unroll
                for (int i = 0; i < 4; ++i) t[i] = tn[i];
            }
        } else {
            // a stage's loads are in flight while the warp waits for a free
            // shared-memory stage (the MMAs of two stages back)
            for (uint32_t g = 0; g < nst; ++g) {
                uint4 a[8], t[4];
                load_a(g, a);
                load_t(g, t);
                if (!convert_stage(g, a, t)) break;
            }
        }
    } else if (warp == kTcMmaWarp) {
        // ---- MMA issue: 4 k-steps x 10 limb pairs per stage ------------------
        if (lane == 0) {
            for (uint32_t g = 0; g < nst; ++g) {
                const uint32_t s = g & 1u, c = g / kTcStagesPerChunk, b = c & 1u;
                const bool first = g % kTcStagesPerChunk == 0;
                const bool last = g % kTcStagesPerChunk == kTcStagesPerChunk - 1 || g + 1 == nst;
                if (first && !wait_bounded(base + kTcAccEmpty + 8u * b, ((c >> 1) & 1u) ^ 1u, abort_flag, p.faults))
                    break;
                if (!wait_bounded(base + kTcFull + 8u * s, (g >> 1) & 1u, abort_flag, p.faults)) break;
                tc_fence_after();
                const uint32_t stage = base + kTcHeader + s * Sh::kStageBytes;
                // Limb plane i of S times limb planes 0..3-i of T lands in classes
                // i..3: the T planes lie back to back in the stage (N = TN per
                // plane) and the classes side by side in tensor memory, so one
                // MMA of N = (4 - i) TN does all of them (4 MMAs per k-step).
                const uint64_t bd0 = sw128_desc(stage + 4u * kTcPlaneA);
#pragma unroll
                for (uint32_t t = 0; t < kTcStageK / 16; ++t) {
#pragma unroll
                    for (uint32_t i = 0; i < 4; ++i) {
                        const uint64_t ad = sw128_desc(stage + i * kTcPlaneA) + 2u * t;  // + 32 bytes per k-step
                        // the chunk's first MMA (i = 0, first k-step) overwrites every class
                        mma_f16(tmem + (b * 4u + i) * (uint32_t)TN, ad, bd0 + 2u * t, Sh::idesc(4u - i),
                                (first && t == 0 && i == 0) ? 0u : 1u);
                    }
                }
                mma_commit(base + kTcEmpty + 8u * s);
                if (last) mma_commit(base + kTcAccFull + 8u * b);
            }
            // every MMA issued completes before the tensor memory is freed (bounded)
            mma_commit(base + kTcDone);
            bool done = false;
            for (uint32_t i = 0; i < kTcSpinLimit && !done; ++i) done = try_wait(base + kTcDone, 0u);
            if (!done) atomicOr(p.faults, PIR_FAULT_WAIT_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ---- drain warps: class accumulators -> u32 totals of this lane's row --
        uint32_t total[TN];
#pragma unroll
        for (int n = 0; n < TN; ++n) total[n] = 0u;
        const uint32_t lane_addr = tmem + ((warp * 32u) << 16);
        bool ok = true;
        for (uint32_t c = 0; c < nch; ++c) {
            const uint32_t b = c & 1u;
            // tcgen05.ld is warp-collective: the lanes agree on whether to go on
            ok = __all_sync(0xffffffffu, wait_bounded(base + kTcAccFull + 8u * b, (c >> 1) & 1u, abort_flag, p.faults));
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (uint32_t d = 0; d < 4; ++d) {
#pragma unroll
                for (uint32_t h = 0; h < (uint32_t)TN / 32u; ++h) {
                    uint32_t r[32];
                    tmem_ld32(lane_addr + (b * 4u + d) * (uint32_t)TN + h * 32u, r);
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        total[h * 32 + e] += (uint32_t)__float2int_rn(__uint_as_float(r[e])) << (8u * d);
                }
            }
            tc_fence_before();
            mbar_arrive(base + kTcAccEmpty + 8u * b);
        }
        const uint32_t m = m0 + warp * 32u + lane;
        if (ok && m < p.B) {
#pragma unroll
            for (int n = 0; n < TN; ++n)
                if (n0 + n < p.W && total[n]) atomicAdd(p.out + (uint64_t)m * p.W + n0 + n, total[n]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kTcMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::kTmemCols)
                     : "memory");
    }
}

// ---- raw tiles by the tensor memory accelerator ------------------------------
// The same product and pipeline for 16-byte-aligned operands, but the S and T
// tiles arrive in shared memory through 2-D tensor-map copies
// (cp.async.bulk.tensor), which fill zeros past the batch, the rows and the
// width.  The conversion warps' global loads cost the load/store pipe one
// wavefront per 32-byte sector; reading the copied words back from shared
// memory costs one per 128 bytes.  The limb planes now hold 32 values of k per
// stage in the 64-byte-swizzled K-major layout, so that two plane stages and
// four raw stages fit the CTA's shared memory.
// Warps: 0-3 drain, 4 issues the MMAs, 5 issues the copies, 6-13 convert.
constexpr uint32_t kT2StageK = 32;
constexpr uint32_t kT2StagesPerChunk = kTcChunkK / kT2StageK;  // 8
constexpr uint32_t kT2PlaneA = kTcM * 64;                        // one S limb plane: 128 rows x 64 B
constexpr uint32_t kT2RawA = kTcM * kT2StageK * 4;               // raw S tile: 128 rows x 32 words
constexpr uint32_t kT2TmaWarp = 5;
constexpr uint32_t kT2ConvWarp0 = 6;
constexpr uint32_t kT2Threads = 32 * (kT2ConvWarp0 + kTcConvWarps);

template <int TN>
struct Tc2Shape {
    // Limb-plane and raw stages: three of each fit with 64-word tiles (a
    // conversion may then run up to two stages ahead of the MMAs; two plane
    // stages or two raw stages measured slower).  32-word tiles have room for
    // a fourth plane stage (measured 2 % faster than a fourth raw stage).
    static constexpr uint32_t kPlaneStages = TN == 64 ? 3 : 4;
    static constexpr uint32_t kRawStages = 3;
    // header offsets (bytes from the 1024-aligned base): one 8-byte mbarrier per stage and role
    static constexpr uint32_t kRawFull = 0, kRawEmpty = kRawFull + 8 * kRawStages,
                              kPlFull = kRawEmpty + 8 * kRawStages, kPlEmpty = kPlFull + 8 * kPlaneStages,
                              kAccFull = kPlEmpty + 8 * kPlaneStages, kAccEmpty = kAccFull + 16,
                              kDone = kAccEmpty + 16, kTmemSlot = kDone + 8, kAbort = kTmemSlot + 4;
    static_assert(kAbort + 4 <= kTcHeader, "header");
    static constexpr uint32_t kPlaneB = TN * 64;           // one T limb plane: TN rows x 64 B
    static constexpr uint32_t kPlaneStage = 4 * kT2PlaneA + 4 * kPlaneB;
    static constexpr uint32_t kRawT = kT2StageK * TN * 4;  // raw T tile: 32 rows of k x TN words
    static constexpr uint32_t kRawStage = kT2RawA + kRawT;
    static constexpr uint32_t kPlanesOff = kTcHeader;
    static constexpr uint32_t kRawOff = kPlanesOff + kPlaneStages * kPlaneStage;
    static constexpr uint32_t kSmem = 1024 /* alignment slack */ + kRawOff + kRawStages * kRawStage;
    static_assert(kSmem <= 227u * 1024u, "shared memory");
    static_assert(kPlaneStage % 1024 == 0 && kRawStage % 1024 == 0 && kT2PlaneA % 1024 == 0 &&
                      kPlaneB % 512 == 0 && kT2RawA % 1024 == 0,
                  "stage and swizzle-atom alignment");
};

// Shared-memory matrix descriptor: K-major operand in 64-byte swizzle atoms
// (8 rows x 64 bytes, 512-byte aligned): start address >> 4 at bits 0-13,
// leading byte offset (unused with this swizzle) 16 >> 4 at bits 16-29,
// stride byte offset between 8-row groups 512 >> 4 at bits 32-45, descriptor
// version 1 at bits 46-47, swizzle mode 64B (4) at bits 61-63.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// byte offset of (row r, k quad q) in a 64-byte-swizzled K-major plane: the
// 16-byte chunk q / 2 of row r moves to chunk (q / 2) ^ ((r / 2) % 4)
__device__ __forceinline__ uint32_t sw64_off(uint32_t r, uint32_t q) {
    return r * 64u + ((((q >> 1) ^ ((r >> 1) & 3u)) << 4) | ((q & 1u) << 3));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 2-D tensor-map copy of the box at (x, y) (x innermost, in elements) into
// shared memory, its bytes counted on `bar`
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int32_t x, int32_t y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

template <int TN>
__global__ void __launch_bounds__(kT2Threads, 1)
    contract_tc2_kernel(const __grid_constant__ CUtensorMap tmap_s, const __grid_constant__ CUtensorMap tmap_t,
                        const TcParams p) {
    using Sh = TcShape<TN>;
    using S2 = Tc2Shape<TN>;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t raw = sm_u32(tc_sm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    char* const gbase = tc_sm + (base - raw);
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(gbase + S2::kAbort);
    const uint32_t m0 = blockIdx.y * kTcM, n0 = blockIdx.z * (uint32_t)TN;
    const uint64_t cfirst = (uint64_t)blockIdx.x * p.cpc;
    const uint32_t nch = (uint32_t)(p.nchunks - cfirst < p.cpc ? p.nchunks - cfirst : p.cpc);
    const uint64_t klast = p.K - (cfirst + nch - 1) * kTcChunkK;
    const uint32_t nst = (nch - 1) * kT2StagesPerChunk +
                         (klast >= kTcChunkK ? kT2StagesPerChunk : (uint32_t)((klast + kT2StageK - 1) / kT2StageK));
    auto plane_stage = [&](uint32_t pq) { return base + S2::kPlanesOff + pq * S2::kPlaneStage; };
    auto raw_stage = [&](uint32_t r) { return base + S2::kRawOff + r * S2::kRawStage; };

    if (threadIdx.x == 0) {
        for (uint32_t r = 0; r < S2::kRawStages; ++r) {
            mbar_init(base + S2::kRawFull + 8u * r, 1u);            // the copying lane's arrival + the bytes
            mbar_init(base + S2::kRawEmpty + 8u * r, kTcConvWarps);  // one arrival per conversion warp
        }
        for (uint32_t pq = 0; pq < S2::kPlaneStages; ++pq) {
            mbar_init(base + S2::kPlFull + 8u * pq, kTcConvThreads);
            mbar_init(base + S2::kPlEmpty + 8u * pq, 1u);
        }
        for (uint32_t b = 0; b < 2; ++b) {
            mbar_init(base + S2::kAccFull + 8u * b, 1u);
            mbar_init(base + S2::kAccEmpty + 8u * b, 32u * kTcDrainWarps);
        }
        mbar_init(base + S2::kDone, 1u);
        *abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTcMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + S2::kTmemSlot),
                     "r"(Sh::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp == kT2TmaWarp && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_s)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_t)) : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + S2::kTmemSlot);

    if (warp >= kT2ConvWarp0) {
        // ---- conversion warps: raw words in shared memory -> fp16 limb planes ----
        // S tile [128 rows][32 words]: thread -> k quad q = ct % 8 of rows it * 32 + ct / 8, so a
        // warp reads four whole 128-byte rows and writes four whole 64-byte plane rows.
        // T tile [32 rows of k][TN words]: thread -> k quad qt (rows 4 qt .. 4 qt + 3) of words
        // 4 n4 .. 4 n4 + 3; a warp takes 8 word quads x 4 k quads (four 128-byte reads per
        // instruction) and writes its plane rows n = 4 n4 + w in the order w = (j + rot) % 4,
        // rot = (n4 / 2) % 4, which puts the eight n4 on eight different (64-byte half,
        // 16-byte chunk) places of the swizzle: two wavefronts per 8-byte store.
        const uint32_t ct = threadIdx.x - 32u * kT2ConvWarp0, cw = ct >> 5;
        const uint32_t q = ct & 7u, rs = ct >> 3;
        constexpr uint32_t kN8 = (uint32_t)TN / 32u;
        const uint32_t n4 = (cw % kN8) * 8u + (lane & 7u), qt = (cw / kN8) * 4u + (lane >> 3);
        const bool has_t = qt < kT2StageK / 4u;
        const uint32_t rot = (n4 >> 1) & 3u;
        // Query rows past the batch are zeros in every stage: their plane rows are
        // cleared once here (ordered before the tensor core's first read by the first
        // stage's proxy fence) and never converted.
        const uint32_t rows_valid = p.B - m0 < kTcM ? p.B - m0 : kTcM;
        if (rows_valid < kTcM) {
            for (uint32_t pq = 0; pq < S2::kPlaneStages; ++pq)
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const uint32_t row = (uint32_t)it * 32u + rs;
                    if (row >= rows_valid)
#pragma unroll
                        for (int pp = 0; pp < 4; ++pp)
                            sts64(plane_stage(pq) + pp * kT2PlaneA + sw64_off(row, q), make_uint2(0u, 0u));
                }
        }
        // The loop, compiled once for a full tile (no row checks: they cost a full
        // tile 8 % when present) and once for a tile with rows past the batch.
        auto convert_all = [&](auto full) {
            constexpr bool kFull = decltype(full)::value;
            for (uint32_t g = 0; g < nst; ++g) {
                const uint32_t r = g % S2::kRawStages, pq = g % S2::kPlaneStages;
                // warp-uniform waits: the lanes meet in __syncwarp below
                if (!__all_sync(0xffffffffu, wait_bounded(base + S2::kRawFull + 8u * r, (g / S2::kRawStages) & 1u,
                                                          abort_flag, p.faults)))
                    break;
                const char* rawp = gbase + (raw_stage(r) - base);
                uint4 a[4], u[4];
#pragma unroll
                for (int it = 0; it < 4; ++it)
                    if (kFull || (uint32_t)it * 32u + rs < rows_valid)
                        a[it] = *reinterpret_cast<const uint4*>(rawp + ((uint32_t)it * 32u + rs) * (kT2StageK * 4u) +
                                                                q * 16u);
                if (has_t) {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        u[e] = *reinterpret_cast<const uint4*>(rawp + kT2RawA + (4u * qt + e) * ((uint32_t)TN * 4u) +
                                                               n4 * 16u);
                }
                if (!__all_sync(0xffffffffu, wait_bounded(base + S2::kPlEmpty + 8u * pq,
                                                          ((g / S2::kPlaneStages) & 1u) ^ 1u, abort_flag, p.faults)))
                    break;
                const uint32_t plane = plane_stage(pq);
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    if (!kFull && (uint32_t)it * 32u + rs >= rows_valid) continue;
                    uint2 pl[4];
                    limbs4(a[it].x, a[it].y, a[it].z, a[it].w, pl);
                    const uint32_t off = sw64_off((uint32_t)it * 32u + rs, q);
#pragma unroll
                    for (int pp = 0; pp < 4; ++pp) sts64(plane + pp * kT2PlaneA + off, pl[pp]);
                }
                if (has_t) {
                    // u[e] = words 4 n4 .. of k row 4 qt + e, rotated: word j = word (j + rot) % 4
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (rot & 1u) u[e] = make_uint4(u[e].y, u[e].z, u[e].w, u[e].x);
                        if (rot & 2u) u[e] = make_uint4(u[e].z, u[e].w, u[e].x, u[e].y);
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        uint2 pl[4];
                        limbs4(word_of(u[0], j), word_of(u[1], j), word_of(u[2], j), word_of(u[3], j), pl);
                        const uint32_t off = sw64_off(4u * n4 + ((j + rot) & 3u), qt);
#pragma unroll
                        for (int pp = 0; pp < 4; ++pp) sts64(plane + 4u * kT2PlaneA + pp * S2::kPlaneB + off, pl[pp]);
                    }
                }
                // The tensor core reads the planes, and the next copy into the raw stage writes,
                // through the async proxy: one fence orders this thread's plane stores and raw
                // reads before both.  (Releasing the raw stage before the conversion, with its own
                // fence, measured slower; without that fence the copy overwrote words not yet read.)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(base + S2::kPlFull + 8u * pq);
                __syncwarp();
                if (lane == 0) mbar_arrive(base + S2::kRawEmpty + 8u * r);  // one arrival per warp
            }
        };
        if (rows_valid == kTcM)
            convert_all(std::true_type{});
        else
            convert_all(std::false_type{});
    } else if (warp == kT2TmaWarp) {
        // ---- copies: raw stage g % 4 once every conversion warp released it ------
        if (lane == 0) {
            uint32_t issued = 0;
            for (uint32_t g = 0; g < nst; ++g) {
                const uint32_t r = g % S2::kRawStages;
                if (g >= S2::kRawStages &&
                    !wait_bounded(base + S2::kRawEmpty + 8u * r, ((g / S2::kRawStages) - 1u) & 1u, abort_flag, p.faults))
                    break;
                const uint32_t bar = base + S2::kRawFull + 8u * r, dst = raw_stage(r);
                mbar_expect_tx(bar, S2::kRawStage);  // whole boxes: the zeros past the edges count too
                const int32_t k0 = (int32_t)(cfirst * kTcChunkK + (uint64_t)g * kT2StageK);
                tma_load_2d(dst, &tmap_s, k0, (int32_t)m0, bar);
                tma_load_2d(dst + kT2RawA, &tmap_t, (int32_t)n0, k0, bar);
                issued = g + 1;
            }
            // The last copy into each raw stage has landed before the CTA exits (bounded):
            // its phase is that stage's last, so a completed one reads as complete.
            for (uint32_t g = issued > S2::kRawStages ? issued - S2::kRawStages : 0u; g < issued; ++g) {
                bool done = false;
                for (uint32_t i = 0; i < kTcSpinLimit && !done; ++i)
                    done = try_wait(base + S2::kRawFull + 8u * (g % S2::kRawStages), (g / S2::kRawStages) & 1u);
                if (!done) atomicOr(p.faults, PIR_FAULT_WAIT_TIMEOUT);
            }
        }
        __syncwarp();
    } else if (warp == kTcMmaWarp) {
        // ---- MMA issue: 2 k-steps x 4 MMAs (N = (4 - i) TN) per stage -------------
        if (lane == 0) {
            for (uint32_t g = 0; g < nst; ++g) {
                const uint32_t pq = g % S2::kPlaneStages, c = g / kT2StagesPerChunk, b = c & 1u;
                const bool first = g % kT2StagesPerChunk == 0;
                const bool last = g % kT2StagesPerChunk == kT2StagesPerChunk - 1 || g + 1 == nst;
                if (first && !wait_bounded(base + S2::kAccEmpty + 8u * b, ((c >> 1) & 1u) ^ 1u, abort_flag, p.faults))
                    break;
                if (!wait_bounded(base + S2::kPlFull + 8u * pq, (g / S2::kPlaneStages) & 1u, abort_flag, p.faults)) break;
                tc_fence_after();
                const uint32_t stage = plane_stage(pq);
                const uint64_t bd0 = sw64_desc(stage + 4u * kT2PlaneA);
#pragma unroll
                for (uint32_t t = 0; t < kT2StageK / 16; ++t) {
#pragma unroll
                    for (uint32_t i = 0; i < 4; ++i) {
                        const uint64_t ad = sw64_desc(stage + i * kT2PlaneA) + 2u * t;  // + 32 bytes per k-step
                        mma_f16(tmem + (b * 4u + i) * (uint32_t)TN, ad, bd0 + 2u * t, Sh::idesc(4u - i),
                                (first && t == 0 && i == 0) ? 0u : 1u);
                    }
                }
                mma_commit(base + S2::kPlEmpty + 8u * pq);
                if (last) mma_commit(base + S2::kAccFull + 8u * b);
            }
            // every MMA issued completes before the tensor memory is freed (bounded)
            mma_commit(base + S2::kDone);
            bool done = false;
            for (uint32_t i = 0; i < kTcSpinLimit && !done; ++i) done = try_wait(base + S2::kDone, 0u);
            if (!done) atomicOr(p.faults, PIR_FAULT_WAIT_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ---- drain warps: class accumulators -> u32 totals of this lane's row --
        uint32_t total[TN];
#pragma unroll
        for (int n = 0; n < TN; ++n) total[n] = 0u;
        const uint32_t lane_addr = tmem + ((warp * 32u) << 16);
        bool ok = true;
        for (uint32_t c = 0; c < nch; ++c) {
            const uint32_t b = c & 1u;
            ok = __all_sync(0xffffffffu, wait_bounded(base + S2::kAccFull + 8u * b, (c >> 1) & 1u, abort_flag, p.faults));
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (uint32_t d = 0; d < 4; ++d) {
#pragma unroll
                for (uint32_t h = 0; h < (uint32_t)TN / 32u; ++h) {
                    uint32_t rr[32];
                    tmem_ld32(lane_addr + (b * 4u + d) * (uint32_t)TN + h * 32u, rr);
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        total[h * 32 + e] += (uint32_t)__float2int_rn(__uint_as_float(rr[e])) << (8u * d);
                }
            }
            tc_fence_before();
            mbar_arrive(base + S2::kAccEmpty + 8u * b);
        }
        const uint32_t m = m0 + warp * 32u + lane;
        if (ok && m < p.B) {
#pragma unroll
            for (int n = 0; n < TN; ++n)
                if (n0 + n < p.W && total[n]) atomicAdd(p.out + (uint64_t)m * p.W + n0 + n, total[n]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kTcMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::kTmemCols)
                     : "memory");
    }
}

template <int TN>
int launch_tc2(const CUtensorMap& ts, const CUtensorMap& tt, const TcParams& p, dim3 grid, cudaStream_t s) {
    using S2 = Tc2Shape<TN>;
    cudaError_t e = cudaFuncSetAttribute(contract_tc2_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S2::kSmem);
    if (e != cudaSuccess) return cuda_fail((int)e, "contract (tcgen05, tensor-map copies) attribute");
    contract_tc2_kernel<TN><<<grid, kT2Threads, S2::kSmem, s>>>(ts, tt, p);
    e = cudaGetLastError();
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "contract (tcgen05, tensor-map copies) launch");
}

template <int TN>
int launch_tc(const TcParams& p, dim3 grid, cudaStream_t s) {
    using Sh = TcShape<TN>;
    cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Sh::kSmem);
    if (e != cudaSuccess) return cuda_fail((int)e, "contract (tcgen05) attribute");
    contract_tc_kernel<TN><<<grid, kTcThreads, Sh::kSmem, s>>>(p);
    e = cudaGetLastError();
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "contract (tcgen05) launch");
}

// ---- tensor maps ---------------------------------------------------------------
// cuTensorMapEncodeTiled through the runtime's driver entry point (the library
// does not link the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        EncodeTiledFn r = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            r = reinterpret_cast<EncodeTiledFn>(f);
        cudaGetLastError();
        return r;
    }();
    return fn;
}

// A row-major u32 matrix of `rows` rows of `cols` words at a pitch of `pitch`
// words, copied in boxes of box_rows x box_cols words; zeros past its edges.
bool encode_u32(CUtensorMap* m, const uint32_t* data, uint64_t cols, uint64_t rows, uint64_t pitch,
                uint32_t box_cols, uint32_t box_rows) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {pitch * 4u};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t elem[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(data), dims, strides, box, elem,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tensor-map kernel unless PIR_TC_TENSOR_MAPS=0 in the environment (read
// at every launch: a comparison knob, the two kernels give the same result).
bool tensor_maps_enabled() {
    const char* e = std::getenv("PIR_TC_TENSOR_MAPS");
    return !(e && e[0] == '0');
}

}  // namespace
}  // namespace dev

int launch_contract_tc(const uint32_t* shares, uint64_t ld, uint32_t batch, const uint32_t* table, uint64_t stride,
                       uint32_t width, uint64_t rows, uint32_t* out, void* stream) {
    uint32_t* faults = device_fault_word();
    if (!faults) return cuda_fail((int)cudaGetLastError(), "device fault word");
    const uint32_t tn = width <= 32 ? 32u : 64u;
    const uint64_t mt = (batch + dev::kTcM - 1) / dev::kTcM, nt = (width + tn - 1) / tn;
    const uint64_t sms = (uint64_t)std::max(1, device_sm_count());
    // one CTA per SM: the output tiles times enough CTAs along k to fill one
    // wave, each taking whole 256-value accumulator chunks
    const uint64_t nchunks = (rows + dev::kTcChunkK - 1) / dev::kTcChunkK;
    uint64_t slices = std::min<uint64_t>(nchunks, std::max<uint64_t>(1, sms / (mt * nt)));
    const uint64_t cpc = (nchunks + slices - 1) / slices;
    slices = (nchunks + cpc - 1) / cpc;
    if (slices > 0x7fffffffull || cpc > 0xffffffffull || mt > 65535 || nt > 65535) return PIR_ERR_UNSUPPORTED;
    dev::TcParams p;
    p.S = shares;
    p.ld = ld;
    p.T = table;
    p.stride = stride;
    p.K = rows;
    p.nchunks = nchunks;
    p.cpc = (uint32_t)cpc;
    p.out = out;
    p.faults = faults;
    p.B = batch;
    p.W = width;
    p.vec = (reinterpret_cast<uintptr_t>(shares) % 16 == 0 && reinterpret_cast<uintptr_t>(table) % 16 == 0 &&
             ld % 4 == 0 && stride % 4 == 0)
                ? 1u
                : 0u;
    const dim3 grid((uint32_t)slices, (uint32_t)mt, (uint32_t)nt);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Aligned operands: the raw tiles by tensor-map copies (S as rows x k words
    // in boxes of 128 x 32, T as k x width words in boxes of 32 x TN), whose
    // strides (multiples of 16 bytes) and extents the encoder checks.
    if (p.vec && dev::tensor_maps_enabled() && rows < 0x80000000ull) {  // copy coordinates are signed 32-bit
        CUtensorMap ts, tt;
        if (dev::encode_u32(&ts, shares, rows, batch, ld, dev::kT2StageK, dev::kTcM) &&
            dev::encode_u32(&tt, table, width, rows, stride, tn, dev::kT2StageK))
            return tn == 32 ? dev::launch_tc2<32>(ts, tt, p, grid, s) : dev::launch_tc2<64>(ts, tt, p, grid, s);
    }
    return tn == 32 ? dev::launch_tc<32>(p, grid, s) : dev::launch_tc<64>(p, grid, s);
}

}  // namespace pir
