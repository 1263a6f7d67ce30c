// Fused DPF full-domain evaluation x table product mod 2^32 for sm_103a.
//
// What it computes (paper Sec. 3.1, Eqs. p1-p3; fusion of Sec. 3.2.4):
//   out[q][w] += sum_{j in rows} y_q(j) * T[j][w]   (mod 2^32)
// where y_q(j) is leaf j of key q's GGM tree:
//   P(0,0) = root;  P(d,j) = AES_{P(d-1,j>>1)}((j&1) || 0^120) ^ C_t[j&1][d],
//   t = lsb(P(d-1,j>>1));  y(j) = (-1)^sigma (word1(P(n,j)) + lsb(P(n,j)) * cw_out).
//
// Structure.  One CTA per SM (512 producer + 256 consumer threads), persistent
// over work items; an item is G queries x 2^r consecutive rows.
//  1. lookup tables, built once per CTA from a T-table column the compiler
//     derives (S-box from GF(2^8)): the four AES column tables Te0..Te3
//     (Te_r = rotl(Te0, 8r)), each with 32 lane-private copies so that lane l
//     always reads bank l.  A lookup is one PRMT (forms (byte << 8) | 4l) plus
//     one LDS; no rotations.
//  2. per item, path: thread g walks query g from the root to the item's
//     range node at depth n - r (one PRF block per level: the child on the path).
//  3. split: level by level in shared memory until each query has one subtree
//     root per thread (SQ = 512/G threads per query); a thread per child while
//     a level has few nodes.
//  4. per-thread depth-first expansion of its subtree (the paper's
//     memory-bounded traversal, Sec. 3.2.3), pending right siblings in a
//     shared-memory stack: O(threads x depth) node storage, not O(L).  One
//     PRF evaluation yields both children (one key schedule, two blocks that
//     share their first two rounds' lookups); for leaves only the 5 output
//     bytes that the share needs are computed in the last round.
//  5. warp-specialised fusion (Sec. 3.2.4): 16 producer warps run steps 2-4
//     and drop every kc (<= kPairs) leaf pairs' shares into one of two
//     shared-memory buffers; 8 consumer warps multiply each buffer, for all
//     G queries at once, into register accumulators against the table rows
//     it indexes (each row read once per CTA), while the producers fill the
//     other buffer.  Named barriers pass the buffers back and forth; the
//     consumers read a query's shares of up to four rows with one load, and
//     for one or two queries per item have the copy engine prefetch the next
//     phase's rows into L2.
//  6. accumulators are summed in shared memory and added to out with one
//     u32 atomicAdd per (query, word); addition mod 2^32 is associative, so
//     the result is bit-exact in any order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "async_copy.cuh"
#include "internal.h"

namespace pir {
namespace dev {

// Tuning knobs (compile-time): consumer warps per CTA, leaf pairs per hand-off.
#ifndef PIR_CONSUMER_WARPS
#define PIR_CONSUMER_WARPS 8
#endif
#ifndef PIR_PAIRS_PER_PHASE
#define PIR_PAIRS_PER_PHASE 4
#endif
constexpr int kProducers = 512;                             // threads that expand the tree
constexpr int kConsumers = 32 * PIR_CONSUMER_WARPS;         // threads that multiply into the table
constexpr int kFusedThreads = kProducers + kConsumers;
constexpr int kMaxChunks = kConsumers;                      // W / VEC limit of the fused product
constexpr int kPlaneBytes = 256 * 256;                     // 256 rows x [32 copies of Te_a | 32 of Te_b]
constexpr int kTablesBytes = 2 * kPlaneBytes;              // plane 0: Te0|Te1, plane 1: Te2|Te3
constexpr int kStackLevels = 8;                            // pending siblings per thread
constexpr int kMaxDfsDepth = kStackLevels + 1;             // levels a thread expands on its own
constexpr int kStackOff = kTablesBytes;
constexpr int kStackBytes = kStackLevels * kProducers * 16;  // 64 KiB
constexpr int kPairs = PIR_PAIRS_PER_PHASE;                // leaf pairs per subtree between MAC phases
constexpr int kYOff = kStackOff + kStackBytes;
constexpr int kYWords = 2 * 2 * kPairs * kProducers;       // two buffers of G x 2kPairs x SQ words
// The same region first holds the split phase's two node buffers (kProducers
// uint4 each) and at the end the per-item reduction (G x W words): size it
// for the largest of the three uses.
constexpr int kSplitWords = 2 * kProducers * 4;
constexpr int kYRegionWords = kYWords > kSplitWords ? kYWords : kSplitWords;
constexpr int kHdrOff = kYOff + 4 * kYRegionWords;
constexpr int kMaxGroup = 8;
constexpr int kHdrBytes = 48 * kMaxGroup;                  // per query slot: QueryHdr
constexpr int kItemOff = kHdrOff + kHdrBytes;              // work-item index broadcast (multi-table kernel)
// Staged table scan (fused_eval_staged_kernel): one more warp issues bulk
// copies of the table rows into a ring of shared-memory stages, each stage one
// level of the DFS stack that the launch's subtrees leave unused (stage s is
// level kStackLevels - s).  Its full and empty mbarriers and an abort flag
// follow the work-item slot.
constexpr int kIssuerThreads = 32;
constexpr int kStagedThreads = kFusedThreads + kIssuerThreads;
constexpr uint32_t kRingStageBytes = kProducers * 16;      // one stack level
constexpr int kRingMaxStages = kStackLevels - 1;           // level 1 always holds staged keys
constexpr int kRingBarOff = kItemOff + 16;                 // full[s] at +8s, empty[s] at +8(kRingMaxStages + s)
constexpr int kRingAbortOff = kRingBarOff + 16 * kRingMaxStages;
constexpr int kSmemBytes = kRingAbortOff + 16;
static_assert(kRingBarOff % 8 == 0, "mbarriers need 8-byte alignment");
static_assert(kSmemBytes <= 232448, "dynamic shared memory above the 227 KiB a CTA may use");
// Polls of a bounded mbarrier wait in the staged scan (each try_wait may also
// suspend the thread): far beyond any copy's latency, short of a hang.
constexpr uint32_t kRingSpinLimit = 1u << 22;
// Widest table row (words) the staged scan takes: four runs of a leaf pair must
// fit one stage.
constexpr uint64_t kRingMaxStride = kRingStageBytes / (4u * 2u * 4u);
#ifndef PIR_RING_MIN_PHASES
#define PIR_RING_MIN_PHASES 4
#endif
#ifndef PIR_RING_FENCE
#define PIR_RING_FENCE 1
#endif
#ifndef PIR_RING_PREFETCH_DEFAULT
#define PIR_RING_PREFETCH_DEFAULT 16
#endif

// The kernel's only shared memory; naming the array (not a pointer to it) in
// every access lets the compiler address it as shared.
extern __shared__ __align__(128) char sm[];

// Offset of `sm` in the CTA's shared window: the window begins with the 1 KiB
// the system reserves per block (cudaDevAttrReservedSharedMemoryPerBlock), and
// these kernels declare no static shared memory.  The table lookups carry it
// as an immediate, so that a lookup is PRMT + LDS [reg + imm] with no address
// add; the host refuses a device that reserves another amount and every
// kernel checks the offset before its first lookup.
constexpr uint32_t kSmemBase = 1024;

struct FusedParams {
    const uint32_t* table;
    uint64_t row_lo, row_hi;
    uint64_t stride;
    uint64_t first_range;
    uint64_t nitems;     // (query group, row range) items at 2^range_log2 rows
    uint64_t nfull;      // items run whole; the other nitems - nfull are cut into pieces
    uint32_t tail_log2;  // pieces of 2^(range_log2 - tail_log2) rows per cut item
    const uint8_t* keys;
    uint32_t* out;
    uint32_t* status;
    uint32_t key_bytes;
    uint32_t width;
    uint32_t batch;
    uint32_t n;
    uint32_t range_log2;
    uint32_t nqg;
    // expand-only mode: shares[q * ld + (row - row_lo)] = y_q(row)
    uint32_t* shares;
    uint64_t ld;
    uint32_t shares_vec;  // 1 when shares and ld allow 16-byte stores
    // bins mode (partial batch retrieval): query q covers rows [q*bin_rows, ...)
    uint64_t bin_rows;
    // staged scan: ring stages (2..kRingMaxStages), chunks the issuing warp
    // prefetches into L2 ahead of the one it copies, and the library's device
    // fault word (a wait that gives up sets PIR_FAULT_WAIT_TIMEOUT there)
    uint32_t ring_stages;
    uint32_t ring_prefetch;
    uint32_t* faults;
};

struct QueryHdr {  // one per query slot of the current item, in shared memory
    const uint8_t* key;
    uint32_t* out;
    uint32_t ok, party, cw_out, prf;
    const uint32_t* trow;  // bins mode: the slot's first table row
    uint64_t rows;         // bins mode: rows in the slot's bin
};
static_assert(sizeof(QueryHdr) * kMaxGroup <= kHdrBytes, "query slot headers exceed their region");

__device__ __forceinline__ QueryHdr* hdr_slot(int g) { return reinterpret_cast<QueryHdr*>(sm + kHdrOff) + g; }

// ---------------------------------------------------------------- GF(2^8)
// The AES S-box from its definition, evaluated by the compiler: S(x) is the
// affine map of x^254, the inverse of x in GF(2^8) modulo x^8+x^4+x^3+x+1
// (0 maps to 0).  Te0[x] holds the bytes 2S, S, S, 3S (byte 0 first): the
// MixColumns column of S(x).
constexpr uint32_t gf_xtime(uint32_t a) { return ((a << 1) ^ ((a & 0x80u) ? 0x1bu : 0u)) & 0xffu; }
constexpr uint32_t gf_mul(uint32_t a, uint32_t b) {
    uint32_t p = 0;
    for (int i = 0; i < 8; ++i) {
        if (b & 1u) p ^= a;
        a = gf_xtime(a);
        b >>= 1;
    }
    return p;
}
constexpr uint32_t sbox_entry(uint32_t x) {
    uint32_t inv = 1, base = x;
    for (int e = 254; e; e >>= 1) {  // square-and-multiply
        if (e & 1) inv = gf_mul(inv, base);
        base = gf_mul(base, base);
    }
    uint32_t s = inv;
    for (int k = 1; k <= 4; ++k) s ^= ((inv << k) | (inv >> (8 - k))) & 0xffu;
    return s ^ 0x63u;
}
struct Te0Table {
    uint32_t v[256];
};
constexpr Te0Table make_te0() {
    Te0Table t{};
    for (uint32_t x = 0; x < 256; ++x) {
        const uint32_t s = sbox_entry(x), s2 = gf_xtime(s);
        t.v[x] = s2 | (s << 8) | (s << 16) | ((s2 ^ s) << 24);
    }
    return t;
}
static_assert(sbox_entry(0) == 0x63u && sbox_entry(1) == 0x7cu, "S-box: affine constant and the inverse of 1");
__constant__ Te0Table kTe0 = make_te0();

// ---------------------------------------------------------------- lookups
// Te_t[x] for this lane sits at plane(t)*64K + x*256 + (t&1)*128 + 4*lane:
// one PRMT builds (x << 8) | (lane base), the plane offset is an immediate.
template <uint32_t OFF>
__device__ __forceinline__ uint32_t lds_at(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
    return v;
}
#define LKT(s, r, t) \
    lds_at<kSmemBase + ((t) >> 1) * kPlaneBytes>(__byte_perm((s), ((t) & 1) ? lane4h : lane4, 0x5504u | ((r) << 4)))
// main rounds: byte r of a column goes through Te_r
#define LK(s, r) LKT(s, r, r)
// S-box byte S(x) sits at byte p of Te_{(p+2)&3}[x]; gather four (one per byte position)
#define SBG(a, b, c, d) __byte_perm(__byte_perm((a), (b), 0x0050u), __byte_perm((c), (d), 0x7200u), 0x7610u)
// SubBytes+ShiftRows column: byte p from byte p of column (c+p)
#define SBCOL(w0, w1, w2, w3) SBG(LKT(w0, 0, 2), LKT(w1, 1, 3), LKT(w2, 2, 0), LKT(w3, 3, 1))

// Whether `sm` sits at kSmemBase of the shared window (uniform over the CTA,
// so a CTA that finds otherwise returns as a whole, before any barrier).
__device__ __forceinline__ bool smem_base_ok(uint32_t* status) {
    if ((uint32_t)__cvta_generic_to_shared(sm) == kSmemBase) return true;
    if (threadIdx.x == 0 && status) atomicOr(status, PIR_STATUS_SMEM_LAYOUT);
    return false;
}

// 4 tables x 256 rows x 32 lane copies = 32768 words, four lanes' copies (16
// bytes) per store.  blockDim.x is a multiple of 32, so a warp covers row x of
// all four tables (its constant read is one broadcast, its store four
// contiguous 128-byte runs).
__device__ void build_tables(int tid) {
#pragma unroll 2
    for (int f = tid; f < 8192; f += (int)blockDim.x) {
        const int x = f >> 5, t = (f >> 3) & 3, q = f & 7;
        const uint32_t v = kTe0.v[x];
        const uint32_t rv = t ? __funnelshift_l(v, v, 8 * t) : v;
        *reinterpret_cast<uint4*>(sm + (t >> 1) * kPlaneBytes + x * 256 + (t & 1) * 128 + q * 16) =
            make_uint4(rv, rv, rv, rv);
    }
    __syncthreads();
}

// Both children of node v before the codewords, c_b = AES_v(b || 0^120).
// With `leaf` set only byte 0 of c_b.x and all of c_b.y are produced (the
// control bit and the Z_2^32 word of a leaf); the rest is left undefined.
__device__ __forceinline__ void prf2(const uint32_t lane4, const uint32_t lane4h, const uint4 v, const bool leaf,
                                     uint4& c0, uint4& c1) {
    uint32_t k0 = v.x, k1 = v.y, k2 = v.z, k3 = v.w;
    const uint32_t s0 = k0, s1 = k1, s2 = k2, s3 = k3;  // round-0 state of block b=0
#define KEYROUND(rc)                                                                        \
    k0 ^= SBG(LKT(k3, 1, 2), LKT(k3, 2, 3), LKT(k3, 3, 0), LKT(k3, 0, 1)) ^ (rc);           \
    k1 ^= k0;                                                                               \
    k2 ^= k1;                                                                               \
    k3 ^= k2;
    KEYROUND(0x01u)
    // round 1: only byte 0 of column 0 differs between the two blocks
    const uint32_t x1 = LK(s1, 1) ^ LK(s2, 2) ^ LK(s3, 3) ^ k0;
    const uint32_t a0 = LK(s0, 0) ^ x1;
    const uint32_t b0 = LK(s0 ^ 1u, 0) ^ x1;
    const uint32_t u1 = LK(s1, 0) ^ LK(s2, 1) ^ LK(s3, 2) ^ LK(s0, 3) ^ k1;
    const uint32_t u2 = LK(s2, 0) ^ LK(s3, 1) ^ LK(s0, 2) ^ LK(s1, 3) ^ k2;
    const uint32_t u3 = LK(s3, 0) ^ LK(s0, 1) ^ LK(s1, 2) ^ LK(s2, 3) ^ k3;
    KEYROUND(0x02u)
    // round 2: columns 1..3 are shared; column 0 feeds one lookup per output column
    const uint32_t z0 = LK(u1, 1) ^ LK(u2, 2) ^ LK(u3, 3) ^ k0;
    const uint32_t z1 = LK(u1, 0) ^ LK(u2, 1) ^ LK(u3, 2) ^ k1;
    const uint32_t z2 = LK(u2, 0) ^ LK(u3, 1) ^ LK(u1, 3) ^ k2;
    const uint32_t z3 = LK(u3, 0) ^ LK(u1, 2) ^ LK(u2, 3) ^ k3;
    uint32_t A0 = LK(a0, 0) ^ z0, A1 = LK(a0, 3) ^ z1, A2 = LK(a0, 2) ^ z2, A3 = LK(a0, 1) ^ z3;
    uint32_t B0 = LK(b0, 0) ^ z0, B1 = LK(b0, 3) ^ z1, B2 = LK(b0, 2) ^ z2, B3 = LK(b0, 1) ^ z3;
    const uint32_t rcon[7] = {0x04u, 0x08u, 0x10u, 0x20u, 0x40u, 0x80u, 0x1bu};
#pragma unroll
    for (int r = 0; r < 7; ++r) {  // rounds 3..9
        KEYROUND(rcon[r])
        const uint32_t a0n = LK(A0, 0) ^ LK(A1, 1) ^ LK(A2, 2) ^ LK(A3, 3) ^ k0;
        const uint32_t a1n = LK(A1, 0) ^ LK(A2, 1) ^ LK(A3, 2) ^ LK(A0, 3) ^ k1;
        const uint32_t a2n = LK(A2, 0) ^ LK(A3, 1) ^ LK(A0, 2) ^ LK(A1, 3) ^ k2;
        const uint32_t a3n = LK(A3, 0) ^ LK(A0, 1) ^ LK(A1, 2) ^ LK(A2, 3) ^ k3;
        const uint32_t b0n = LK(B0, 0) ^ LK(B1, 1) ^ LK(B2, 2) ^ LK(B3, 3) ^ k0;
        const uint32_t b1n = LK(B1, 0) ^ LK(B2, 1) ^ LK(B3, 2) ^ LK(B0, 3) ^ k1;
        const uint32_t b2n = LK(B2, 0) ^ LK(B3, 1) ^ LK(B0, 2) ^ LK(B1, 3) ^ k2;
        const uint32_t b3n = LK(B3, 0) ^ LK(B0, 1) ^ LK(B1, 2) ^ LK(B2, 3) ^ k3;
        A0 = a0n; A1 = a1n; A2 = a2n; A3 = a3n;
        B0 = b0n; B1 = b1n; B2 = b2n; B3 = b3n;
    }
    KEYROUND(0x36u)
#undef KEYROUND
    // round 10: SubBytes + ShiftRows + AddRoundKey
    if (leaf) {
        c0.x = LKT(A0, 0, 2) ^ k0;
        c0.y = SBCOL(A1, A2, A3, A0) ^ k1;
        c1.x = LKT(B0, 0, 2) ^ k0;
        c1.y = SBCOL(B1, B2, B3, B0) ^ k1;
        c0.z = c0.w = c1.z = c1.w = 0u;
    } else {
        c0.x = SBCOL(A0, A1, A2, A3) ^ k0;
        c0.y = SBCOL(A1, A2, A3, A0) ^ k1;
        c0.z = SBCOL(A2, A3, A0, A1) ^ k2;
        c0.w = SBCOL(A3, A0, A1, A2) ^ k3;
        c1.x = SBCOL(B0, B1, B2, B3) ^ k0;
        c1.y = SBCOL(B1, B2, B3, B0) ^ k1;
        c1.z = SBCOL(B2, B3, B0, B1) ^ k2;
        c1.w = SBCOL(B3, B0, B1, B2) ^ k3;
    }
}

// One child alone, c_b = AES_v(b || 0^120): the key schedule and one block
// (200 lookups against 333 for both).  For the dependent levels, where a node
// is expanded on its own and its thread's instruction stream is the latency:
// the path to an item's range needs only the child on the path, and a split
// level with few nodes gives each child its own thread.
__device__ __forceinline__ void key_round(uint32_t lane4, uint32_t lane4h, uint32_t& k0, uint32_t& k1, uint32_t& k2,
                                          uint32_t& k3, uint32_t rc) {
    k0 ^= SBG(LKT(k3, 1, 2), LKT(k3, 2, 3), LKT(k3, 3, 0), LKT(k3, 0, 1)) ^ rc;
    k1 ^= k0;
    k2 ^= k1;
    k3 ^= k2;
}
__device__ __forceinline__ uint4 prf1(uint32_t lane4, uint32_t lane4h, const uint4 v, uint32_t b) {
    uint32_t k0 = v.x, k1 = v.y, k2 = v.z, k3 = v.w;
    uint32_t s0 = k0 ^ b, s1 = k1, s2 = k2, s3 = k3;  // round 0: plaintext xor key
    const uint32_t rcon[9] = {0x01u, 0x02u, 0x04u, 0x08u, 0x10u, 0x20u, 0x40u, 0x80u, 0x1bu};
#pragma unroll
    for (int rnd = 0; rnd < 9; ++rnd) {  // rounds 1..9
        key_round(lane4, lane4h, k0, k1, k2, k3, rcon[rnd]);
        const uint32_t t0 = LK(s0, 0) ^ LK(s1, 1) ^ LK(s2, 2) ^ LK(s3, 3) ^ k0;
        const uint32_t t1 = LK(s1, 0) ^ LK(s2, 1) ^ LK(s3, 2) ^ LK(s0, 3) ^ k1;
        const uint32_t t2 = LK(s2, 0) ^ LK(s3, 1) ^ LK(s0, 2) ^ LK(s1, 3) ^ k2;
        const uint32_t t3 = LK(s3, 0) ^ LK(s0, 1) ^ LK(s1, 2) ^ LK(s2, 3) ^ k3;
        s0 = t0;
        s1 = t1;
        s2 = t2;
        s3 = t3;
    }
    key_round(lane4, lane4h, k0, k1, k2, k3, 0x36u);
    // round 10: SubBytes + ShiftRows + AddRoundKey
    return make_uint4(SBCOL(s0, s1, s2, s3) ^ k0, SBCOL(s1, s2, s3, s0) ^ k1, SBCOL(s2, s3, s0, s1) ^ k2,
                      SBCOL(s3, s0, s1, s2) ^ k3);
}

// Both children under the ChaCha20 PRF: block 0 of ChaCha20 (RFC 8439) with
// key v || 0^128, counter 0, nonce 0; words 0..3 are child 0, 4..7 child 1.
#define CHACHA_QR(a, b, c, d)                                    \
    a += b; d ^= a; d = __byte_perm(d, 0u, 0x1032u);             \
    c += d; b ^= c; b = __funnelshift_l(b, b, 12);               \
    a += b; d ^= a; d = __byte_perm(d, 0u, 0x2103u);             \
    c += d; b ^= c; b = __funnelshift_l(b, b, 7);
__device__ __forceinline__ void prf2_chacha(const uint4 v, uint4& c0, uint4& c1) {
    constexpr uint32_t K0 = 0x61707865u, K1 = 0x3320646eu, K2 = 0x79622d32u, K3 = 0x6b206574u;
    uint32_t x0 = K0, x1 = K1, x2 = K2, x3 = K3, x4 = v.x, x5 = v.y, x6 = v.z, x7 = v.w;
    uint32_t x8 = 0, x9 = 0, x10 = 0, x11 = 0, x12 = 0, x13 = 0, x14 = 0, x15 = 0;
#pragma unroll 2
    for (int i = 0; i < 10; ++i) {
        CHACHA_QR(x0, x4, x8, x12) CHACHA_QR(x1, x5, x9, x13) CHACHA_QR(x2, x6, x10, x14) CHACHA_QR(x3, x7, x11, x15)
        CHACHA_QR(x0, x5, x10, x15) CHACHA_QR(x1, x6, x11, x12) CHACHA_QR(x2, x7, x8, x13) CHACHA_QR(x3, x4, x9, x14)
    }
    c0 = make_uint4(x0 + K0, x1 + K1, x2 + K2, x3 + K3);
    c1 = make_uint4(x4 + v.x, x5 + v.y, x6 + v.z, x7 + v.w);
}
#undef CHACHA_QR

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }

// Children of v: PRF plus the codeword pair C_{lsb(v)}[0][d], C_{lsb(v)}[1][d]
// (w0, w1).  `chacha` selects the key's PRF (uniform per query, so per warp in
// the DFS).
__device__ __forceinline__ void expand_with(uint32_t lane4, uint32_t lane4h, uint4 v, bool leaf, bool chacha, uint4 w0,
                                            uint4 w1, uint4& c0, uint4& c1) {
    if (chacha)
        prf2_chacha(v, c0, c1);
    else
        prf2(lane4, lane4h, v, leaf, c0, c1);
    c0 = xor4(c0, w0);
    c1 = xor4(c1, w1);
}

// Children of v at depth d (1-based) of `key` in global memory.
__device__ __forceinline__ void expand(uint32_t lane4, uint32_t lane4h, const uint8_t* key, uint32_t d, uint4 v,
                                       bool leaf, bool chacha, uint4& c0, uint4& c1) {
    // the codewords' address is known before the PRF: issue the loads first
    const uint4* cw = reinterpret_cast<const uint4*>(key + PIR_KEY_HEADER_BYTES + 64u * (d - 1) + 32u * (v.x & 1u));
    const uint4 w0 = __ldg(cw), w1 = __ldg(cw + 1);
    expand_with(lane4, lane4h, v, leaf, chacha, w0, w1, c0, c1);
}

// Before the depth-first phase the stack region holds a copy of each query
// slot's key (kKeySlotBytes apart), so that the path walk and the split, one
// dependent level after another, read their codewords from shared memory.
constexpr int kKeySlotBytes = PIR_KEY_HEADER_BYTES + 64 * PIR_MAX_DOMAIN_BITS;
static_assert(kMaxGroup * kKeySlotBytes <= kStackBytes, "staged keys exceed the stack region");
static_assert(kKeySlotBytes % 16 == 0, "key slots must keep 16-byte alignment");
__device__ __forceinline__ const uint4* staged_key(int g) {
    return reinterpret_cast<const uint4*>(sm + kStackOff + g * kKeySlotBytes);
}
__device__ __forceinline__ void expand_staged(uint32_t lane4, uint32_t lane4h, int g, uint32_t d, uint4 v, bool chacha,
                                              uint4& c0, uint4& c1) {
    const uint4* cw = staged_key(g) + (PIR_KEY_HEADER_BYTES / 16) + 4u * (d - 1) + 2u * (v.x & 1u);
    expand_with(lane4, lane4h, v, false, chacha, cw[0], cw[1], c0, c1);
}

// Child b of v at depth d (1-based) of staged key g: PRF plus the codeword
// C_{lsb(v)}[b][d].
__device__ __forceinline__ uint4 expand1_staged(uint32_t lane4, uint32_t lane4h, int g, uint32_t d, uint4 v, uint32_t b,
                                                bool chacha) {
    const uint4* cw = staged_key(g) + (PIR_KEY_HEADER_BYTES / 16) + 4u * (d - 1) + 2u * (v.x & 1u) + b;
    uint4 c;
    if (chacha) {  // one ChaCha20 block holds both children
        uint4 c0, c1;
        prf2_chacha(v, c0, c1);
        c = b ? c1 : c0;
    } else {
        c = prf1(lane4, lane4h, v, b);
    }
    return xor4(c, cw[0]);
}

// Split levels with at most this many nodes give each child its own thread.
constexpr int kPairNodes = 128;

// Pending right sibling at relative level `lvl` (1..8) of thread `tid`.
__device__ __forceinline__ uint4* stack_slot(int lvl, int tid) {
    return reinterpret_cast<uint4*>(sm + kStackOff) + (lvl - 1) * kProducers + tid;
}

template <int VEC>
__device__ __forceinline__ void load_row(const uint32_t* p, uint32_t (&v)[VEC]) {
    if constexpr (VEC == 4) {
        const uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        v[0] = __ldg(p);
    }
}

// Bulk prefetch of a byte range into L2 by the copy engine (no registers, no
// shared memory; completes on its own).  addr 16-byte aligned, bytes a
// multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* addr, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(addr), "r"(bytes) : "memory");
}

// Table rows that one hand-off phase multiplies, per CTA, above which the
// next phase is not prefetched (all CTAs' two phases in flight must fit L2).
#ifndef PIR_PF_MAX_KIB
#define PIR_PF_MAX_KIB 256
#endif
#ifndef PIR_PF_AHEAD
#define PIR_PF_AHEAD 1
#endif
#ifndef PIR_PF_EARLY
#define PIR_PF_EARLY 0
#endif
constexpr uint32_t kPrefetchMaxBytes = PIR_PF_MAX_KIB * 1024u;
// Phases whose rows are asked of L2 ahead of the one being multiplied, and
// whether the first of them are asked for at the start of the item (while its
// path walk and split run) rather than when the consumers start.
constexpr uint32_t kPfAhead = PIR_PF_AHEAD;
constexpr bool kPfEarly = PIR_PF_EARLY != 0;

// Consumers ask L2 for the rows of leaf pairs kbase..kbase+kc-1 of every
// subtree ahead of the phase that multiplies them: per subtree one run of 2kc
// consecutive rows, clipped to the table (16-byte rows only, VEC == 4).
__device__ __forceinline__ void prefetch_phase(const FusedParams& p, uint64_t r0, int m, uint32_t nsub, uint32_t kbase,
                                               uint32_t kc, uint32_t ct) {
    for (uint32_t l = ct; l < nsub; l += kConsumers) {
        uint64_t a = r0 + ((uint64_t)l << m) + 2ull * kbase, b = a + 2ull * kc;
        a = a > p.row_lo ? a : p.row_lo;
        b = b < p.row_hi ? b : p.row_hi;
        if (a >= b) continue;
        const uint64_t bytes = ((b - a - 1) * p.stride + p.width) * 4ull;
        prefetch_l2(p.table + (a - p.row_lo) * p.stride, (uint32_t)bytes);
    }
}

// The same for every query slot's own bin (bins mode).
template <int G>
__device__ __forceinline__ void prefetch_phase_bins(const FusedParams& p, uint64_t r0, int m, uint32_t nsub,
                                                    uint32_t kbase, uint32_t kc, uint32_t ct) {
    for (uint32_t i = ct; i < (uint32_t)G * nsub; i += kConsumers) {
        const uint32_t g = i / nsub, l = i - g * nsub;
        const QueryHdr* h = hdr_slot((int)g);
        if (!h->trow) continue;
        const uint64_t a = r0 + ((uint64_t)l << m) + 2ull * kbase;
        uint64_t b = a + 2ull * kc;
        b = b < h->rows ? b : h->rows;
        if (a >= b) continue;
        const uint64_t bytes = ((b - a - 1) * p.stride + p.width) * 4ull;
        prefetch_l2(h->trow + a * p.stride, (uint32_t)bytes);
    }
}

template <int G, bool BINS>
__device__ __forceinline__ void prefetch_rows(const FusedParams& p, uint64_t r0, int m, uint32_t nsub, uint32_t kbase,
                                              uint32_t kc, uint32_t ct) {
    if constexpr (BINS)
        prefetch_phase_bins<G>(p, r0, m, nsub, kbase, kc, ct);
    else
        prefetch_phase(p, r0, m, nsub, kbase, kc, ct);
}

// Table rows a consumer thread has in flight when an item holds one or two
// queries (the scan is then as heavy as the expansion): a multiple of 4.
#ifndef PIR_SMALLG_ROWS
#define PIR_SMALLG_ROWS 8
#endif
constexpr int kSmallGroupRows = PIR_SMALLG_ROWS;
static_assert(kSmallGroupRows % 4 == 0, "rows in flight in groups of four");

// Named barriers between producers and consumers: kBarFull + b marks share
// buffer b as filled, kBarFree + b as consumed (barrier 0 is __syncthreads).
constexpr int kBarFull = 1, kBarFree = 3;
__device__ __forceinline__ void bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Rows in groups of R (R = 2 or 4): rows (j, l), ..., (j, l + R - 1) with l a
// multiple of R have adjacent shares for every query, so one 64- or 128-bit
// load fetches a query's shares of the whole group.  Group q of the phase is
// rows R q .. R q + R - 1 in the phase's row order (all with the same j when
// the subtree count 2^sd is at least R); consumer (c, rg) takes groups rg,
// rg + nrg, ..., with 8 (G <= 2) or 4 rows in flight.
template <int G, int VEC, int R>
__device__ __forceinline__ void mac_rows_grouped(const FusedParams& p, const uint32_t* yb, uint64_t r0, int m, int sd,
                                                 uint32_t kbase, uint32_t nrows, uint32_t (&acc)[G][VEC], uint32_t c,
                                                 uint32_t rg, uint32_t nrg) {
    static_assert(R == 2 || R == 4, "rows per group");
    constexpr int SQ = kProducers / G;
    constexpr int UG = (G <= 2 ? kSmallGroupRows : 4) / R;
    const uint32_t submask = (1u << sd) - 1u;
    const uint32_t ngroups = nrows / R;
    for (uint32_t q0 = rg; q0 < ngroups; q0 += UG * nrg) {
        uint32_t tv[UG][R][VEC];
        uint32_t yi[UG];
        bool any[UG];
#pragma unroll
        for (int u = 0; u < UG; ++u) {
            const uint32_t q = q0 + u * nrg;
            const uint32_t rr = (uint32_t)R * q;
            const uint32_t j = rr >> sd, l = rr & submask;
            yi[u] = j * SQ + l;
            any[u] = false;
#pragma unroll
            for (int h = 0; h < R; ++h) {
                const uint64_t row = r0 + ((uint64_t)(l + h) << m) + 2ull * kbase + j;
                const bool ok = q < ngroups && row >= p.row_lo && row < p.row_hi;
                any[u] |= ok;
                if (ok) {
                    load_row<VEC>(p.table + (row - p.row_lo) * p.stride + (uint64_t)c * VEC, tv[u][h]);
                } else {
#pragma unroll
                    for (int i = 0; i < VEC; ++i) tv[u][h][i] = 0;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UG; ++u) {
            if (!any[u]) continue;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                uint32_t y[R];
                if constexpr (R == 4) {
                    const uint4 v = *reinterpret_cast<const uint4*>(yb + g * 2 * kPairs * SQ + yi[u]);
                    y[0] = v.x; y[1] = v.y; y[2] = v.z; y[3] = v.w;
                } else {
                    const uint2 v = *reinterpret_cast<const uint2*>(yb + g * 2 * kPairs * SQ + yi[u]);
                    y[0] = v.x; y[1] = v.y;
                }
#pragma unroll
                for (int i = 0; i < VEC; ++i) {
                    uint32_t a = acc[g][i];
#pragma unroll
                    for (int h = 0; h < R; ++h) a += y[h] * tv[u][h][i];
                    acc[g][i] = a;
                }
            }
        }
    }
}

// Consumer thread `ct` of kConsumers: multiply the shares of leaf pairs
// kbase..kbase+kc-1 of every subtree (buffer yb) into acc.  Consumer (c, rg)
// owns words c*VEC..c*VEC+VEC-1 of every G query.  With two or more subtrees
// it takes rows in groups whose shares it loads together (mac_rows_grouped);
// with one subtree, rows rg, rg+nrg, ..., U at a time, U rows' loads issued
// before their multiply-adds (U = 8 for one or two queries per item, where the
// scan is a large share of the work, else 4).
template <int G, int VEC>
__device__ __forceinline__ void mac_phase(const FusedParams& p, const uint32_t* yb, uint64_t r0, int m, int sd,
                                          uint32_t kbase, uint32_t kc, uint32_t (&acc)[G][VEC], uint32_t ct) {
    constexpr int SQ = kProducers / G;
    const uint32_t nc = p.width / VEC;
    const uint32_t nrg = kConsumers / nc;
    const uint32_t c = ct % nc, rg = ct / nc;
    if (rg >= nrg) return;
    const uint32_t nrows = (2u * kc) << sd;
    const uint32_t submask = (1u << sd) - 1u;
    if constexpr (VEC == 4) {  // (groups of four with 32-bit table loads would spill at G = 8)
        if (sd >= 2) {
            mac_rows_grouped<G, VEC, 4>(p, yb, r0, m, sd, kbase, nrows, acc, c, rg, nrg);
            return;
        }
    }
    if (sd >= 1) {
        mac_rows_grouped<G, VEC, 2>(p, yb, r0, m, sd, kbase, nrows, acc, c, rg, nrg);
        return;
    }
    constexpr int U = G <= 2 ? kSmallGroupRows : 4;
    for (uint32_t rr0 = rg; rr0 < nrows; rr0 += U * nrg) {
        uint32_t tv[U][VEC];
        uint32_t yi[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t rr = rr0 + u * nrg;
            const uint32_t j = rr >> sd, l = rr & submask;
            const uint64_t row = r0 + ((uint64_t)l << m) + 2ull * kbase + j;
            ok[u] = rr < nrows && row >= p.row_lo && row < p.row_hi;
            yi[u] = j * SQ + l;
            if (ok[u]) {
                load_row<VEC>(p.table + (row - p.row_lo) * p.stride + (uint64_t)c * VEC, tv[u]);
            } else {
#pragma unroll
                for (int i = 0; i < VEC; ++i) tv[u][i] = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!ok[u]) continue;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t y = yb[g * 2 * kPairs * SQ + yi[u]];
#pragma unroll
                for (int i = 0; i < VEC; ++i) acc[g][i] += y * tv[u][i];
            }
        }
    }
}

// Bins mode (partial batch retrieval): the G slots are G bins, each with its
// own rows.  The consumers form G teams of kConsumers/G threads; team g
// multiplies only slot g's shares, against slot g's rows (bin-relative index
// r0 + (l << m) + 2*kbase + j), into acc[0].  128-bit loads only.
template <int G>
__device__ __forceinline__ void mac_phase_bins(const FusedParams& p, const uint32_t* yb, uint64_t r0, int m, int sd,
                                               uint32_t kbase, uint32_t kc, uint32_t (&acc)[G][4], uint32_t ct) {
    constexpr int SQ = kProducers / G;
    constexpr uint32_t kTeam = kConsumers / G;
    const uint32_t g = ct / kTeam, t = ct % kTeam;
    const uint32_t nc = p.width / 4u;
    const uint32_t nrg = kTeam / nc;
    const uint32_t c = t % nc, rg = t / nc;
    const QueryHdr* h = hdr_slot((int)g);
    if (rg >= nrg || !h->out) return;
    const uint32_t* trow = h->trow;
    const uint64_t bin_rows = h->rows;
    const uint32_t* ys = yb + g * 2 * kPairs * SQ;
    const uint32_t nrows = (2u * kc) << sd;
    const uint32_t submask = (1u << sd) - 1u;
    constexpr int U = 8;
    for (uint32_t rr0 = rg; rr0 < nrows; rr0 += U * nrg) {
        uint32_t tv[U][4];
        uint32_t yi[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t rr = rr0 + u * nrg;
            const uint32_t j = rr >> sd, l = rr & submask;
            const uint64_t rel = r0 + ((uint64_t)l << m) + 2ull * kbase + j;
            ok[u] = rr < nrows && rel < bin_rows;
            yi[u] = j * SQ + l;
            if (ok[u]) {
                load_row<4>(trow + rel * p.stride + (uint64_t)c * 4u, tv[u]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) tv[u][i] = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!ok[u]) continue;
            const uint32_t y = ys[yi[u]];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[0][i] += y * tv[u][i];
        }
    }
}

// ---------------------------------------------------------------- staged scan
// The rows one hand-off phase multiplies are, for every subtree l of the item,
// one run of 2kc consecutive rows (leaf pairs kbase..kbase+kc-1 of subtree l).
// The staged kernel moves them into shared memory with the bulk-copy engine:
// chunk ch of a phase is the runs of subtrees ch*rpc .. ch*rpc+rpc-1, one ring
// stage each, and chunks go through the ring phase by phase.
struct RingGeom {
    uint32_t kc;   // leaf pairs per subtree per phase
    uint32_t rpc;  // runs per chunk: a power of two, at least 4
    uint32_t nch;  // chunks per phase
    bool on;       // whether this item's table scan goes through the ring
};

// For an item whose subtrees are 2^m rows deep, 2^sd of them.  Both the
// issuing warp and the consumers derive it, so they walk the same chunks.
__device__ __forceinline__ RingGeom ring_geom(const FusedParams& p, int sd, int m) {
    RingGeom g{};
    const uint32_t npairs = 1u << (m - 1);
    uint32_t kc = max(1u, min((uint32_t)kPairs, npairs / PIR_RING_MIN_PHASES));
    const uint32_t pair_bytes = 2u * (uint32_t)p.stride * 4u;  // one leaf pair's rows
    while (kc > 1 && 4u * kc * pair_bytes > kRingStageBytes) kc >>= 1;
    const uint32_t fit = kRingStageBytes / (kc * pair_bytes);
    uint32_t rpc = fit ? 1u << (31 - __clz(fit)) : 0u;
    rpc = min(rpc, 1u << sd);
    g.kc = kc;
    g.rpc = rpc;
    g.nch = rpc ? (1u << sd) / rpc : 0u;
    g.on = p.ring_stages >= 2 && rpc >= 4;
    return g;
}

__device__ __forceinline__ char* ring_stage(uint32_t s) {
    return sm + kStackOff + (kStackLevels - 1 - (int)s) * (int)kRingStageBytes;
}
__device__ __forceinline__ uint32_t ring_full(uint32_t s) { return smem_addr(sm + kRingBarOff) + 8u * s; }
__device__ __forceinline__ uint32_t ring_empty(uint32_t s) {
    return smem_addr(sm + kRingBarOff) + 8u * (kRingMaxStages + s);
}
__device__ __forceinline__ volatile uint32_t* ring_abort() {
    return reinterpret_cast<volatile uint32_t*>(sm + kRingAbortOff);
}

// The part of run u of chunk ch inside [row_lo, row_hi): its first row and the
// bytes of its span (zero when the run lies outside).
__device__ __forceinline__ uint32_t ring_run(const FusedParams& p, uint64_t r0, int m, uint32_t kbase,
                                             const RingGeom& g, uint32_t ch, uint32_t u, uint64_t& first,
                                             uint32_t& skip) {
    const uint64_t a = r0 + ((uint64_t)(ch * g.rpc + u) << m) + 2ull * kbase;
    const uint64_t b = a + 2ull * g.kc;
    const uint64_t lo = a > p.row_lo ? a : p.row_lo, hi = b < p.row_hi ? b : p.row_hi;
    first = lo;
    skip = (uint32_t)(lo - a);
    return lo < hi ? (uint32_t)(((hi - lo - 1) * p.stride + p.width) * 4u) : 0u;
}

// Issuing warp: chunk ch of the phase at leaf pair kbase into ring stage s.
// Lane 0 arrives on the stage's full barrier with the chunk's byte count, then
// every lane starts the copies of its runs (rpc <= 512, so at most 16 each).
// Table rows and their copies in shared memory keep the table's row pitch.
__device__ __forceinline__ void ring_issue(const FusedParams& p, uint64_t r0, int m, uint32_t kbase,
                                           const RingGeom& g, uint32_t ch, uint32_t s, uint32_t lane) {
    const uint32_t bar = ring_full(s);
    const uint32_t dst0 = smem_addr(ring_stage(s));
    const uint32_t row_bytes = (uint32_t)p.stride * 4u;
    uint32_t total = 0;
    for (uint32_t u = lane; u < g.rpc; u += 32) {
        uint64_t first;
        uint32_t skip;
        total += ring_run(p, r0, m, kbase, g, ch, u, first, skip);
    }
    total = __reduce_add_sync(0xffffffffu, total);
    if (lane == 0) mbar_expect_tx(bar, total);
    __syncwarp();
    for (uint32_t u = lane; u < g.rpc; u += 32) {
        uint64_t first;
        uint32_t skip;
        const uint32_t bytes = ring_run(p, r0, m, kbase, g, ch, u, first, skip);
        if (bytes)
            bulk_g2s(dst0 + (u * 2u * g.kc + skip) * row_bytes, p.table + (first - p.row_lo) * p.stride, bytes, bar);
    }
}

// The same rows asked of L2 ahead of their copy (the copy engine fetches them
// while the ring is still full).
__device__ __forceinline__ void ring_prefetch(const FusedParams& p, uint64_t r0, int m, uint32_t kbase,
                                              const RingGeom& g, uint32_t ch, uint32_t lane) {
    for (uint32_t u = lane; u < g.rpc; u += 32) {
        uint64_t first;
        uint32_t skip;
        const uint32_t bytes = ring_run(p, r0, m, kbase, g, ch, u, first, skip);
        if (bytes) prefetch_l2(p.table + (first - p.row_lo) * p.stride, bytes);
    }
}

// Consumer thread ct: multiply chunk ch of the phase at leaf pair kbase (ring
// stage `stage`, shares in yb) into acc.  Consumer (c, rg) owns words
// 4c..4c+3; it takes groups of four runs u..u+3 at the same row j of their
// runs, whose shares are adjacent for every query (one 128-bit load each).
template <int G>
__device__ __forceinline__ void mac_chunk(const FusedParams& p, const uint32_t* yb, const char* stage, uint64_t r0,
                                          int m, uint32_t kbase, const RingGeom& g, uint32_t ch,
                                          uint32_t (&acc)[G][4], uint32_t ct) {
    constexpr int SQ = kProducers / G;
    const uint32_t nc = p.width / 4u;
    const uint32_t nrg = kConsumers / nc;
    const uint32_t c = ct % nc, rg = ct / nc;
    if (rg >= nrg) return;
    const uint32_t two_kc = 2u * g.kc;
    const uint32_t ngroups = (g.rpc / 4u) * two_kc;
    const uint32_t row_bytes = (uint32_t)p.stride * 4u;
    for (uint32_t q = rg; q < ngroups; q += nrg) {
        const uint32_t j = q & (two_kc - 1u), u = (q / two_kc) * 4u;
        const uint32_t l = ch * g.rpc + u;
        uint4 t[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint64_t row = r0 + ((uint64_t)(l + h) << m) + 2ull * kbase + j;
            t[h] = (row >= p.row_lo && row < p.row_hi)
                       ? *reinterpret_cast<const uint4*>(stage + ((u + h) * two_kc + j) * row_bytes + c * 16u)
                       : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int a = 0; a < G; ++a) {
            const uint4 y = *reinterpret_cast<const uint4*>(yb + (a * 2 * kPairs + j) * SQ + l);
            acc[a][0] += y.x * t[0].x + y.y * t[1].x + y.z * t[2].x + y.w * t[3].x;
            acc[a][1] += y.x * t[0].y + y.y * t[1].y + y.z * t[2].y + y.w * t[3].y;
            acc[a][2] += y.x * t[0].z + y.y * t[1].z + y.z * t[2].z + y.w * t[3].z;
            acc[a][3] += y.x * t[0].w + y.y * t[1].w + y.z * t[2].w + y.w * t[3].w;
        }
    }
}

// Position in the ring over the launch: chunks passed (the same count in the
// issuing warp and in every consumer) and, in the issuing warp, one past the
// last chunk whose copies it started.
struct RingState {
    uint32_t seq = 0;
    uint32_t issued = 0;
};

// Issuing warp: chunks k0 .. k1-1 of the item (phase-major), each into stage
// seq % S after the consumers have released that stage's previous use.  A wait
// that gives up records the fault and stops all further copies of the CTA.
__device__ __forceinline__ void ring_issue_range(const FusedParams& p, uint64_t r0, int m, const RingGeom& g,
                                                 uint32_t k0, uint32_t k1, uint32_t ktotal, RingState& rs,
                                                 uint32_t lane) {
    const uint32_t S = p.ring_stages;
    for (uint32_t k = k0; k < k1; ++k, ++rs.seq) {
        const uint32_t seq = rs.seq;
        if (*ring_abort()) continue;
        const uint32_t s = seq % S, round = seq / S;
        if (round >= 1) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(ring_empty(s), (round - 1u) & 1u, kRingSpinLimit);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicOr(p.faults, PIR_FAULT_WAIT_TIMEOUT);
                    *ring_abort() = 1u;
                }
                __syncwarp();
                continue;
            }
        }
        if (PIR_RING_FENCE) fence_proxy_async_smem();  // the consumers' reads of the stage before its refill
        ring_issue(p, r0, m, (k / g.nch) * g.kc, g, k % g.nch, s, lane);
        rs.issued = seq + 1u;
        const uint32_t kp = k + p.ring_prefetch;
        if (p.ring_prefetch && kp < ktotal) ring_prefetch(p, r0, m, (kp / g.nch) * g.kc, g, kp % g.nch, lane);
    }
}

// Writes this thread's last 2*kc leaf shares (rows row_base .. row_base+2kc-1)
// to the materialised share matrix.
template <int G>
__device__ __forceinline__ void store_phase(const FusedParams& p, const uint32_t* yb, uint32_t* dst, int g, int l,
                                            uint64_t row_base, uint32_t kc) {
    constexpr int SQ = kProducers / G;
    if (kc == 2 && p.shares_vec && row_base >= p.row_lo && row_base + 4 <= p.row_hi &&
        ((row_base - p.row_lo) & 3u) == 0) {
        uint4 v;
        v.x = yb[(g * 2 * kPairs + 0) * SQ + l];
        v.y = yb[(g * 2 * kPairs + 1) * SQ + l];
        v.z = yb[(g * 2 * kPairs + 2) * SQ + l];
        v.w = yb[(g * 2 * kPairs + 3) * SQ + l];
        *reinterpret_cast<uint4*>(dst + (row_base - p.row_lo)) = v;
        return;
    }
    for (uint32_t j = 0; j < 2 * kc; ++j) {
        const uint64_t row = row_base + j;
        if (row >= p.row_lo && row < p.row_hi) dst[row - p.row_lo] = yb[(g * 2 * kPairs + j) * SQ + l];
    }
}

// One work item: the queries in the header slots (set by the caller) over the
// 2^r rows starting at r0 (1 <= r <= n).  MAT = false: fused share x table product (a1-a6)
// with kConsumers consumer threads after the kProducers producers;
// MAT = true: producers only, leaf shares written to each slot's `out`.
// STAGED: a last warp copies the table rows into the shared-memory ring and the
// consumers multiply them from there; `seq` counts the ring's chunks over the
// launch (the same in the issuing warp and every consumer).
// Ends with a barrier, so shared memory is free for the next item.
template <int G, int VEC, bool MAT, bool BINS, bool STAGED = false>
__device__ __forceinline__ void run_item(const FusedParams& p, uint64_t r0, int r, RingState& rs) {
    constexpr int SQ = kProducers / G;
    constexpr int LOG_SQ = (SQ == 512) ? 9 : (SQ == 256) ? 8 : (SQ == 128) ? 7 : 6;
    constexpr int NT = MAT ? kProducers : STAGED ? kStagedThreads : kFusedThreads;
    static_assert(!STAGED || (VEC == 4 && !MAT && !BINS && G <= 4), "staged scan: 128-bit rows, fused, G <= 4");
    static_assert(G * 2 * kPairs * SQ * 2 <= kYWords, "share buffers exceed their region");
    static_assert(2 * kProducers * (int)sizeof(uint4) <= 4 * kYRegionWords, "split buffers exceed their region");
    static_assert(kMaxGroup * 512 <= kYRegionWords, "reduction of the widest supported rows exceeds its region");
    static_assert(G <= kMaxGroup, "too many query slots");

    const int tid = threadIdx.x;
    const bool producer = tid < kProducers;
    const bool issuer = STAGED && tid >= kFusedThreads;
    const uint32_t lane4 = (uint32_t)(tid & 31) << 2, lane4h = lane4 | 128u;
    uint32_t* ybuf = reinterpret_cast<uint32_t*>(sm + kYOff);
    const int n = (int)p.n;
    const int sd = min(LOG_SQ, r - 1);
    const int m = r - sd;
    const uint32_t npairs = 1u << (m - 1);
    RingGeom ring{};
    if constexpr (STAGED) ring = ring_geom(p, sd, m);
    // chunks of this item in the ring, and how many the issuing warp starts
    // before the path walk (the ring is empty between items, so those need no wait)
    const uint32_t ring_chunks = ring.on ? (npairs / ring.kc) * ring.nch : 0u;
    const uint32_t ring_early = min(ring_chunks, STAGED ? p.ring_stages : 0u);
    if (issuer && ring.on) {
        const uint32_t lane = (uint32_t)tid & 31u;
        ring_issue_range(p, r0, m, ring, 0, ring_early, ring_chunks, rs, lane);
    }
    const int nsub = 1 << sd;
    // leaf pairs per hand-off: at most kPairs, and small enough that an item has
    // four phases where it can, so that the scan of one phase overlaps the
    // expansion of the next even when an item is small
    uint32_t kc = ring.on ? ring.kc : max(1u, min((uint32_t)kPairs, npairs >> 2));
    // With one or two queries per item the table scan weighs as much as the
    // expansion: the consumers then have the copy engine prefetch the rows of
    // the phases kPfAhead ahead into L2, with phases small enough that
    // kPfAhead + 1 of every CTA's fit there; the first ones while the item's
    // path walk and split run.  (With more queries per item the rows are
    // reused G times and the prefetch only costs issue slots.)
    bool pf = false;
    if ((G <= 2 || BINS) && VEC == 4 && !MAT && !ring.on) {
        // bins mode: every slot reads its own rows, so the scan never amortises
        const uint64_t pair_bytes = (BINS ? (uint64_t)G : 1u) * nsub * 2u * p.stride * 4u;  // one leaf pair of every subtree
        while (kc > 1 && pair_bytes * kc > kPrefetchMaxBytes) kc >>= 1;
        pf = pair_bytes * kc <= kPrefetchMaxBytes;
    }
    const uint32_t nphases = npairs / kc;
    const uint32_t pf_first = pf ? min(nphases, (uint32_t)kPfAhead) : 0u;
    if (kPfEarly && pf && !producer && !issuer)
        for (uint32_t a = 0; a < pf_first; ++a)
            prefetch_rows<G, BINS>(p, r0, m, (uint32_t)nsub, a * kc, kc, (uint32_t)(tid - kProducers));

    // ---- stage the group's keys in shared memory ---------------------------
    {
        const uint32_t kw = p.key_bytes / 16u;  // key length in 16-byte words
        for (uint32_t i = tid; i < (uint32_t)G * kw; i += NT) {
            const uint32_t g = i / kw, w = i - g * kw;
            const uint8_t* key = hdr_slot((int)g)->key;
            if (key)
                reinterpret_cast<uint4*>(sm + kStackOff + g * kKeySlotBytes)[w] =
                    __ldg(reinterpret_cast<const uint4*>(key) + w);
        }
    }
    __syncthreads();

    // ---- key headers and the path to this item's range node ---------------
    uint4* bufA = reinterpret_cast<uint4*>(ybuf);
    uint4* bufB = bufA + kProducers;
    if (tid < G) {
        QueryHdr* h = hdr_slot(tid);
        uint32_t ok = 0, party = 0, cwo = 0, prf = 0;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (h->key) {
            const uint4 hw = staged_key(tid)[0];
            ok = hw.x == kKeyMagic && (hw.y & 0xffu) == kKeyVersion && ((hw.y >> 8) & 0xffu) == p.n &&
                 ((hw.y >> 16) & 0xffu) <= 1u && (hw.y >> 24) <= PIR_PRF_CHACHA20;
            if (ok) {
                party = (hw.y >> 16) & 1u;
                prf = hw.y >> 24;
                cwo = hw.z;
                v = staged_key(tid)[1];
                for (int d = 1; d <= n - r; ++d) {  // only the child on the path
                    const uint32_t b = (uint32_t)(r0 >> (n - d)) & 1u;
                    v = expand1_staged(lane4, lane4h, tid, (uint32_t)d, v, b, prf != 0);
                }
            } else if (p.status) {
                atomicOr(p.status, PIR_STATUS_BAD_KEY);
            }
        }
        h->ok = ok;
        h->party = party;
        h->cw_out = cwo;
        h->prf = prf;
        bufA[tid] = v;
    }
    __syncthreads();

    // ---- split to one subtree root per producer thread ----------------------
    for (int i = 0; i < sd; ++i) {
        const uint4* src = (i & 1) ? bufB : bufA;
        uint4* dst = (i & 1) ? bufA : bufB;
        if ((G << i) <= kPairNodes) {
            if (tid < 2 * (G << i)) {  // thread 2 node + b computes child b of node (g << i) + idx
                const int node = tid >> 1, g = node >> i;
                const uint32_t b = (uint32_t)tid & 1u;
                const uint4 v = src[node];
                const QueryHdr* h = hdr_slot(g);
                dst[2 * node + (int)b] =
                    h->ok ? expand1_staged(lane4, lane4h, g, (uint32_t)(n - r + i + 1), v, b, h->prf != 0) : v;
            }
        } else if (tid < (G << i)) {
            const int g = tid >> i, idx = tid & ((1 << i) - 1);
            const uint4 v = src[tid];
            uint4 c0 = v, c1 = v;
            const QueryHdr* h = hdr_slot(g);
            if (h->ok) expand_staged(lane4, lane4h, g, (uint32_t)(n - r + i + 1), v, h->prf != 0, c0, c1);
            dst[(g << (i + 1)) + 2 * idx] = c0;
            dst[(g << (i + 1)) + 2 * idx + 1] = c1;
        }
        __syncthreads();
    }
    const int g = producer ? tid / SQ : 0, l = producer ? tid % SQ : 0;
    const QueryHdr* hq = hdr_slot(g);
    const bool act = producer && l < nsub && hq->ok != 0;
    uint4 node = make_uint4(0, 0, 0, 0);
    if (producer && l < nsub) node = ((sd & 1) ? bufB : bufA)[(g << sd) + l];
    __syncthreads();  // share buffers alias the split buffers

    uint32_t acc[G][VEC];
#pragma unroll
    for (int a = 0; a < G; ++a)
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[a][i] = 0;

    if (producer) {
        // ---- depth-first expansion; hand over shares every kc leaf pairs ----
        const uint32_t party = hq->party, cwo = hq->cw_out;
        const bool chacha = hq->prf != 0;
        const uint8_t* key = hq->key;
        const int d0 = n - r + sd;  // depth of this thread's subtree root
        int lvl = 0;
        uint32_t k = 0, phase = 0;
        for (;;) {
            const bool leaf = lvl + 1 == m;
            uint4 c0 = node, c1 = node;
            if (act) expand(lane4, lane4h, key, (uint32_t)(d0 + lvl + 1), node, leaf, chacha, c0, c1);
            if (leaf) {
                uint32_t y0 = 0, y1 = 0;
                if (act) {
                    y0 = c0.y + (c0.x & 1u) * cwo;
                    y1 = c1.y + (c1.x & 1u) * cwo;
                    if (party) {
                        y0 = 0u - y0;
                        y1 = 0u - y1;
                    }
                }
                uint32_t* yb = ybuf + (phase & 1u) * (kYWords / 2);
                const uint32_t j = 2u * (k % kc);
                yb[(g * 2 * kPairs + j) * SQ + l] = y0;
                yb[(g * 2 * kPairs + j + 1) * SQ + l] = y1;
                ++k;
                if (k % kc == 0) {
                    if constexpr (MAT) {
                        // each thread stores only what it wrote itself: no barrier needed
                        if (hq->out && l < nsub)
                            store_phase<G>(p, yb, hq->out, g, l, r0 + ((uint64_t)l << m) + 2ull * (k - kc), kc);
                    } else {
                        bar_arrive(kBarFull + (int)(phase & 1u), kFusedThreads);
                    }
                    ++phase;
                    if constexpr (!MAT) {
                        // the next buffer was filled two phases ago: wait until it is consumed
                        if (phase >= 2 && phase < nphases) bar_sync(kBarFree + (int)(phase & 1u), kFusedThreads);
                    }
                }
                if (k == npairs) break;
                lvl = m - 1 - (__ffs((int)k) - 1);
                node = *stack_slot(lvl, tid);
            } else {
                *stack_slot(lvl + 1, tid) = c1;
                node = c0;
                ++lvl;
            }
        }
    } else if (issuer) {
        // ---- issuing warp: the rest of the item's chunks, as stages free up ----
        if (ring.on) ring_issue_range(p, r0, m, ring, ring_early, ring_chunks, ring_chunks, rs, (uint32_t)tid & 31u);
    } else if (STAGED && ring.on) {
        if constexpr (STAGED) {
            // ---- consumers, staged: every chunk of a filled buffer from its ring stage ----
            const uint32_t ct = (uint32_t)(tid - kProducers), lane = (uint32_t)tid & 31u;
            const uint32_t S = p.ring_stages;
            for (uint32_t ph = 0; ph < nphases; ++ph) {
                bar_sync(kBarFull + (int)(ph & 1u), kFusedThreads);
                const uint32_t* yb = ybuf + (ph & 1u) * (kYWords / 2);
                for (uint32_t ch = 0; ch < ring.nch; ++ch, ++rs.seq) {
                    const uint32_t st = rs.seq % S;
                    if (!*ring_abort() && !mbar_wait_bounded(ring_full(st), (rs.seq / S) & 1u, kRingSpinLimit)) {
                        if (lane == 0) atomicOr(p.faults, PIR_FAULT_WAIT_TIMEOUT);
                        *ring_abort() = 1u;
                    }
                    // after a failed wait the stages hold nothing trustworthy: keep the
                    // barriers' counts, skip the arithmetic
                    if (!*ring_abort()) mac_chunk<G>(p, yb, ring_stage(st), r0, m, ph * kc, ring, ch, acc, ct);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(ring_empty(st));
                }
                if (ph + 2 < nphases) bar_arrive(kBarFree + (int)(ph & 1u), kFusedThreads);
            }
        }
    } else if constexpr (!MAT) {
        // ---- consumers: multiply every filled buffer into the accumulators ----
        const uint32_t ct = (uint32_t)(tid - kProducers);
        if (!kPfEarly)
            for (uint32_t a = 0; a < pf_first; ++a) prefetch_rows<G, BINS>(p, r0, m, (uint32_t)nsub, a * kc, kc, ct);
        for (uint32_t ph = 0; ph < nphases; ++ph) {
            if (pf && ph + kPfAhead < nphases)
                prefetch_rows<G, BINS>(p, r0, m, (uint32_t)nsub, (ph + kPfAhead) * kc, kc, ct);
            bar_sync(kBarFull + (int)(ph & 1u), kFusedThreads);
            if constexpr (BINS)
                mac_phase_bins<G>(p, ybuf + (ph & 1u) * (kYWords / 2), r0, m, sd, ph * kc, kc, acc, ct);
            else
                mac_phase<G, VEC>(p, ybuf + (ph & 1u) * (kYWords / 2), r0, m, sd, ph * kc, kc, acc, ct);
            if (ph + 2 < nphases) bar_arrive(kBarFree + (int)(ph & 1u), kFusedThreads);
        }
    }

    __syncthreads();
    if constexpr (MAT) return;
    // ---- reduce the consumers' partial sums, then one atomic per word -------
    const uint32_t W = p.width;
    uint32_t* red = ybuf;
    for (uint32_t i = tid; i < G * W; i += NT) red[i] = 0;
    __syncthreads();
    if (issuer) {
        // the issuing warp holds no partial sums
    } else if (!producer && BINS) {
        // team g holds slot g's partial sums in acc[0]
        const uint32_t ct = (uint32_t)(tid - kProducers);
        constexpr uint32_t kTeam = kConsumers / G;
        const uint32_t g = ct / kTeam, t = ct % kTeam;
        const uint32_t nc = W / VEC, nrg = kTeam / nc;
        const uint32_t c = t % nc, rg = t / nc;
        if (rg < nrg) {
#pragma unroll
            for (int i = 0; i < VEC; ++i)
                if (acc[0][i]) atomicAdd(&red[g * W + c * VEC + i], acc[0][i]);
        }
    } else if (!producer) {
        const uint32_t ct = (uint32_t)(tid - kProducers);
        const uint32_t nc = W / VEC, nrg = kConsumers / nc;
        const uint32_t c = ct % nc, rg = ct / nc;
        if (nc < 32 && (nc & (nc - 1)) == 0) {
            // every consumer thread is in a row group; lanes lane, lane + nc, ... of a
            // warp hold the same words: add them across the warp first (mod 2^32)
            for (uint32_t off = 16; off >= nc; off >>= 1)
#pragma unroll
                for (int a = 0; a < G; ++a)
#pragma unroll
                    for (int i = 0; i < VEC; ++i) acc[a][i] += __shfl_xor_sync(0xffffffffu, acc[a][i], off);
            if ((tid & 31) < (int)nc) {
#pragma unroll
                for (int a = 0; a < G; ++a)
#pragma unroll
                    for (int i = 0; i < VEC; ++i)
                        if (acc[a][i]) atomicAdd(&red[a * W + c * VEC + i], acc[a][i]);
            }
        } else if (rg < nrg) {
#pragma unroll
            for (int a = 0; a < G; ++a)
#pragma unroll
                for (int i = 0; i < VEC; ++i)
                    if (acc[a][i]) atomicAdd(&red[a * W + c * VEC + i], acc[a][i]);
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i < G * W; i += NT) {
        const uint32_t a = i / W;
        const uint32_t v = red[i];
        uint32_t* o = hdr_slot((int)a)->out;
        if (o && v) atomicAdd(o + (i - a * W), v);
    }
    __syncthreads();
}

// q = a / b, r = a % b, in 32-bit arithmetic when both fit (the 64-bit divide
// is a long software sequence).
__device__ __forceinline__ void divmod(uint64_t a, uint64_t b, uint64_t& q, uint64_t& r) {
    if (((a | b) >> 32) == 0) {
        const uint32_t q32 = (uint32_t)a / (uint32_t)b;
        q = q32;
        r = (uint32_t)a - q32 * (uint32_t)b;
    } else {
        q = a / b;
        r = a - q * b;
    }
}

// Persistent grid over items (query group, row range), query groups fastest so
// that items running at the same time share table rows through L2.  The first
// nfull items (whole rounds of the grid) run whole; each later one is cut into
// 2^tail_log2 pieces, so that the last round keeps every CTA busy.  Pieces with
// the same index run side by side, again query groups fastest.
template <int G, int VEC, bool MAT, bool BINS, bool STAGED = false>
__device__ __forceinline__ void eval_items(const FusedParams& p) {
    if (!smem_base_ok(p.status)) return;
    RingState rs;
    if (STAGED && threadIdx.x == 0) {
        for (uint32_t st = 0; st < p.ring_stages; ++st) {
            mbar_init(ring_full(st), 1);                // the issuing lane's arrival + the copies' bytes
            mbar_init(ring_empty(st), kConsumers / 32);  // one arrival per consumer warp
        }
        *ring_abort() = 0u;
        fence_mbarrier_init();
    }  // (build_tables ends with a CTA barrier)
    // (the launch parameters are read before the tables are built, so that their
    // first constant-cache misses overlap the fill)
    const uint64_t rest = p.nitems - p.nfull;
    const uint64_t total = p.nfull + (rest << p.tail_log2);
    // rows the items cover: the evaluated rows, or a bin's rows (bins mode)
    const uint64_t lo = BINS ? 0 : p.row_lo, hi = BINS ? p.bin_rows : p.row_hi;
    build_tables(threadIdx.x);
    for (uint64_t it = blockIdx.x; it < total; it += gridDim.x) {
        uint64_t item = it, piece = 0;
        int r = (int)p.range_log2;
        if (it >= p.nfull) {
            uint64_t k;
            divmod(it - p.nfull, rest, piece, k);
            item = p.nfull + k;
            r -= (int)p.tail_log2;
        }
        uint64_t range, qg64;
        divmod(item, p.nqg, range, qg64);
        const uint32_t qg = (uint32_t)qg64;
        const uint64_t r0 = ((p.first_range + range) << p.range_log2) + (piece << r);
        if (r0 >= hi || r0 + (1ull << r) <= lo) continue;  // a piece outside the rows (uniform per CTA)
        if (threadIdx.x < G) {
            const uint32_t q = qg * G + threadIdx.x;
            QueryHdr* h = hdr_slot(threadIdx.x);
            const bool valid = q < p.batch;
            if constexpr (BINS) {  // slot = bin q: rows [q * bin_rows, min(+bin_rows, row_hi))
                const uint64_t first = (uint64_t)q * p.bin_rows;
                h->trow = valid ? p.table + first * p.stride : nullptr;
                h->rows = valid ? (p.row_hi - first < p.bin_rows ? p.row_hi - first : p.bin_rows) : 0;
            }
            h->key = valid ? p.keys + (uint64_t)q * p.key_bytes : nullptr;
            if constexpr (MAT)
                h->out = valid ? p.shares + (uint64_t)q * p.ld : nullptr;
            else
                h->out = valid ? p.out + (uint64_t)q * p.width : nullptr;
        }
        __syncthreads();
        run_item<G, VEC, MAT, BINS, STAGED>(p, r0, r, rs);
    }
    if (STAGED && threadIdx.x >= kFusedThreads && *ring_abort()) {
        // copies may still be landing after an abort: see this warp's last ones
        // in (bounded) before the CTA's shared memory goes to the next CTA
        const uint32_t S = p.ring_stages;
        const uint32_t first = rs.issued > S ? rs.issued - S : 0u;
        if ((threadIdx.x & 31) == 0)
            for (uint32_t k = first; k < rs.issued; ++k)
                mbar_wait_bounded(ring_full(k % S), (k / S) & 1u, kRingSpinLimit);
        __syncwarp();
    }
}

template <int G, int VEC>
__global__ void __launch_bounds__(kFusedThreads, 1) fused_eval_kernel(const FusedParams p) {
    eval_items<G, VEC, false, false>(p);
}

// The fused kernel with its table scan staged through shared memory by the
// bulk-copy engine (one more warp issues the copies; 128-bit rows, G <= 4).
template <int G>
__global__ void __launch_bounds__(kStagedThreads, 1) fused_eval_staged_kernel(const FusedParams p) {
    eval_items<G, 4, false, false, true>(p);
}

// Partial batch retrieval: G bins per work item, each slot with its own rows.
template <int G>
__global__ void __launch_bounds__(kFusedThreads, 1) bins_eval_kernel(const FusedParams p) {
    eval_items<G, 4, false, true>(p);
}

template <int G>
__global__ void __launch_bounds__(kProducers, 1) expand_materialise_kernel(const FusedParams p) {
    eval_items<G, 1, true, false>(p);
}

// ------------------------------------------------ many small trees, breadth first
// Expansion only, for a batch of keys over a small domain (the bins of
// partial batch retrieval).  Each key's tree is cut into 2^u units, the
// subtrees at depth u; CTA c takes units [c*upc, c*upc + upc), walks each
// unit's root down from its key's root (u levels, one block each) and then
// expands all its units together, level by level, over its 512 threads.  The
// nodes of a level lie unit-major in shared memory after the lookup tables
// (node i = unit * 2^l + j, children 2i and 2i + 1), in one of two buffers by
// the level's parity; the leaf parents write the leaf shares straight to
// shares[key * ld + leaf].  With the units spread evenly over every SM and
// each level's nodes over every thread, no work item leaves threads or SMs
// idle, as G-query items on a small tree do (1024 bins of 2^10 rows make 128
// such items for 152 SMs; as 4096 units of 2^8 leaves they make 27 per SM).
constexpr int kBfsOff = kTablesBytes;
constexpr int kBfsLastBytes = 64 * 1024;   // the leaf parents' level: up to 4096 nodes
constexpr int kBfsOtherBytes = 32 * 1024;  // the level above it: up to 2048 nodes
constexpr int kBfsHdrOff = kBfsOff + kBfsLastBytes + kBfsOtherBytes;
constexpr uint32_t kBfsMaxUnits = 64;      // units per CTA (one 16-byte header each)
constexpr uint32_t kBfsMaxLeaves = 2u * kBfsLastBytes / 16u;  // leaves per CTA
constexpr int kBfsSmemBytes = kBfsHdrOff + 16 * (int)kBfsMaxUnits;
static_assert(kBfsSmemBytes <= 232448, "dynamic shared memory above the 227 KiB a CTA may use");
static_assert(kBfsMaxLeaves / 4u * 16u <= (uint32_t)kBfsOtherBytes, "the level above the leaf parents fits");

struct BfsParams {
    const uint8_t* keys;
    uint32_t key_bytes;
    uint32_t n;      // tree levels of every key
    uint32_t u;      // unit depth: 2^u units per key, 0 <= u < n
    uint32_t nunits; // keys << u
    uint32_t upc;    // units per CTA
    uint32_t* shares;
    uint64_t ld;     // shares[key * ld + j]
    uint64_t rows;   // leaves j < rows are written
    uint32_t vec2;   // shares 8-byte aligned and ld even: leaf pairs as one 8-byte store
    uint32_t* status;
};

// Child b of v at depth d (1-based) of `key` in global memory: PRF plus the
// codeword C_{lsb(v)}[b][d].
__device__ __forceinline__ uint4 expand1(uint32_t lane4, uint32_t lane4h, const uint8_t* key, uint32_t d, uint4 v,
                                         uint32_t b, bool chacha) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(key + PIR_KEY_HEADER_BYTES + 64u * (d - 1) +
                                                         32u * (v.x & 1u) + 16u * b));
    uint4 c;
    if (chacha) {
        uint4 c0, c1;
        prf2_chacha(v, c0, c1);
        c = b ? c1 : c0;
    } else {
        c = prf1(lane4, lane4h, v, b);
    }
    return xor4(c, w);
}

// The expansion of a BFS CTA's units.  KEEP: the leaf shares stay in shared
// memory at yleaf[unit * 2^(n-u) + leaf] (unit-major), instead of going to
// p.shares; the level above the leaf parents, where yleaf lies, is free by
// then.  Ends with the leaf parents' loop (no barrier after it).
template <bool KEEP>
__device__ __forceinline__ void bfs_expand(const BfsParams& p, uint32_t* yleaf) {
    const int tid = threadIdx.x;
    const uint32_t lane4 = (uint32_t)(tid & 31) << 2, lane4h = lane4 | 128u;
    const uint32_t t0 = blockIdx.x * p.upc;
    const uint32_t nt = min(p.upc, p.nunits - t0);
    const int n = (int)p.n, u = (int)p.u, h = n - u;  // levels below a unit's root
    uint4* hdr = reinterpret_cast<uint4*>(sm + kBfsHdrOff);  // per unit: its key's ok, party, cw_out, PRF
    uint4* const buf_last = reinterpret_cast<uint4*>(sm + kBfsOff);
    uint4* const buf_other = reinterpret_cast<uint4*>(sm + kBfsOff + kBfsLastBytes);
    auto level = [&](int l) { return ((l ^ (h - 1)) & 1) ? buf_other : buf_last; };
    auto key_of = [&](uint32_t t) { return p.keys + (uint64_t)((t0 + t) >> u) * p.key_bytes; };
    build_tables(tid);  // ends with a CTA barrier

    // ---- headers and unit roots: u levels down from the key's root ----------
    for (uint32_t t = (uint32_t)tid; t < nt; t += kProducers) {
        const uint4* key = reinterpret_cast<const uint4*>(key_of(t));
        const uint4 hw = __ldg(key);
        const uint32_t ok = hw.x == kKeyMagic && (hw.y & 0xffu) == kKeyVersion && ((hw.y >> 8) & 0xffu) == p.n &&
                            ((hw.y >> 16) & 0xffu) <= 1u && (hw.y >> 24) <= PIR_PRF_CHACHA20;
        if (!ok && p.status) atomicOr(p.status, PIR_STATUS_BAD_KEY);
        hdr[t] = make_uint4(ok, (hw.y >> 16) & 1u, hw.z, hw.y >> 24);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (ok) {
            v = __ldg(key + 1);
            const uint32_t path = (t0 + t) & ((1u << u) - 1u);
            for (int d = 1; d <= u; ++d)  // only the child on the path
                v = expand1(lane4, lane4h, key_of(t), (uint32_t)d, v, (path >> (u - d)) & 1u, (hw.y >> 24) != 0);
        }
        level(0)[t] = v;
    }
    __syncthreads();

    // ---- internal levels below the unit roots: level l -> l + 1 -------------
    for (int l = 0; l + 1 < h; ++l) {
        const uint4* src = level(l);
        uint4* dst = level(l + 1);
        const uint32_t cnt = nt << l;
        const uint32_t depth = (uint32_t)(u + l + 1);  // of the children
        if (cnt <= (uint32_t)kProducers / 2) {
            // few nodes: a thread per child, one AES block each (the level's latency)
            if ((uint32_t)tid < 2u * cnt) {
                const uint32_t i = (uint32_t)tid >> 1, b = (uint32_t)tid & 1u, t = i >> l;
                const uint4 hd = hdr[t], v = src[i];
                dst[2u * i + b] = hd.x ? expand1(lane4, lane4h, key_of(t), depth, v, b, hd.w != 0) : v;
            }
        } else {
            for (uint32_t i = (uint32_t)tid; i < cnt; i += kProducers) {
                const uint32_t t = i >> l;
                const uint4 hd = hdr[t], v = src[i];
                uint4 c0 = v, c1 = v;
                if (hd.x) expand(lane4, lane4h, key_of(t), depth, v, false, hd.w != 0, c0, c1);
                dst[2u * i] = c0;
                dst[2u * i + 1u] = c1;
            }
        }
        __syncthreads();
    }

    // ---- leaf parents -> leaf shares, y = (-1)^party (word1 + lsb * cw_out) --
    const uint4* src = level(h - 1);
    const uint32_t cnt = nt << (h - 1);
    const uint32_t jmask = (1u << (h - 1)) - 1u;
    for (uint32_t i = (uint32_t)tid; i < cnt; i += kProducers) {
        const uint32_t t = i >> (h - 1), g = t0 + t;
        // leaf within the key: the unit's first leaf plus this pair's offset
        const uint64_t j = ((uint64_t)(g & ((1u << u) - 1u)) << h) + 2ull * (i & jmask);
        const uint4 hd = hdr[t];
        uint32_t y0 = 0, y1 = 0;
        if (hd.x) {
            uint4 c0, c1;
            expand(lane4, lane4h, key_of(t), (uint32_t)n, src[i], true, hd.w != 0, c0, c1);
            y0 = c0.y + (c0.x & 1u) * hd.z;
            y1 = c1.y + (c1.x & 1u) * hd.z;
            if (hd.y) {
                y0 = 0u - y0;
                y1 = 0u - y1;
            }
        }
        if constexpr (KEEP) {
            const uint32_t l = (i & jmask) * 2u;
            yleaf[(t << h) + l] = y0;
            yleaf[(t << h) + l + 1u] = y1;
            continue;
        }
        uint32_t* dst = p.shares + (uint64_t)(g >> u) * p.ld + j;
        if (j + 1 < p.rows) {
            if (p.vec2)
                *reinterpret_cast<uint2*>(dst) = make_uint2(y0, y1);
            else {
                dst[0] = y0;
                dst[1] = y1;
            }
        } else if (j < p.rows) {
            dst[0] = y0;
        }
    }
}

__global__ void __launch_bounds__(kProducers, 1) expand_bfs_kernel(const BfsParams p) {
    if (!smem_base_ok(p.status)) return;
    bfs_expand<false>(p, nullptr);
}

// ------------------------------- partial batch retrieval: expansion, then rows
// The breadth-first expansion above with the leaf shares kept in shared
// memory, followed in the same CTA by the product with the table rows of its
// own units (Sec. 4, batch PIR: a bin's rows meet only its own query).  A
// unit's rows are one contiguous run of the dense table; the CTA brings them
// in, in pieces of at most kPbrStageBytes, by bulk copies into a ring laid
// over the lookup tables (no longer needed), multiplies each row by its
// unit's leaf share, and adds its sums into the bin's output words when the
// bin changes (a bin's units are consecutive).  No share vector reaches HBM
// (Sec. 3.2.4).  Every wait is bounded; one that gives up sets
// PIR_FAULT_WAIT_TIMEOUT and the CTA skips the rest of its products.  (The
// two phases do not overlap: every CTA expands, then every CTA reads, so the
// step costs the expansion plus one streaming pass over the table.  An L2
// prefetch of each CTA's first rows during the expansion measured slower.)
constexpr uint32_t kPbrStageBytes = 32 * 1024;
constexpr uint32_t kPbrStages = (uint32_t)kTablesBytes / kPbrStageBytes;
constexpr int kPbrBarOff = kBfsSmemBytes;  // kPbrStages full barriers
constexpr int kPbrAbortOff = kPbrBarOff + 8 * (int)kPbrStages;
constexpr int kPbrSmemBytes = kPbrAbortOff + 16;
constexpr uint32_t kPbrSpinLimit = 1u << 22;
static_assert(kPbrStages >= 2 && kPbrStages * kPbrStageBytes <= (uint32_t)kTablesBytes, "ring over the tables");
static_assert(kPbrSmemBytes <= 232448, "dynamic shared memory above the 227 KiB a CTA may use");
static_assert(kBfsOff == kTablesBytes && kBfsLastBytes >= 4 * 2048, "reduction buffer in the leaf parents' level");

struct PbrParams {
    BfsParams b;
    const uint32_t* table;  // dense rows: row j at table + j * width
    uint64_t table_rows;
    uint64_t bin_rows;      // bin k: rows [k * bin_rows, k * bin_rows + bin_rows)
    uint32_t width;         // words, a multiple of 4, at most 2048
    uint32_t rpp;           // rows per piece (a piece is at most kPbrStageBytes)
    uint32_t ppu;           // pieces per unit: ceil(2^(n-u) / rpp)
    uint32_t* out;          // nbins x width words, accumulated into (zeroed by the caller)
    uint32_t* faults;       // the library's device fault word
};

struct PbrPiece {
    uint64_t row0;  // first table row
    uint32_t rows;  // rows to copy and multiply (0 past the bin or the table)
    uint32_t t;     // unit of the CTA
    uint32_t leaf;  // unit-relative leaf of row0
};

// Piece k of the CTA whose first unit is t0.
__device__ __forceinline__ PbrPiece pbr_piece(const PbrParams& p, uint32_t t0, uint32_t k) {
    const uint32_t h = p.b.n - p.b.u;
    const uint32_t t = k / p.ppu, pi = k - t * p.ppu;
    const uint32_t g = t0 + t;
    const uint64_t key = g >> p.b.u;
    const uint32_t leaf = pi * p.rpp;
    const uint64_t j0 = ((uint64_t)(g & ((1u << p.b.u) - 1u)) << h) + leaf;  // bin-relative row
    uint64_t rows = min((uint64_t)p.rpp, (uint64_t)((1ull << h) - leaf));
    rows = j0 < p.bin_rows ? min(rows, p.bin_rows - j0) : 0;
    const uint64_t row0 = key * p.bin_rows + j0;
    rows = row0 < p.table_rows ? min(rows, p.table_rows - row0) : 0;
    return PbrPiece{row0, (uint32_t)rows, t, leaf};
}

__global__ void __launch_bounds__(kProducers, 1) pbr_bfs_scan_kernel(const PbrParams p) {
    if (!smem_base_ok(p.b.status)) return;
    const int tid = threadIdx.x;
    const uint32_t t0 = blockIdx.x * p.b.upc;
    const uint32_t nt = min(p.b.upc, p.b.nunits - t0);
    const uint32_t npieces = nt * p.ppu;
    const uint32_t h = p.b.n - p.b.u;
    const uint32_t W = p.width;
    const uint32_t bar0 = smem_addr(sm + kPbrBarOff);
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(sm + kPbrAbortOff);
    if (tid == 0) {
        for (uint32_t st = 0; st < kPbrStages; ++st) mbar_init(bar0 + 8u * st, 1u);
        *abort_flag = 0u;
        fence_mbarrier_init();
    }
    uint32_t* yleaf = reinterpret_cast<uint32_t*>(sm + kBfsOff + kBfsLastBytes);
    bfs_expand<true>(p.b, yleaf);  // (its table set-up ends with a CTA barrier: the mbarriers are visible)

    // ---- the CTA's rows: a ring of kPbrStages pieces over the lookup tables ----
    fence_proxy_async_smem();  // the tables' generic accesses before the copies overwrite them
    __syncthreads();           // ... and every leaf share is in yleaf
    uint32_t issued = 0;  // pieces copies were started for (thread 0)
    auto issue = [&](uint32_t k) {
        issued = k + 1;
        const PbrPiece pc = pbr_piece(p, t0, k);
        const uint32_t st = k % kPbrStages, bytes = pc.rows * W * 4u;
        mbar_expect_tx(bar0 + 8u * st, bytes);
        if (bytes) bulk_g2s(smem_addr(sm + st * kPbrStageBytes), p.table + pc.row0 * W, bytes, bar0 + 8u * st);
    };
    if (tid == 0)
        for (uint32_t k = 0; k < min(kPbrStages, npieces); ++k) issue(k);
    const uint32_t nc = W / 4u, nrg = (uint32_t)kProducers / nc;
    const uint32_t c = (uint32_t)tid % nc, rg = (uint32_t)tid / nc;
    const bool active = rg < nrg;
    uint32_t* red = reinterpret_cast<uint32_t*>(sm + kBfsOff);  // the leaf parents' level: free now
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
    // this thread's sums into the bin's output words (every thread of the CTA)
    auto flush = [&](uint64_t key) {
        for (uint32_t i = (uint32_t)tid; i < W; i += kProducers) red[i] = 0u;
        __syncthreads();
        if (nc < 32 && (nc & (nc - 1)) == 0) {  // lanes lane, lane + nc, ... hold the same words
            for (uint32_t off = 16; off >= nc; off >>= 1)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
            if (((uint32_t)tid & 31u) < nc)
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (acc[i]) atomicAdd(&red[c * 4u + i], acc[i]);
        } else if (active) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (acc[i]) atomicAdd(&red[c * 4u + i], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = 0u;
        __syncthreads();
        for (uint32_t i = (uint32_t)tid; i < W; i += kProducers)
            if (red[i]) atomicAdd(p.out + key * W + i, red[i]);
        __syncthreads();  // red is cleared again by the next flush
    };
    uint64_t cur = (uint64_t)t0 >> p.b.u;
    for (uint32_t k = 0; k < npieces; ++k) {
        const PbrPiece pc = pbr_piece(p, t0, k);
        const uint64_t key = (uint64_t)(t0 + pc.t) >> p.b.u;
        if (key != cur) {  // uniform: every thread walks the same pieces
            flush(cur);
            cur = key;
        }
        const uint32_t st = k % kPbrStages;
        if (!*abort_flag && !mbar_wait_bounded(bar0 + 8u * st, (k / kPbrStages) & 1u, kPbrSpinLimit)) {
            if (tid == 0) atomicOr(p.faults, PIR_FAULT_WAIT_TIMEOUT);
            *abort_flag = 1u;
        }
        if (!*abort_flag && active && pc.rows) {
            const char* stage = sm + st * kPbrStageBytes;
            const uint32_t* ys = yleaf + (pc.t << h) + pc.leaf;
            for (uint32_t rr = rg; rr < pc.rows; rr += nrg) {
                const uint4 v = *reinterpret_cast<const uint4*>(stage + (rr * W + c * 4u) * 4u);
                const uint32_t y = ys[rr];
                acc[0] += y * v.x;
                acc[1] += y * v.y;
                acc[2] += y * v.z;
                acc[3] += y * v.w;
            }
        }
        fence_proxy_async_smem();  // these reads before the next copy into the stage
        __syncthreads();
        if (tid == 0 && !*abort_flag && k + kPbrStages < npieces) issue(k + kPbrStages);
    }
    flush(cur);
    if (tid == 0 && *abort_flag) {
        // copies still landing after a wait gave up: see the last one of each stage
        // in (bounded; its phase is the stage's last, so a finished one reads as such)
        for (uint32_t k = issued > kPbrStages ? issued - kPbrStages : 0u; k < issued; ++k)
            mbar_wait_bounded(bar0 + 8u * (k % kPbrStages), (k / kPbrStages) & 1u, kPbrSpinLimit);
    }
}


// Many tables of different sizes and widths in one launch.  Items are
// (table, row range, up to 8 queries of that table); CTAs take the next item
// from a counter, so uneven items balance themselves.
template <int VEC>
__global__ void __launch_bounds__(kFusedThreads, 1) multi_eval_kernel(const MultiParams mp) {
    if (!smem_base_ok(mp.status)) return;
    build_tables(threadIdx.x);
    uint64_t* s_item = reinterpret_cast<uint64_t*>(sm + kItemOff);
    for (;;) {
        if (threadIdx.x == 0) *s_item = atomicAdd(reinterpret_cast<unsigned long long*>(mp.counter), 1ull);
        __syncthreads();
        const uint64_t it = *s_item;  // every thread reads it before run_item's first barrier
        if (it >= mp.nitems) break;
        const MultiItem& w = mp.items[it];
        const MultiTable& tb = mp.tables[w.table];
        FusedParams p{};
        p.table = tb.data;
        p.row_lo = 0;
        p.row_hi = tb.rows;
        p.stride = tb.stride;
        p.status = mp.status;
        p.key_bytes = tb.key_bytes;
        p.width = tb.width;
        p.n = tb.n;
        p.range_log2 = tb.range_log2;
        if (threadIdx.x < kMaxGroup) {
            const uint32_t q = w.q[threadIdx.x];
            QueryHdr* h = hdr_slot(threadIdx.x);
            h->key = q != kNoQuery ? mp.keys + mp.key_off[q] : nullptr;
            h->out = q != kNoQuery ? mp.out + mp.out_off[q] : nullptr;
        }
        __syncthreads();
        const uint64_t r0 = w.range << tb.range_log2;
        const int r = (int)tb.range_log2;
        RingState rs;  // (no ring here)
        switch (w.group) {  // uniform over the CTA
            case 1: run_item<1, VEC, false, false>(p, r0, r, rs); break;
            case 2: run_item<2, VEC, false, false>(p, r0, r, rs); break;
            case 4: run_item<4, VEC, false, false>(p, r0, r, rs); break;
            default: run_item<kMaxGroup, VEC, false, false>(p, r0, r, rs); break;
        }
    }
}

// Sets a kernel's dynamic shared memory limit once per device (the attribute
// is per function and device; setting it costs ~1 us, a launch-path cost worth
// avoiding for latency-bound single queries).  Thread-safe: setting it twice
// is harmless.
// A device reset drops the attribute: a launch refused after the attribute
// was recorded as set sets it again (force) and retries once (a refused launch
// enqueues nothing).
template <typename Kern>
cudaError_t smem_attribute_once(Kern kern, int bytes, bool force = false) {
    static std::atomic<uint64_t> done{0};  // one bit per device, per kernel
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (!force && bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

template <typename Kern>
cudaError_t launch_kernel(Kern kern, const FusedParams& p, uint32_t ctas, int threads, cudaStream_t s) {
    cudaError_t e = smem_attribute_once(kern, kSmemBytes);
    if (e != cudaSuccess) return e;
    kern<<<ctas, threads, kSmemBytes, s>>>(p);
    e = cudaGetLastError();
    if (e == cudaErrorInvalidValue) {
        e = smem_attribute_once(kern, kSmemBytes, true);
        if (e != cudaSuccess) return e;
        kern<<<ctas, threads, kSmemBytes, s>>>(p);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace dev

// ------------------------------------------------------------------ host side

// The lookups' immediate offsets assume the shared window reserves kSmemBase
// bytes per block ahead of the kernel's own shared memory.
static bool reserved_smem_ok() {
    static int cached[64] = {};  // 0 unknown, 1 ok, 2 not
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (!cached[dev]) {
        int r = -1;
        if (cudaDeviceGetAttribute(&r, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) return false;
        cached[dev] = r == (int)dev::kSmemBase ? 1 : 2;
    }
    return cached[dev] == 1;
}

int device_sm_count() {
    static std::atomic<int> cached[64] = {};  // per device; the SM count of a device never changes
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64 && (sms = cached[dev].load(std::memory_order_relaxed)) > 0) return sms;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64) cached[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

static int log_sq(uint32_t group) {
    const int sq = dev::kProducers / (int)group;
    int l = 0;
    while ((1 << l) < sq) ++l;
    return l;
}

static uint64_t items_for(uint64_t row_lo, uint64_t rows, uint32_t r, uint32_t nqg) {
    if (rows == 0) return 0;
    const uint64_t first = row_lo >> r, last = (row_lo + rows - 1) >> r;
    return (last - first + 1) * nqg;
}

// Rows per work item.  An item costs about n dependent PRF levels of latency
// (the path walk, the split and the subtree depth, each level a few hundred
// cycles that the SM cannot fill) plus its G x 2^r tree nodes of throughput
// work; a CTA runs its items one after another.  Pick r minimising
//   ceil(items / CTAs) x (n x kLevelNodes + G x 2^r),
// kLevelNodes being one level's latency in units of one node's work at the
// SM's full rate (~0.75 us against ~5.9 ns, measured on GB300).
//
// With static round-robin over C = min(items, SMs) CTAs, floor(items / C)
// whole rounds leave items mod C for a last round in which the other CTAs
// idle.  Cut into 2^s pieces of 2^(r-s) rows, those items spread over every
// CTA at the price of one more path walk per piece:
//   floor(items / C) x (n x kLevelNodes + G x 2^r)
//     + ceil((items mod C) x 2^s / C) x (n x kLevelNodes + G x 2^(r-s)).
constexpr uint64_t kLevelNodes = 130;
constexpr int kMaxTailLog2 = 3;
static double schedule_cost(uint64_t items, int sms, uint32_t n, uint32_t g, int r, int s) {
    if (items == 0) return 0.0;
    const uint64_t c = std::min<uint64_t>(items, (uint64_t)sms);
    const double lat = (double)n * (double)kLevelNodes;
    const uint64_t whole = s > 0 ? items / c : (items + c - 1) / c;
    const uint64_t cut = s > 0 ? items - whole * c : 0;
    const uint64_t tail_rounds = ((cut << s) + c - 1) / c;
    return (double)whole * (lat + (double)g * (double)(1ull << r)) +
           (double)tail_rounds * (lat + (double)g * (double)(1ull << (r - s)));
}
static int pick_tail_log2(uint64_t items, int sms, uint32_t n, uint32_t g, int r) {
    int best = 0;
    double best_cost = schedule_cost(items, sms, n, g, r, 0);
    for (int s = 1; s <= std::min(kMaxTailLog2, r - 1); ++s) {
        const double cost = schedule_cost(items, sms, n, g, r, s);
        if (cost < best_cost) {
            best_cost = cost;
            best = s;
        }
    }
    return best;
}
static int pick_range_log2(uint64_t row_lo, uint64_t rows, uint32_t n, uint32_t g, uint32_t nqg, int r_min, int r_max,
                           int sms, bool tail) {
    int best = r_max;
    double best_cost = -1.0;
    for (int r = r_max; r >= r_min; --r) {
        const uint64_t items = items_for(row_lo, rows, (uint32_t)r, nqg);
        const int s = tail ? pick_tail_log2(items, sms, n, g, r) : 0;
        const double cost = schedule_cost(items, sms, n, g, r, s);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = r;
        }
    }
    return best;
}

uint32_t plan_tail_log2(uint64_t row_lo, uint64_t rows, uint32_t n, uint32_t group, uint32_t batch,
                        uint32_t range_log2) {
    const uint32_t nqg = (batch + group - 1) / group;
    const uint64_t items = items_for(row_lo, rows, range_log2, nqg);
    return (uint32_t)pick_tail_log2(items, std::max(1, device_sm_count()), n, group, (int)range_log2);
}

// Ring stages of a staged launch of this plan: the DFS stack levels that its
// subtrees (at most 2^m rows deep, the whole items' depth) and its staged keys
// leave free, at most kRingMaxStages.
static int ring_stages_for(const pir_plan& plan) {
    const int r = (int)plan.range_log2;
    const int m = r - std::min(log_sq(plan.group), r - 1);
    const int key_levels =
        (int)((plan.group * (uint32_t)dev::kKeySlotBytes + dev::kRingStageBytes - 1) / dev::kRingStageBytes);
    return std::min(dev::kRingMaxStages, dev::kStackLevels - std::max(m - 1, key_levels));
}

int plan_check_staged(const pir_plan& plan, uint32_t n, uint32_t width, uint64_t stride, bool vec_ok) {
    const int rc = plan_check(plan, n, width, vec_ok);
    if (rc != PIR_OK) return rc;
    if (plan.vec != 4 || plan.group > 4 || stride > dev::kRingMaxStride || ring_stages_for(plan) < 2)
        return PIR_ERR_UNSUPPORTED;
    return PIR_OK;
}

int plan_check(const pir_plan& plan, uint32_t n, uint32_t width, bool vec_ok) {
    if (plan.group != 1 && plan.group != 2 && plan.group != 4 && plan.group != 8) return PIR_ERR_UNSUPPORTED;
    if (plan.vec != 1 && plan.vec != 4) return PIR_ERR_UNSUPPORTED;
    if (plan.vec == 4 && (!vec_ok || width % 4 != 0)) return PIR_ERR_UNSUPPORTED;
    if (width == 0 || width / plan.vec > (uint32_t)dev::kMaxChunks) return PIR_ERR_UNSUPPORTED;
    if ((uint64_t)plan.group * width > (uint64_t)dev::kYRegionWords) return PIR_ERR_UNSUPPORTED;
    const int r = (int)plan.range_log2;
    if (r < 1 || r > (int)n) return PIR_ERR_UNSUPPORTED;
    const int sd = std::min(log_sq(plan.group), r - 1);
    if (r - sd > dev::kMaxDfsDepth) return PIR_ERR_UNSUPPORTED;
    if (plan.tail_log2 > (uint32_t)std::min(kMaxTailLog2, r - 1)) return PIR_ERR_UNSUPPORTED;
    return PIR_OK;
}

// The planner is a pure function of its arguments; evaluations of one shape
// on the latency-bound path (a lone query per call) reuse its answer.
int plan_fused(uint64_t rows, uint64_t row_lo, uint32_t n, uint32_t width, uint32_t batch, bool vec_ok,
               pir_plan* plan) {
    using Key = std::tuple<int, uint64_t, uint64_t, uint32_t, uint32_t, uint32_t, bool>;
    static std::mutex mu;
    static std::map<Key, pir_plan> memo;
    const int sms = std::max(1, device_sm_count());
    const Key key{sms, rows, row_lo, n, width, batch, vec_ok};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = memo.find(key);
        if (it != memo.end()) {
            *plan = it->second;
            return PIR_OK;
        }
    }
    const int rc = plan_fused_sms(rows, row_lo, n, width, batch, vec_ok, sms, plan);
    if (rc == PIR_OK) {
        std::lock_guard<std::mutex> lock(mu);
        if (memo.size() >= 4096) memo.clear();
        memo.emplace(key, *plan);
    }
    return rc;
}

int plan_fused_sms(uint64_t rows, uint64_t row_lo, uint32_t n, uint32_t width, uint32_t batch, bool vec_ok, int sms,
                   pir_plan* plan) {
    if (width == 0 || batch == 0 || n == 0 || sms < 1) return PIR_ERR_ARG;
    pir_plan pl{};
    pl.vec = (vec_ok && width % 4 == 0) ? 4 : 1;
    if (width / pl.vec > (uint32_t)dev::kMaxChunks) return PIR_ERR_UNSUPPORTED;
    uint32_t g = 8;
    while (g > 1 && (g > batch || (uint64_t)g * width > (uint64_t)dev::kYRegionWords)) g >>= 1;
    if ((uint64_t)g * width > (uint64_t)dev::kYRegionWords) return PIR_ERR_UNSUPPORTED;
    pl.group = g;
    const uint32_t nqg = (batch + g - 1) / g;
    const int lsq = log_sq(g);
    // subtrees at most kMaxDfsDepth deep; below r = log2(512/G) + 1 fewer than all producers
    // get a subtree, which a latency-bound item (one query, a small table) can afford
    const int r = pick_range_log2(row_lo, rows, n, g, nqg, 1, std::min((int)n, lsq + dev::kMaxDfsDepth), sms, true);
    pl.range_log2 = (uint32_t)r;
    const uint64_t items = items_for(row_lo, rows, (uint32_t)r, nqg);
    pl.tail_log2 = (uint32_t)pick_tail_log2(items, sms, n, g, r);
    pl.ctas = (uint32_t)std::min<uint64_t>(items, (uint64_t)sms);
    *plan = pl;
    return PIR_OK;
}

static dev::FusedParams make_params(const EvalRequest& req, const pir_plan& plan) {
    dev::FusedParams p{};
    p.table = req.table;
    p.row_lo = req.row_lo;
    p.row_hi = req.row_hi;
    p.stride = req.stride;
    p.first_range = req.row_lo >> plan.range_log2;
    p.keys = req.dkeys;
    p.out = req.dout;
    p.status = req.dstatus;
    p.key_bytes = (uint32_t)key_bytes(req.n);
    p.width = req.width;
    p.batch = req.batch;
    p.n = req.n;
    p.range_log2 = plan.range_log2;
    p.nqg = (req.batch + plan.group - 1) / plan.group;
    p.nitems = items_for(req.row_lo, req.row_hi - req.row_lo, plan.range_log2, p.nqg);
    // whole rounds of the grid run whole items; the rest are cut into pieces
    const uint64_t c = std::min<uint64_t>(p.nitems, (uint64_t)std::max(1, device_sm_count()));
    p.tail_log2 = plan.tail_log2;
    p.nfull = plan.tail_log2 && c ? p.nitems / c * c : p.nitems;
    return p;
}

static uint32_t grid_for(uint64_t items) {
    const int sms = std::max(1, device_sm_count());
    return (uint32_t)std::min<uint64_t>(items, (uint64_t)sms);
}

// Many small trees: the batch's keys, cut into 2^u units each, spread evenly
// over up to one CTA per SM, every CTA expanding its units breadth first
// (expand_bfs_kernel).  PIR_ERR_UNSUPPORTED where a CTA would hold more than
// kBfsMaxUnits units or kBfsMaxLeaves leaves for every u, or the rows do not
// start at the domain's first leaf.
// The breadth-first kernels' cut of `batch` trees of n levels: unit depth u
// with the fewest leaves on the busiest CTA (ties: the smaller u, fewer path
// walks), within the CTA's level buffers and header slots.  False when no u fits.
static bool bfs_cut(uint32_t batch, uint32_t n, int* u_out, uint64_t* upc_out) {
    if (batch == 0 || n == 0 || n > 31) return false;
    const uint64_t sms = (uint64_t)std::max(1, device_sm_count());
    int best_u = -1;
    uint64_t best_upc = 0, best_load = ~0ull;
    for (int u = 0; u <= std::min(3, (int)n - 1); ++u) {
        const uint64_t units = (uint64_t)batch << u;
        const uint64_t upc = (units + std::min(units, sms) - 1) / std::min(units, sms);
        const uint64_t load = upc << (n - u);  // leaves of the busiest CTA
        if (upc > dev::kBfsMaxUnits || load > dev::kBfsMaxLeaves || units > 0xffffffffull) continue;
        if (load < best_load) {
            best_load = load;
            best_u = u;
            best_upc = upc;
        }
    }
    *u_out = best_u;
    *upc_out = best_upc;
    return best_u >= 0;
}

static int launch_expand_bfs(const EvalRequest& req, uint32_t* shares, uint64_t ld, cudaStream_t s) {
    if (req.row_lo != 0) return PIR_ERR_UNSUPPORTED;
    int best_u = -1;
    uint64_t best_upc = 0;
    if (!bfs_cut(req.batch, req.n, &best_u, &best_upc)) return PIR_ERR_UNSUPPORTED;
    dev::BfsParams p{};
    p.keys = req.dkeys;
    p.key_bytes = (uint32_t)key_bytes(req.n);
    p.n = req.n;
    p.u = (uint32_t)best_u;
    p.nunits = req.batch << best_u;
    p.upc = (uint32_t)best_upc;
    p.shares = shares;
    p.ld = ld;
    p.rows = req.row_hi;
    p.vec2 = ((reinterpret_cast<uintptr_t>(shares) & 7u) == 0 && ld % 2 == 0) ? 1u : 0u;
    p.status = req.dstatus;
    const uint32_t ctas = (uint32_t)((p.nunits + best_upc - 1) / best_upc);
    cudaError_t e = dev::smem_attribute_once(dev::expand_bfs_kernel, dev::kBfsSmemBytes);
    for (int attempt = 0; e == cudaSuccess && attempt < 2; ++attempt) {
        dev::expand_bfs_kernel<<<ctas, dev::kProducers, dev::kBfsSmemBytes, s>>>(p);
        e = cudaGetLastError();
        if (e != cudaErrorInvalidValue || attempt > 0) break;
        e = dev::smem_attribute_once(dev::expand_bfs_kernel, dev::kBfsSmemBytes, true);  // after a reset
    }
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "expand_bfs launch");
}

// Partial batch retrieval in one launch (pbr_bfs_scan_kernel).  Clears dout
// first.  PIR_ERR_UNSUPPORTED unless the table is dense (stride == width), its
// rows 16-byte multiples of at most 2048 words, and the bins' trees fit the
// breadth-first cut.
int launch_pbr_fused(const uint32_t* table, uint64_t rows, uint32_t width, uint64_t stride, uint64_t bin_rows,
                     uint32_t n, const uint8_t* dkeys, uint32_t nbins, uint32_t* dout, uint32_t* dstatus,
                     void* stream) {
    if (!reserved_smem_ok()) return PIR_ERR_UNSUPPORTED;
    if (stride != width || width % 4 != 0 || width > 2048 || (reinterpret_cast<uintptr_t>(table) & 15u) != 0)
        return PIR_ERR_UNSUPPORTED;
    int u = -1;
    uint64_t upc = 0;
    if (!bfs_cut(nbins, n, &u, &upc)) return PIR_ERR_UNSUPPORTED;
    uint32_t* faults = device_fault_word();
    if (!faults) return cuda_fail((int)cudaGetLastError(), "device fault word");
    dev::PbrParams p{};
    p.b.keys = dkeys;
    p.b.key_bytes = (uint32_t)key_bytes(n);
    p.b.n = n;
    p.b.u = (uint32_t)u;
    p.b.nunits = nbins << u;
    p.b.upc = (uint32_t)upc;
    p.b.rows = bin_rows;
    p.b.status = dstatus;
    const uint32_t h = n - (uint32_t)u;
    p.table = table;
    p.table_rows = rows;
    p.bin_rows = bin_rows;
    p.width = width;
    p.rpp = (uint32_t)std::min<uint64_t>(std::max<uint32_t>(1u, dev::kPbrStageBytes / (width * 4u)), 1ull << h);
    p.ppu = (uint32_t)(((1ull << h) + p.rpp - 1) / p.rpp);
    p.out = dout;
    p.faults = faults;
    const uint32_t ctas = (uint32_t)((p.b.nunits + upc - 1) / upc);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(dout, 0, (uint64_t)nbins * width * sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail((int)e, "memset shares");
    e = dev::smem_attribute_once(dev::pbr_bfs_scan_kernel, dev::kPbrSmemBytes);
    for (int attempt = 0; e == cudaSuccess && attempt < 2; ++attempt) {
        dev::pbr_bfs_scan_kernel<<<ctas, dev::kProducers, dev::kPbrSmemBytes, s>>>(p);
        e = cudaGetLastError();
        if (e != cudaErrorInvalidValue || attempt > 0) break;
        e = dev::smem_attribute_once(dev::pbr_bfs_scan_kernel, dev::kPbrSmemBytes, true);  // after a reset
    }
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "pbr_bfs_scan launch");
}

int launch_materialise(const EvalRequest& req, const pir_plan& plan, uint32_t* shares, uint64_t ld, void* stream) {
    if (!reserved_smem_ok()) return PIR_ERR_UNSUPPORTED;
    {
        const int rc = launch_expand_bfs(req, shares, ld, reinterpret_cast<cudaStream_t>(stream));
        if (rc != PIR_ERR_UNSUPPORTED) return rc;
    }
    dev::FusedParams p = make_params(req, plan);
    p.shares = shares;
    p.ld = ld;
    p.shares_vec = ((reinterpret_cast<uintptr_t>(shares) & 15u) == 0 && ld % 4 == 0) ? 1u : 0u;
    if (p.nitems == 0) return PIR_OK;
    const uint32_t ctas = grid_for(p.nitems);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (plan.group) {
        case 1: e = dev::launch_kernel(dev::expand_materialise_kernel<1>, p, ctas, dev::kProducers, s); break;
        case 2: e = dev::launch_kernel(dev::expand_materialise_kernel<2>, p, ctas, dev::kProducers, s); break;
        case 4: e = dev::launch_kernel(dev::expand_materialise_kernel<4>, p, ctas, dev::kProducers, s); break;
        default: e = dev::launch_kernel(dev::expand_materialise_kernel<8>, p, ctas, dev::kProducers, s); break;
    }
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "expand_materialise launch");
}

int multi_group() { return dev::kMaxGroup; }
int multi_max_range_log2() { return log_sq(dev::kMaxGroup) + dev::kMaxDfsDepth; }

int plan_range_log2(uint64_t rows, uint32_t n, uint32_t group, uint32_t nqg) {
    const int lsq = log_sq(group);
    return pick_range_log2(0, rows, n, group, nqg, 1, std::min((int)n, lsq + dev::kMaxDfsDepth),
                           std::max(1, device_sm_count()), false);
}

int launch_multi(const MultiParams& mp, bool vec, void* stream) {
    if (!reserved_smem_ok()) return PIR_ERR_UNSUPPORTED;
    if (mp.nitems == 0) return PIR_OK;
    const uint32_t ctas = grid_for(mp.nitems);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto kern = vec ? dev::multi_eval_kernel<4> : dev::multi_eval_kernel<1>;
    for (int attempt = 0; attempt < 2; ++attempt) {  // the second sets the attribute again (after a reset)
        cudaError_t e = vec ? dev::smem_attribute_once(dev::multi_eval_kernel<4>, dev::kSmemBytes, attempt > 0)
                            : dev::smem_attribute_once(dev::multi_eval_kernel<1>, dev::kSmemBytes, attempt > 0);
        if (e != cudaSuccess) return cuda_fail((int)e, "multi_eval attribute");
        kern<<<ctas, dev::kFusedThreads, dev::kSmemBytes, s>>>(mp);
        e = cudaGetLastError();
        if (e == cudaSuccess) return PIR_OK;
        if (e != cudaErrorInvalidValue || attempt > 0) return cuda_fail((int)e, "multi_eval launch");
    }
    return PIR_OK;
}

// Partial batch retrieval: `batch` bins of bin_rows rows (the last clipped to
// the table), n = pir_domain_bits(bin_rows).  G bins per item, as many as the
// consumer teams allow (W/4 column chunks per team of kConsumers/G threads);
// item row ranges as for a batch of that many queries over one bin.
int plan_bins(uint64_t bin_rows, uint32_t n, uint32_t width, uint32_t nbins, pir_plan* plan) {
    if (width == 0 || nbins == 0 || n == 0 || width % 4) return PIR_ERR_ARG;
    uint32_t g = 8;
    while (g > 1 && (g > nbins || (uint64_t)g * width > (uint64_t)dev::kYRegionWords ||
                     width / 4 > (uint32_t)dev::kConsumers / g))
        g >>= 1;
    if (width / 4 > (uint32_t)dev::kConsumers / g || (uint64_t)g * width > (uint64_t)dev::kYRegionWords)
        return PIR_ERR_UNSUPPORTED;
    pir_plan pl{};
    pl.vec = 4;
    pl.group = g;
    const uint32_t nqg = (nbins + g - 1) / g;
    const int lsq = log_sq(g);
    const int sms = std::max(1, device_sm_count());
    const int r = pick_range_log2(0, bin_rows, n, g, nqg, 1,
                                  std::min((int)n, lsq + dev::kMaxDfsDepth), sms, true);
    pl.range_log2 = (uint32_t)r;
    const uint64_t items = items_for(0, bin_rows, (uint32_t)r, nqg);
    pl.tail_log2 = (uint32_t)pick_tail_log2(items, sms, n, g, r);
    pl.ctas = (uint32_t)std::min<uint64_t>(items, (uint64_t)sms);
    *plan = pl;
    return PIR_OK;
}

int launch_bins(const EvalRequest& req, uint64_t bin_rows, const pir_plan& plan, void* stream) {
    if (!reserved_smem_ok()) return PIR_ERR_UNSUPPORTED;
    // items: (bin group, range within a bin); every bin spans bin_rows rows of its tree
    EvalRequest one = req;
    one.row_lo = 0;
    one.row_hi = bin_rows;
    dev::FusedParams p = make_params(one, plan);
    p.row_hi = req.row_hi;  // the table's rows: clips the last bin
    p.bin_rows = bin_rows;
    if (p.nitems == 0) return PIR_OK;
    const uint32_t ctas = grid_for(p.nitems);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    switch (plan.group) {
        case 1: e = dev::launch_kernel(dev::bins_eval_kernel<1>, p, ctas, dev::kFusedThreads, s); break;
        case 2: e = dev::launch_kernel(dev::bins_eval_kernel<2>, p, ctas, dev::kFusedThreads, s); break;
        case 4: e = dev::launch_kernel(dev::bins_eval_kernel<4>, p, ctas, dev::kFusedThreads, s); break;
        default: e = dev::launch_kernel(dev::bins_eval_kernel<8>, p, ctas, dev::kFusedThreads, s); break;
    }
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "bins_eval launch");
}

// Chunks of the staged scan that the issuing warp asks L2 for ahead of the one
// it copies (0: none).  A tuning knob: PIR_RING_PREFETCH_CHUNKS in the
// environment overrides the default, read once per process.
static uint32_t ring_prefetch_chunks() {
    static const uint32_t v = [] {
        const char* e = std::getenv("PIR_RING_PREFETCH_CHUNKS");
        return e ? (uint32_t)std::strtoul(e, nullptr, 10) : (uint32_t)PIR_RING_PREFETCH_DEFAULT;
    }();
    return v;
}

int launch_fused(const EvalRequest& req, const pir_plan& plan, void* stream) {
    if (!reserved_smem_ok()) return PIR_ERR_UNSUPPORTED;
    dev::FusedParams p = make_params(req, plan);
    if (p.nitems == 0) return PIR_OK;
    const uint32_t ctas = grid_for(p.nitems);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (plan.strategy == PIR_STRATEGY_FUSED_STAGED) {
        if (plan_check_staged(plan, req.n, req.width, req.stride, plan.vec == 4) != PIR_OK ||
            (reinterpret_cast<uintptr_t>(req.table) & 15u) != 0 || req.stride % 4 != 0)
            return PIR_ERR_UNSUPPORTED;
        p.ring_stages = (uint32_t)ring_stages_for(plan);
        p.ring_prefetch = ring_prefetch_chunks();
        p.faults = device_fault_word();
        if (!p.faults) return cuda_fail((int)cudaGetLastError(), "fault word address");
        switch (plan.group) {
            case 1: e = dev::launch_kernel(dev::fused_eval_staged_kernel<1>, p, ctas, dev::kStagedThreads, s); break;
            case 2: e = dev::launch_kernel(dev::fused_eval_staged_kernel<2>, p, ctas, dev::kStagedThreads, s); break;
            default: e = dev::launch_kernel(dev::fused_eval_staged_kernel<4>, p, ctas, dev::kStagedThreads, s); break;
        }
        return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "fused_eval_staged launch");
    }
    if (plan.vec == 4) {
        switch (plan.group) {
            case 1: e = dev::launch_kernel(dev::fused_eval_kernel<1, 4>, p, ctas, dev::kFusedThreads, s); break;
            case 2: e = dev::launch_kernel(dev::fused_eval_kernel<2, 4>, p, ctas, dev::kFusedThreads, s); break;
            case 4: e = dev::launch_kernel(dev::fused_eval_kernel<4, 4>, p, ctas, dev::kFusedThreads, s); break;
            default: e = dev::launch_kernel(dev::fused_eval_kernel<8, 4>, p, ctas, dev::kFusedThreads, s); break;
        }
    } else {
        switch (plan.group) {
            case 1: e = dev::launch_kernel(dev::fused_eval_kernel<1, 1>, p, ctas, dev::kFusedThreads, s); break;
            case 2: e = dev::launch_kernel(dev::fused_eval_kernel<2, 1>, p, ctas, dev::kFusedThreads, s); break;
            case 4: e = dev::launch_kernel(dev::fused_eval_kernel<4, 1>, p, ctas, dev::kFusedThreads, s); break;
            default: e = dev::launch_kernel(dev::fused_eval_kernel<8, 1>, p, ctas, dev::kFusedThreads, s); break;
        }
    }
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "fused_eval launch");
}

}  // namespace pir
