// Fused DPF full-domain evaluation x table product mod 2^32 for sm_103a.
//
// What it computes (paper Sec. 3.1, Eqs. p1-p3; fusion of Sec. 3.2.4):
//   out[q][w] += sum_{j in rows} y_q(j) * T[j][w]   (mod 2^32)
// where y_q(j) is leaf j of key q's GGM tree:
//   P(0,0) = root;  P(d,j) = AES_{P(d-1,j>>1)}((j&1) || 0^120) ^ C_t[j&1][d],
//   t = lsb(P(d-1,j>>1));  y(j) = (-1)^sigma (word1(P(n,j)) + lsb(P(n,j)) * cw_out).
//
// Structure of one CTA (256 threads), which owns G queries x 2^r rows:
//  1. lookup table: S-box derived in-kernel from GF(2^8), expanded to the
//     column table Te0 with 32 interleaved copies so that lane l always reads
//     bank l (conflict-free, 1 LDS per lookup, index formed with one PRMT).
//  2. path: thread g walks query g from the root to the CTA's range node at
//     depth n - r (one PRF per level).
//  3. split: level by level in shared memory until each query has one
//     subtree root per thread (SQ = 256/G threads per query).
//  4. per-thread depth-first expansion of its subtree (the paper's
//     memory-bounded traversal, Sec. 3.2.3, with the pending right siblings
//     in a shared-memory stack: memory O(threads * depth), not O(L)).  Each
//     PRF evaluation yields both children (one key schedule, two blocks that
//     share their first two rounds' lookups).
//  5. every kPairs leaf pairs the CTA stops and multiplies the fresh leaf
//     shares of all G queries into register accumulators against the table
//     rows they index, reading each row once for all G queries (Sec. 3.2.4).
//  6. accumulators are summed in shared memory and added to out with one
//     u32 atomicAdd per (query, word); addition mod 2^32 is associative, so
//     the result is bit-exact in any order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace pir {
namespace dev {

constexpr int kThreads = 256;
constexpr int kRowBytes = 256;                  // one row per byte value x
constexpr int kLookupBytes = 256 * kRowBytes;   // 64 KiB: [0,128) Te0 copies, [128,256) stack
constexpr int kStackLevels = 8;                 // 256 rows x 8 slots / 256 threads
constexpr int kMaxDfsDepth = kStackLevels + 1;  // levels a thread expands on its own
constexpr int kPairs = 2;                       // leaf pairs per subtree between MAC phases
constexpr int kYBufWords = 2048;                // two buffers of G x 2kPairs x SQ words
constexpr int kHdrWords = 3 * 8;
constexpr int kSmemBytes = kLookupBytes + 4 * kYBufWords + 4 * kHdrWords;

// The kernel's only shared memory; naming the array (not a pointer to it) in
// every access lets the compiler address it as shared with an immediate base.
extern __shared__ __align__(128) char sm[];

struct FusedParams {
    const uint32_t* table;
    uint64_t row_lo, row_hi;
    uint64_t stride;
    uint64_t first_range;
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
};

// ---------------------------------------------------------------- GF(2^8)
__device__ __forceinline__ uint32_t xtime(uint32_t a) { return ((a << 1) ^ (0x1bu & (0u - (a >> 7)))) & 0xffu; }

__device__ uint32_t gf_mul(uint32_t a, uint32_t b) {
    uint32_t p = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        p ^= a & (0u - (b & 1u));
        a = xtime(a);
        b >>= 1;
    }
    return p;
}

// S(x) = affine(x^254); x^254 = x^2 * x^4 * ... * x^128 is the inverse in GF(2^8)
__device__ uint32_t sbox_entry(uint32_t x) {
    uint32_t sq = gf_mul(x, x), inv = sq;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        sq = gf_mul(sq, sq);
        inv = gf_mul(inv, sq);
    }
    uint32_t s = inv;
#pragma unroll
    for (int k = 1; k <= 4; ++k) s ^= ((inv << k) | (inv >> (8 - k))) & 0xffu;
    return s ^ 0x63u;
}

// ---------------------------------------------------------------- lookups
// Row x of the lookup area holds Te0[x] at byte 4*l for every lane l, so the
// address of lane l's copy of Te0[byte r of s] is (byte << 8) | 4l: one PRMT.
#define LK(s, r) (*reinterpret_cast<const uint32_t*>(sm + __byte_perm((s), lane4, 0x5504u | ((r) << 4))))
#define R8(x) __funnelshift_l((x), (x), 8)
#define R16(x) __funnelshift_l((x), (x), 16)
#define R24(x) __funnelshift_l((x), (x), 24)
// S-box bytes sit in byte 1 of Te0: gather four of them into one word
#define SB4(a, b, c, d) __byte_perm(__byte_perm((a), (b), 0x0051u), __byte_perm((c), (d), 0x5100u), 0x7610u)

__device__ void build_lookup(int tid) {
    uint32_t* words = reinterpret_cast<uint32_t*>(sm);
    // staging of the 256 Te0 values in the spare halves of rows 0..7
    {
        const uint32_t s = sbox_entry((uint32_t)tid);
        const uint32_t s2 = xtime(s);
        const uint32_t te = s2 | (s << 8) | (s << 16) | ((s2 ^ s) << 24);
        words[(tid >> 5) * 64 + 32 + (tid & 31)] = te;
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
        const int w = i * kThreads + tid;
        const int x = w >> 5;
        words[x * 64 + (w & 31)] = words[(x >> 5) * 64 + 32 + (x & 31)];
    }
    __syncthreads();
}

// Both children of node v, before the codewords: c_b = AES_v(b || 0^120).
__device__ __forceinline__ void prf2(const uint32_t lane4, const uint4 v, uint4& c0, uint4& c1) {
    uint32_t k0 = v.x, k1 = v.y, k2 = v.z, k3 = v.w;
    const uint32_t s0 = k0, s1 = k1, s2 = k2, s3 = k3;  // round-0 state (block b=0)
    uint32_t t;
#define KEYROUND(rc)                                                   \
    t = SB4(LK(k3, 1), LK(k3, 2), LK(k3, 3), LK(k3, 0)) ^ (rc);        \
    k0 ^= t;                                                           \
    k1 ^= k0;                                                          \
    k2 ^= k1;                                                          \
    k3 ^= k2;
    KEYROUND(0x01u)
    // round 1: only byte 0 of column 0 differs between the two blocks
    const uint32_t x1 = R8(LK(s1, 1)) ^ R16(LK(s2, 2)) ^ R24(LK(s3, 3)) ^ k0;
    const uint32_t a0 = LK(s0, 0) ^ x1;
    const uint32_t b0 = LK(s0 ^ 1u, 0) ^ x1;
    const uint32_t u1 = LK(s1, 0) ^ R8(LK(s2, 1)) ^ R16(LK(s3, 2)) ^ R24(LK(s0, 3)) ^ k1;
    const uint32_t u2 = LK(s2, 0) ^ R8(LK(s3, 1)) ^ R16(LK(s0, 2)) ^ R24(LK(s1, 3)) ^ k2;
    const uint32_t u3 = LK(s3, 0) ^ R8(LK(s0, 1)) ^ R16(LK(s1, 2)) ^ R24(LK(s2, 3)) ^ k3;
    KEYROUND(0x02u)
    // round 2: columns 1..3 are shared, column 0 feeds one lookup per output column
    const uint32_t z0 = R8(LK(u1, 1)) ^ R16(LK(u2, 2)) ^ R24(LK(u3, 3)) ^ k0;
    const uint32_t z1 = LK(u1, 0) ^ R8(LK(u2, 1)) ^ R16(LK(u3, 2)) ^ k1;
    const uint32_t z2 = LK(u2, 0) ^ R8(LK(u3, 1)) ^ R24(LK(u1, 3)) ^ k2;
    const uint32_t z3 = LK(u3, 0) ^ R16(LK(u1, 2)) ^ R24(LK(u2, 3)) ^ k3;
    uint32_t A0 = LK(a0, 0) ^ z0, A1 = R24(LK(a0, 3)) ^ z1, A2 = R16(LK(a0, 2)) ^ z2, A3 = R8(LK(a0, 1)) ^ z3;
    uint32_t B0 = LK(b0, 0) ^ z0, B1 = R24(LK(b0, 3)) ^ z1, B2 = R16(LK(b0, 2)) ^ z2, B3 = R8(LK(b0, 1)) ^ z3;
    const uint32_t rcon[7] = {0x04u, 0x08u, 0x10u, 0x20u, 0x40u, 0x80u, 0x1bu};
#pragma unroll
    for (int r = 0; r < 7; ++r) {  // rounds 3..9
        KEYROUND(rcon[r])
        const uint32_t a0n = LK(A0, 0) ^ R8(LK(A1, 1)) ^ R16(LK(A2, 2)) ^ R24(LK(A3, 3)) ^ k0;
        const uint32_t a1n = LK(A1, 0) ^ R8(LK(A2, 1)) ^ R16(LK(A3, 2)) ^ R24(LK(A0, 3)) ^ k1;
        const uint32_t a2n = LK(A2, 0) ^ R8(LK(A3, 1)) ^ R16(LK(A0, 2)) ^ R24(LK(A1, 3)) ^ k2;
        const uint32_t a3n = LK(A3, 0) ^ R8(LK(A0, 1)) ^ R16(LK(A1, 2)) ^ R24(LK(A2, 3)) ^ k3;
        const uint32_t b0n = LK(B0, 0) ^ R8(LK(B1, 1)) ^ R16(LK(B2, 2)) ^ R24(LK(B3, 3)) ^ k0;
        const uint32_t b1n = LK(B1, 0) ^ R8(LK(B2, 1)) ^ R16(LK(B3, 2)) ^ R24(LK(B0, 3)) ^ k1;
        const uint32_t b2n = LK(B2, 0) ^ R8(LK(B3, 1)) ^ R16(LK(B0, 2)) ^ R24(LK(B1, 3)) ^ k2;
        const uint32_t b3n = LK(B3, 0) ^ R8(LK(B0, 1)) ^ R16(LK(B1, 2)) ^ R24(LK(B2, 3)) ^ k3;
        A0 = a0n; A1 = a1n; A2 = a2n; A3 = a3n;
        B0 = b0n; B1 = b1n; B2 = b2n; B3 = b3n;
    }
    KEYROUND(0x36u)
#undef KEYROUND
    // round 10: SubBytes + ShiftRows + AddRoundKey
    c0.x = SB4(LK(A0, 0), LK(A1, 1), LK(A2, 2), LK(A3, 3)) ^ k0;
    c0.y = SB4(LK(A1, 0), LK(A2, 1), LK(A3, 2), LK(A0, 3)) ^ k1;
    c0.z = SB4(LK(A2, 0), LK(A3, 1), LK(A0, 2), LK(A1, 3)) ^ k2;
    c0.w = SB4(LK(A3, 0), LK(A0, 1), LK(A1, 2), LK(A2, 3)) ^ k3;
    c1.x = SB4(LK(B0, 0), LK(B1, 1), LK(B2, 2), LK(B3, 3)) ^ k0;
    c1.y = SB4(LK(B1, 0), LK(B2, 1), LK(B3, 2), LK(B0, 3)) ^ k1;
    c1.z = SB4(LK(B2, 0), LK(B3, 1), LK(B0, 2), LK(B1, 3)) ^ k2;
    c1.w = SB4(LK(B3, 0), LK(B0, 1), LK(B1, 2), LK(B2, 3)) ^ k3;
}

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }

// Children of v at depth d (1-based) of key `key`: AES plus C_{lsb(v)}[b][d].
__device__ __forceinline__ void expand(uint32_t lane4, const uint8_t* key, uint32_t d, uint4 v,
                                       uint4& c0, uint4& c1) {
    prf2(lane4, v, c0, c1);
    const uint4* cw = reinterpret_cast<const uint4*>(key + PIR_KEY_HEADER_BYTES + 64u * (d - 1) + 32u * (v.x & 1u));
    c0 = xor4(c0, __ldg(cw));
    c1 = xor4(c1, __ldg(cw + 1));
}

// Pending right sibling at relative level `lvl` (1..8) of thread `tid`:
// slot (lvl-1)*256 + tid in the spare halves of the lookup rows.
__device__ __forceinline__ uint4* stack_slot(int lvl, int tid) {
    const int s = (lvl - 1) * kThreads + tid;
    return reinterpret_cast<uint4*>(sm + (s >> 3) * kRowBytes + 128 + (s & 7) * 16);
}

template <int G, int VEC>
__device__ __forceinline__ void load_row(const uint32_t* p, uint32_t (&v)[VEC]) {
    if constexpr (VEC == 4) {
        const uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        v[0] = __ldg(p);
    }
}

// Multiply the shares of the last `kc` leaf pairs of every subtree into acc.
template <int G, int VEC>
__device__ __forceinline__ void mac_phase(const FusedParams& p, const uint32_t* yb, uint64_t r0, int m, int sd,
                                          uint32_t kbase, uint32_t kc, uint32_t (&acc)[G][VEC], int tid) {
    constexpr int SQ = kThreads / G;
    const uint32_t nc = p.width / VEC;
    const uint32_t nrg = kThreads / nc;
    const uint32_t c = (uint32_t)tid % nc, rg = (uint32_t)tid / nc;
    if (rg >= nrg) return;
    const uint32_t nrows = (2u * kc) << sd;
    const uint32_t submask = (1u << sd) - 1u;
    for (uint32_t rr = rg; rr < nrows; rr += nrg) {
        const uint32_t j = rr >> sd, l = rr & submask;
        const uint64_t row = r0 + ((uint64_t)l << m) + 2ull * kbase + j;
        if (row < p.row_lo || row >= p.row_hi) continue;
        uint32_t tv[VEC];
        load_row<G, VEC>(p.table + (row - p.row_lo) * p.stride + (uint64_t)c * VEC, tv);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t y = yb[(g * 2 * kPairs + j) * SQ + l];
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[g][i] += y * tv[i];
        }
    }
}

// Writes this thread's last 2*kc leaf shares (rows row_base .. row_base+2kc-1)
// to the materialised share matrix.
template <int G>
__device__ __forceinline__ void store_phase(const FusedParams& p, const uint32_t* yb, uint32_t q, int g, int l,
                                            uint64_t row_base, uint32_t kc) {
    constexpr int SQ = kThreads / G;
    uint32_t* dst = p.shares + (uint64_t)q * p.ld;
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

// The whole CTA program.  MAT = false: fused share x table product (a1-a6).
// MAT = true: expansion only, leaf shares written to p.shares (a7 baseline).
template <int G, int VEC, bool MAT>
__device__ __forceinline__ void eval_body(const FusedParams& p) {
    constexpr int SQ = kThreads / G;
    constexpr int LOG_SQ = (SQ == 256) ? 8 : (SQ == 128) ? 7 : (SQ == 64) ? 6 : 5;
    static_assert(G * 2 * kPairs * SQ * 2 <= kYBufWords, "share buffers exceed their region");

    const int tid = threadIdx.x;
    const uint32_t lane4 = (uint32_t)(tid & 31) << 2;
    uint32_t* ybuf = reinterpret_cast<uint32_t*>(sm + kLookupBytes);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(sm + kLookupBytes + 4 * kYBufWords);  // ok[G], party[G], cwo[G]

    const uint32_t qg = blockIdx.x % p.nqg;
    const uint64_t r0 = (p.first_range + blockIdx.x / p.nqg) << p.range_log2;
    const int n = (int)p.n, r = (int)p.range_log2;
    const int sd = min(LOG_SQ, r - 1);
    const int m = r - sd;

    build_lookup(tid);

    // ---- key headers and the path to this CTA's range node ---------------
    uint4* bufA = reinterpret_cast<uint4*>(ybuf);
    uint4* bufB = bufA + kThreads;
    if (tid < G) {
        const uint32_t q = qg * G + tid;
        uint32_t ok = 0, party = 0, cwo = 0;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (q < p.batch) {
            const uint8_t* key = p.keys + (uint64_t)q * p.key_bytes;
            const uint4 h = __ldg(reinterpret_cast<const uint4*>(key));
            ok = h.x == kKeyMagic && (h.y & 0xffu) == kKeyVersion && ((h.y >> 8) & 0xffu) == p.n &&
                 ((h.y >> 16) & 0xffu) <= 1u && (h.y >> 24) == 0u;
            if (ok) {
                party = (h.y >> 16) & 1u;
                cwo = h.z;
                v = __ldg(reinterpret_cast<const uint4*>(key + 16));
                for (int d = 1; d <= n - r; ++d) {
                    const uint32_t b = (uint32_t)(r0 >> (n - d)) & 1u;
                    uint4 c0, c1;
                    expand(lane4, key, (uint32_t)d, v, c0, c1);
                    v = b ? c1 : c0;
                }
            } else if (p.status) {
                atomicOr(p.status, PIR_STATUS_BAD_KEY);
            }
        }
        hdr[tid] = ok;
        hdr[G + tid] = party;
        hdr[2 * G + tid] = cwo;
        bufA[tid] = v;
    }
    __syncthreads();

    // ---- split to one subtree root per thread ------------------------------
    for (int i = 0; i < sd; ++i) {
        const uint4* src = (i & 1) ? bufB : bufA;
        uint4* dst = (i & 1) ? bufA : bufB;
        if (tid < (G << i)) {
            const int g = tid >> i, idx = tid & ((1 << i) - 1);
            const uint4 v = src[tid];
            uint4 c0 = v, c1 = v;
            if (hdr[g]) {
                const uint8_t* key = p.keys + (uint64_t)(qg * G + g) * p.key_bytes;
                expand(lane4, key, (uint32_t)(n - r + i + 1), v, c0, c1);
            }
            dst[(g << (i + 1)) + 2 * idx] = c0;
            dst[(g << (i + 1)) + 2 * idx + 1] = c1;
        }
        __syncthreads();
    }
    const int g = tid / SQ, l = tid % SQ;
    const int nsub = 1 << sd;
    const bool act = l < nsub && hdr[g] != 0;
    const uint32_t party = hdr[G + g], cwo = hdr[2 * G + g];
    uint4 node = make_uint4(0, 0, 0, 0);
    if (l < nsub) node = ((sd & 1) ? bufB : bufA)[(g << sd) + l];
    const uint8_t* key = p.keys + (uint64_t)(qg * G + (act ? g : 0)) * p.key_bytes;
    __syncthreads();  // share buffers alias the split buffers

    // ---- depth-first expansion with periodic table products ----------------
    uint32_t acc[G][VEC];
#pragma unroll
    for (int a = 0; a < G; ++a)
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[a][i] = 0;

    const int d0 = n - r + sd;  // depth of this thread's subtree root
    const uint32_t npairs = 1u << (m - 1);
    const uint32_t kc = npairs < (uint32_t)kPairs ? npairs : (uint32_t)kPairs;
    int lvl = 0;
    uint32_t k = 0, phase = 0;
    for (;;) {
        uint4 c0 = node, c1 = node;
        if (act) expand(lane4, key, (uint32_t)(d0 + lvl + 1), node, c0, c1);
        if (lvl + 1 == m) {
            uint32_t y0 = 0, y1 = 0;
            if (act) {
                y0 = c0.y + (c0.x & 1u) * cwo;
                y1 = c1.y + (c1.x & 1u) * cwo;
                if (party) {
                    y0 = 0u - y0;
                    y1 = 0u - y1;
                }
            }
            uint32_t* yb = ybuf + (phase & 1u) * (kYBufWords / 2);
            const uint32_t j = 2u * (k % kc);
            yb[(g * 2 * kPairs + j) * SQ + l] = y0;
            yb[(g * 2 * kPairs + j + 1) * SQ + l] = y1;
            ++k;
            if (k % kc == 0) {
                if constexpr (MAT) {
                    // each thread stores only what it wrote itself: no barrier needed
                    const uint32_t q = qg * G + g;
                    if (q < p.batch && l < nsub)
                        store_phase<G>(p, yb, q, g, l, r0 + ((uint64_t)l << m) + 2ull * (k - kc), kc);
                } else {
                    __syncthreads();
                    mac_phase<G, VEC>(p, yb, r0, m, sd, k - kc, kc, acc, tid);
                }
                ++phase;
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

    if constexpr (MAT) return;
    // ---- reduce the per-thread partial sums, then one atomic per word ------
    __syncthreads();
    const uint32_t W = p.width;
    uint32_t* red = ybuf;
    for (uint32_t i = tid; i < G * W; i += kThreads) red[i] = 0;
    __syncthreads();
    {
        const uint32_t nc = W / VEC, nrg = kThreads / nc;
        const uint32_t c = (uint32_t)tid % nc, rg = (uint32_t)tid / nc;
        if (rg < nrg) {
#pragma unroll
            for (int a = 0; a < G; ++a)
#pragma unroll
                for (int i = 0; i < VEC; ++i)
                    if (acc[a][i]) atomicAdd(&red[a * W + c * VEC + i], acc[a][i]);
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i < G * W; i += kThreads) {
        const uint32_t a = i / W, q = qg * G + a;
        const uint32_t v = red[i];
        if (q < p.batch && v) atomicAdd(&p.out[(uint64_t)q * W + (i - a * W)], v);
    }
}

template <int G, int VEC>
__global__ void __launch_bounds__(kThreads, 3) fused_eval_kernel(const FusedParams p) {
    eval_body<G, VEC, false>(p);
}

template <int G>
__global__ void __launch_bounds__(kThreads, 3) expand_materialise_kernel(const FusedParams p) {
    eval_body<G, 1, true>(p);
}

template <typename Kern>
cudaError_t launch_kernel(Kern kern, const FusedParams& p, uint32_t ctas, cudaStream_t s) {
    // the attribute is per function and device; setting it each launch costs ~1 us and is always correct
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    kern<<<ctas, kThreads, kSmemBytes, s>>>(p);
    return cudaGetLastError();
}

template <int G, int VEC>
cudaError_t launch_one(const FusedParams& p, uint32_t ctas, cudaStream_t s) {
    return launch_kernel(fused_eval_kernel<G, VEC>, p, ctas, s);
}

}  // namespace dev

// ------------------------------------------------------------------ host side

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

static int log_sq(uint32_t group) { return group == 1 ? 8 : group == 2 ? 7 : group == 4 ? 6 : 5; }

static uint64_t ctas_for(uint64_t row_lo, uint64_t rows, uint32_t r, uint32_t nqg) {
    if (rows == 0) return 0;
    const uint64_t first = row_lo >> r, last = (row_lo + rows - 1) >> r;
    return (last - first + 1) * nqg;
}

int plan_check(const pir_plan& plan, uint32_t n, uint32_t width, bool vec_ok) {
    if (plan.group != 1 && plan.group != 2 && plan.group != 4 && plan.group != 8) return PIR_ERR_UNSUPPORTED;
    if (plan.vec != 1 && plan.vec != 4) return PIR_ERR_UNSUPPORTED;
    if (plan.vec == 4 && (!vec_ok || width % 4 != 0)) return PIR_ERR_UNSUPPORTED;
    if (width == 0 || width / plan.vec > (uint32_t)dev::kThreads) return PIR_ERR_UNSUPPORTED;
    if ((uint64_t)plan.group * width > (uint64_t)dev::kYBufWords) return PIR_ERR_UNSUPPORTED;
    const int r = (int)plan.range_log2;
    if (r < 1 || r > (int)n) return PIR_ERR_UNSUPPORTED;
    const int sd = std::min(log_sq(plan.group), r - 1);
    if (r - sd > dev::kMaxDfsDepth) return PIR_ERR_UNSUPPORTED;
    return PIR_OK;
}

int plan_fused(uint64_t rows, uint64_t row_lo, uint32_t n, uint32_t width, uint32_t batch, bool vec_ok,
               pir_plan* plan) {
    if (width == 0 || batch == 0 || n == 0) return PIR_ERR_ARG;
    pir_plan pl{};
    pl.vec = (vec_ok && width % 4 == 0) ? 4 : 1;
    if (width / pl.vec > (uint32_t)dev::kThreads) return PIR_ERR_UNSUPPORTED;
    uint32_t g = 8;
    while (g > 1 && (g > batch || (uint64_t)g * width > (uint64_t)dev::kYBufWords)) g >>= 1;
    if ((uint64_t)g * width > (uint64_t)dev::kYBufWords) return PIR_ERR_UNSUPPORTED;
    pl.group = g;
    const uint32_t nqg = (batch + g - 1) / g;
    const int lsq = log_sq(g);
    int r = std::min((int)n, lsq + dev::kMaxDfsDepth);
    const int sms = std::max(1, device_sm_count());
    const uint64_t target = (uint64_t)sms * 3 * 4;  // about four waves of resident CTAs
    while (r > std::min((int)n, lsq + 1) && ctas_for(row_lo, rows, (uint32_t)r, nqg) < target) --r;
    pl.range_log2 = (uint32_t)r;
    pl.ctas = (uint32_t)ctas_for(row_lo, rows, (uint32_t)r, nqg);
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
    return p;
}

int launch_materialise(const EvalRequest& req, const pir_plan& plan, uint32_t* shares, uint64_t ld, void* stream) {
    dev::FusedParams p = make_params(req, plan);
    p.shares = shares;
    p.ld = ld;
    p.shares_vec = ((reinterpret_cast<uintptr_t>(shares) & 15u) == 0 && ld % 4 == 0) ? 1u : 0u;
    const uint64_t ctas = ctas_for(req.row_lo, req.row_hi - req.row_lo, plan.range_log2, p.nqg);
    if (ctas == 0) return PIR_OK;
    if (ctas > 0x7fffffffull) return PIR_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (plan.group) {
        case 1: e = dev::launch_kernel(dev::expand_materialise_kernel<1>, p, (uint32_t)ctas, s); break;
        case 2: e = dev::launch_kernel(dev::expand_materialise_kernel<2>, p, (uint32_t)ctas, s); break;
        case 4: e = dev::launch_kernel(dev::expand_materialise_kernel<4>, p, (uint32_t)ctas, s); break;
        default: e = dev::launch_kernel(dev::expand_materialise_kernel<8>, p, (uint32_t)ctas, s); break;
    }
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "expand_materialise launch");
}

int launch_fused(const EvalRequest& req, const pir_plan& plan, void* stream) {
    const uint32_t g = plan.group;
    dev::FusedParams p = make_params(req, plan);
    const uint64_t ctas = ctas_for(req.row_lo, req.row_hi - req.row_lo, plan.range_log2, p.nqg);
    if (ctas == 0) return PIR_OK;
    if (ctas > 0x7fffffffull) return PIR_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    const uint32_t c = (uint32_t)ctas;
    if (plan.vec == 4) {
        switch (g) {
            case 1: e = dev::launch_one<1, 4>(p, c, s); break;
            case 2: e = dev::launch_one<2, 4>(p, c, s); break;
            case 4: e = dev::launch_one<4, 4>(p, c, s); break;
            default: e = dev::launch_one<8, 4>(p, c, s); break;
        }
    } else {
        switch (g) {
            case 1: e = dev::launch_one<1, 1>(p, c, s); break;
            case 2: e = dev::launch_one<2, 1>(p, c, s); break;
            case 4: e = dev::launch_one<4, 1>(p, c, s); break;
            default: e = dev::launch_one<8, 1>(p, c, s); break;
        }
    }
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "fused_eval launch");
}

}  // namespace pir
