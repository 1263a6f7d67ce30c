// Share matrix x table mod 2^32 on CUDA cores: the unfused second half of the
// level-by-level baseline (paper Sec. 3.2.2 / 3.2.4: DPF output B x L times the
// table L x W as one matrix-matrix product, Sec. 3.1).
//
//   out[b][w] += sum_{k < rows} S[b][k] * T[k][w]   (mod 2^32)
//
// Split-K tiles: each CTA owns a 64 x 64 output tile and a slice of k; the
// slice's partial sums are added with u32 atomics (associative mod 2^32, so
// bit-exact in any order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace pir {
namespace dev {

constexpr int kCtBM = 64;  // queries per tile
constexpr int kCtBN = 64;  // words per tile
constexpr int kCtBK = 32;  // k per smem stage
constexpr int kCtPadS = 65;  // [k][b] row stride: consecutive k land on distinct banks

__global__ void __launch_bounds__(256) contract_imad_kernel(const uint32_t* __restrict__ S, uint64_t ld, uint32_t B,
                                                            const uint32_t* __restrict__ T, uint64_t stride,
                                                            uint32_t W, uint64_t K, uint64_t kslice,
                                                            uint32_t* __restrict__ out) {
    __shared__ uint32_t sS[kCtBK * kCtPadS];  // sS[k][b]
    __shared__ __align__(16) uint32_t sT[kCtBK * kCtBN];  // sT[k][w]
    const int tid = threadIdx.x;
    const uint32_t b0 = blockIdx.y * kCtBM, w0 = blockIdx.z * kCtBN;
    const uint64_t k0 = (uint64_t)blockIdx.x * kslice;
    const uint64_t k1 = k0 + kslice < K ? k0 + kslice : K;
    const int tb = (tid >> 4) * 4, tw = (tid & 15) * 4;  // this thread's 4 x 4 outputs
    uint32_t acc[4][4] = {};

    // loaders: S tile lane k = tid%32 over rows b = (tid/32)*8 + i (128-byte row segments);
    // T tile lane w = tid%64 over k = (tid/64)*8 + i.  Both smem stores are conflict-free.
    const int ls_k = tid & 31, ls_b = (tid >> 5) * 8;
    const int lt_w = tid & 63, lt_k = (tid >> 6) * 8;
    for (uint64_t kt = k0; kt < k1; kt += kCtBK) {
        {
            const uint64_t k = kt + ls_k;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t b = b0 + ls_b + i;
                sS[ls_k * kCtPadS + ls_b + i] = (b < B && k < k1) ? __ldg(S + (uint64_t)b * ld + k) : 0u;
            }
        }
        {
            const uint32_t w = w0 + lt_w;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint64_t k = kt + lt_k + i;
                sT[(lt_k + i) * kCtBN + lt_w] = (k < k1 && w < W) ? __ldg(T + k * stride + w) : 0u;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kCtBK; ++kk) {
            uint32_t a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sS[kk * kCtPadS + tb + i];
            const uint4 t = *reinterpret_cast<const uint4*>(&sT[kk * kCtBN + tw]);
            const uint32_t bv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t b = b0 + tb + i;
        if (b >= B) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t w = w0 + tw + j;
            if (w < W && acc[i][j]) atomicAdd(&out[(uint64_t)b * W + w], acc[i][j]);
        }
    }
}

// ---- the same product on the tensor pipe, exactly, with 8-bit limbs -------
//
// With S = sum_i s_i 2^{8i} and T = sum_j t_j 2^{8j} (bytes s_i, t_j), the
// product mod 2^32 is sum_{i+j<=3} s_i t_j 2^{8(i+j)}: ten u8 x u8 products
// in four shift classes d = i + j.  Each class accumulates in s32 tensor-core
// accumulators (mma.sync m16n8k32 .u8.u8.s32) and is folded into a u32 total
// every kFoldK values of k, before any class can exceed 2^31 (d = 3 holds
// four products of at most 255^2: 4096 * 4 * 65025 < 2^31), so the result
// does not depend on how the accumulator treats overflow.  The shared-memory
// tiles hold the operands already split into byte planes: plane p, row, then
// one u32 per 4 consecutive k (4 bytes), the layout of an MMA fragment.
constexpr int kMmBM = 64, kMmBN = 64, kMmBK = 64;
constexpr int kMmRS = kMmBK / 4 + 4;  // u32 per plane row: 16 k-quads + 4 pad (conflict-free fragment reads)
constexpr int kFoldK = 4096;

// byte-transpose of four words: plane p gets byte p of w0..w3
__device__ __forceinline__ void byte_planes(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t (&p)[4]) {
    const uint32_t t0 = __byte_perm(w0, w1, 0x5140u), t1 = __byte_perm(w2, w3, 0x5140u);
    const uint32_t t2 = __byte_perm(w0, w1, 0x7362u), t3 = __byte_perm(w2, w3, 0x7362u);
    p[0] = __byte_perm(t0, t1, 0x5410u);
    p[1] = __byte_perm(t0, t1, 0x7632u);
    p[2] = __byte_perm(t2, t3, 0x5410u);
    p[3] = __byte_perm(t2, t3, 0x7632u);
}

__device__ __forceinline__ void mma_u8(uint32_t (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) contract_mma_u8_kernel(const uint32_t* __restrict__ S, uint64_t ld,
                                                              uint32_t B, const uint32_t* __restrict__ T,
                                                              uint64_t stride, uint32_t W, uint64_t K,
                                                              uint64_t kslice, uint32_t* __restrict__ out) {
    __shared__ uint32_t sA[4][kMmBM][kMmRS];  // [limb][query row][k quad]
    __shared__ uint32_t sB[4][kMmBN][kMmRS];  // [limb][table word][k quad]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int mt = warp & 3, nh = warp >> 2;  // warp tile: rows mt*16.., words nh*32..
    const uint32_t b0 = blockIdx.y * kMmBM, w0 = blockIdx.z * kMmBN;
    const uint64_t k0 = (uint64_t)blockIdx.x * kslice;
    const uint64_t k1 = k0 + kslice < K ? k0 + kslice : K;

    uint32_t cls[4][4][4];  // [shift class d][n tile][fragment element]
    uint32_t total[4][4];   // folded u32 result, [n tile][element]
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            total[nt][e] = 0;
#pragma unroll
            for (int d = 0; d < 4; ++d) cls[d][nt][e] = 0;
        }

    uint32_t since_fold = 0;
    for (uint64_t kt = k0; kt < k1; kt += kMmBK) {
        // ---- stage the S tile: thread -> row tid/4, k quads (tid%4) + 4u -------
        {
            const uint32_t b = b0 + (tid >> 2);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = (tid & 3) + 4 * u;
                const uint64_t k = kt + 4 * q;
                uint32_t w[4] = {0, 0, 0, 0};
                if (b < B) {
                    const uint32_t* src = S + (uint64_t)b * ld + k;
                    if (k + 3 < k1 && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
                        const uint4 v = __ldg(reinterpret_cast<const uint4*>(src));
                        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) w[e] = (k + e < k1) ? __ldg(src + e) : 0u;
                    }
                }
                uint32_t pl[4];
                byte_planes(w[0], w[1], w[2], w[3], pl);
#pragma unroll
                for (int p = 0; p < 4; ++p) sA[p][tid >> 2][q] = pl[p];
            }
        }
        // ---- stage the T tile: thread -> word (tid/32)*8 + tid%8, k quads (tid/8)%4 + 4u
        {
            const int wl = ((tid >> 5) << 3) + (tid & 7);
            const uint32_t w = w0 + wl;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = ((tid >> 3) & 3) + 4 * u;
                const uint64_t k = kt + 4 * q;
                uint32_t v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = (w < W && k + e < k1) ? __ldg(T + (k + e) * stride + w) : 0u;
                uint32_t pl[4];
                byte_planes(v[0], v[1], v[2], v[3], pl);
#pragma unroll
                for (int p = 0; p < 4; ++p) sB[p][wl][q] = pl[p];
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kMmBK / 32; ++ks) {
            uint32_t a[4][4];  // [limb][fragment register]
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                a[p][0] = sA[p][mt * 16 + gid][ks * 8 + tig];
                a[p][1] = sA[p][mt * 16 + gid + 8][ks * 8 + tig];
                a[p][2] = sA[p][mt * 16 + gid][ks * 8 + 4 + tig];
                a[p][3] = sA[p][mt * 16 + gid + 8][ks * 8 + 4 + tig];
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int col = nh * 32 + nt * 8 + gid;
                uint32_t bl[4][2];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    bl[p][0] = sB[p][col][ks * 8 + tig];
                    bl[p][1] = sB[p][col][ks * 8 + 4 + tig];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; i + j < 4; ++j) mma_u8(cls[i + j][nt], a[i], bl[j][0], bl[j][1]);
            }
        }
        __syncthreads();
        since_fold += kMmBK;
        if (since_fold >= kFoldK || kt + kMmBK >= k1) {
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    total[nt][e] += cls[0][nt][e] + (cls[1][nt][e] << 8) + (cls[2][nt][e] << 16) + (cls[3][nt][e] << 24);
#pragma unroll
                    for (int d = 0; d < 4; ++d) cls[d][nt][e] = 0;
                }
            since_fold = 0;
        }
    }
    // D fragment: elements (gid, 2tig), (gid, 2tig+1), (gid+8, 2tig), (gid+8, 2tig+1)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t b = b0 + mt * 16 + gid + ((e >> 1) << 3);
            const uint32_t w = w0 + nh * 32 + nt * 8 + 2 * tig + (e & 1);
            if (b < B && w < W && total[nt][e]) atomicAdd(&out[(uint64_t)b * W + w], total[nt][e]);
        }
}

}  // namespace dev

// Largest batch for which PIR_CONTRACT_AUTO picks the streaming scan.  The
// scan reads the table once per 8 queries; the tcgen05 engine converts a
// whole 128-query tile whatever the batch, and with rows of 32 words or fewer
// each share word feeds half as many products.  On GB300 (ms, scan / tcgen05):
// 2^20 x 64 words 0.116 / 0.167 at 16 queries, 0.170 / 0.168 at 24;
// 2^18 x 128 words 0.066 / 0.095 at 16, 0.098 / 0.093 at 24; 2^22 x 32 words
// 0.453 / 0.572 at 32, 0.568 / 0.573 at 40.  IMAD is never the fastest.
constexpr uint32_t kAutoScanMaxBatchWide = 16;    // rows wider than 32 words
constexpr uint32_t kAutoScanMaxBatchNarrow = 32;  // rows of at most 32 words

int launch_contract(const uint32_t* shares, uint64_t ld, uint32_t batch, const uint32_t* table, uint64_t stride,
                    uint32_t width, uint64_t rows, uint32_t* out, int engine, void* stream) {
    if (engine == PIR_CONTRACT_AUTO)  // the engine measured fastest for the shape on GB300
        engine = batch <= (width <= 32 ? kAutoScanMaxBatchNarrow : kAutoScanMaxBatchWide) &&
                         scan_supported(shares, ld, table, stride, width)
                     ? PIR_CONTRACT_SCAN
                     : PIR_CONTRACT_TC_F16;
    if (engine == PIR_CONTRACT_SCAN) return launch_scan(shares, ld, batch, table, stride, width, rows, out, stream);
    if (engine == PIR_CONTRACT_TC_F16)
        return launch_contract_tc(shares, ld, batch, table, stride, width, rows, out, stream);
    if (engine == PIR_CONTRACT_MMA_U8) {
        const uint32_t by = (batch + dev::kMmBM - 1) / dev::kMmBM, bz = (width + dev::kMmBN - 1) / dev::kMmBN;
        const int sms = std::max(1, device_sm_count());
        uint64_t slices = std::max<uint64_t>(1, (uint64_t)sms * 8 / ((uint64_t)by * bz));
        uint64_t kslice = (rows + slices - 1) / slices;
        kslice = std::max<uint64_t>(dev::kMmBK, (kslice + dev::kMmBK - 1) / dev::kMmBK * dev::kMmBK);
        slices = (rows + kslice - 1) / kslice;
        if (slices > 0x7fffffffull || by > 65535 || bz > 65535) return PIR_ERR_UNSUPPORTED;
        dim3 grid((uint32_t)slices, by, bz);
        dev::contract_mma_u8_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
            shares, ld, batch, table, stride, width, rows, kslice, out);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "contract (u8 limbs) launch");
    }
    if (engine != PIR_CONTRACT_IMAD) return PIR_ERR_UNSUPPORTED;
    const uint32_t by = (batch + dev::kCtBM - 1) / dev::kCtBM, bz = (width + dev::kCtBN - 1) / dev::kCtBN;
    const int sms = std::max(1, device_sm_count());
    // enough k-slices for about eight resident tile waves, each slice a multiple of the stage depth
    uint64_t slices = std::max<uint64_t>(1, (uint64_t)sms * 8 / ((uint64_t)by * bz));
    uint64_t kslice = (rows + slices - 1) / slices;
    kslice = std::max<uint64_t>(dev::kCtBK, (kslice + dev::kCtBK - 1) / dev::kCtBK * dev::kCtBK);
    slices = (rows + kslice - 1) / kslice;
    if (slices > 0x7fffffffull || by > 65535 || bz > 65535) return PIR_ERR_UNSUPPORTED;
    dim3 grid((uint32_t)slices, by, bz);
    dev::contract_imad_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        shares, ld, batch, table, stride, width, rows, kslice, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "contract launch");
}

}  // namespace pir
