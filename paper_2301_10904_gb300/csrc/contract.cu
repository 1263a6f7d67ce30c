// Share matrix x table mod 2^32 on CUDA cores: the unfused second half of the
// level-by-level baseline (paper Sec. 3.2.2 / 3.2.4: DPF output B x L times the
// table L x W, "batched together as a single matrix-matrix multiplication",
// Sec. 3.1).
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

}  // namespace dev

int launch_contract(const uint32_t* shares, uint64_t ld, uint32_t batch, const uint32_t* table, uint64_t stride,
                    uint32_t width, uint64_t rows, uint32_t* out, int engine, void* stream) {
    if (engine != 0) return PIR_ERR_UNSUPPORTED;
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
