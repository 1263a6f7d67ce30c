// Share matrix x table mod 2^32 for a few queries: a streaming scan of the
// table, bound by HBM bandwidth.  With a small batch the product of Sec. 3.1
// (a batch of queries to one table is one matrix-matrix product) does a few
// multiply-adds per table byte, so every table row should leave HBM once, at
// full bandwidth (Sec. 3.2.4: the table read is the memory-bound part).
//
//   out[b][w] += sum_{k < K} S[b][k] * T[k][w]   (mod 2^32),  b < B <= 8
//
// The copy engine streams chunks of R consecutive table rows, and the same R
// share words of every query, into a ring of kScanStages shared-memory stages
// (cp.async.bulk, completion counted in bytes on a "full" mbarrier per stage).
// One warp issues the copies; 8 consumer warps multiply each chunk into
// register accumulators while the next stages are in flight, and release a
// stage by arriving on its "empty" mbarrier, which the issuing warp waits on
// before refilling it: no CTA-wide barrier per chunk.  Every wait is bounded.  Consumer (c, rg) owns words 4c..4c+3 of rows
// 4rg..4rg+3 of a chunk, so that it reads four shares of a query with one
// 128-bit load.  Partial sums meet in shared memory, then one u32
// atomicAdd per (query, word) per CTA; addition mod 2^32 is associative, so
// the result is bit-exact in any order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "async_copy.cuh"
#include "internal.h"

namespace pir {
namespace dev {

constexpr int kScanConsumers = 256;                 // threads that multiply (8 warps)
constexpr int kScanConsumerWarps = kScanConsumers / 32;
constexpr int kScanThreads = kScanConsumers + 32;    // + one warp that issues the copies
constexpr int kScanStages = 4;
constexpr uint32_t kScanTableStageBytes = 16384;  // table bytes per stage (target)
constexpr uint32_t kScanMaxRows = 512;            // rows per chunk cap (bounds the share slots)
constexpr uint32_t kScanMaxWidth = 1024;          // words per row (R >= 4 keeps stages <= 16 KiB)
constexpr uint32_t kScanHeader = 128;             // full mbarriers [0,32), empty [32,64), abort flag at 64
constexpr int kScanConsumerBar = 1;               // named barrier of the consumer warps
constexpr uint32_t kScanSpinLimit = 1u << 22;     // bounded waits (each try_wait may also suspend)

// Set (bitwise) when a wait in one of the library's kernels gave up; read and
// cleared by pir_device_status.
__device__ uint32_t g_device_faults;

struct ScanParams {
    const uint32_t* S;
    uint64_t ld;
    const uint32_t* T;
    uint64_t stride;
    uint64_t K;
    uint64_t nchunks;
    uint32_t* out;
    uint32_t B, W;
    uint32_t R;            // rows per chunk, multiple of 4
    uint32_t stage_bytes;  // R * stride * 4 (table slot) + 8 * R * 4 (share slots)
    // diagonal form (partial batch retrieval): S is one share per table row, row k
    // belonging to query k / bin_rows; each CTA takes chunks_per_cta consecutive chunks
    uint64_t bin_rows;
    uint64_t chunks_per_cta;
};

extern __shared__ __align__(128) char scan_sm[];

// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    return mbar_wait_bounded(bar, parity, kScanSpinLimit);
}
__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(kScanConsumerBar), "n"(kScanConsumers) : "memory");
}

// Thread 0: start the copies of chunk c into stage s.  Table rows
// [k0, k0 + nr) as one run of (nr - 1) * stride + W words; for every query the
// first nr & ~3 share words (the rest of a ragged last chunk is read by the
// consumers directly).
__device__ __forceinline__ void scan_issue(const ScanParams& p, uint32_t s, uint64_t c) {
    const uint64_t k0 = c * p.R;
    const uint32_t nr = (uint32_t)(p.K - k0 < p.R ? p.K - k0 : p.R), nr4 = nr & ~3u;
    const uint32_t tbytes = (uint32_t)(((uint64_t)(nr - 1) * p.stride + p.W) * 4u);
    const uint32_t sbytes = nr4 * 4u;
    const uint32_t bar = smem_addr(scan_sm) + 8u * s;
    const uint32_t dst = smem_addr(scan_sm + kScanHeader) + s * p.stage_bytes;
    mbar_expect_tx(bar, tbytes + p.B * sbytes);
    bulk_g2s(dst, p.T + k0 * p.stride, tbytes, bar);
    if (sbytes)
        for (uint32_t b = 0; b < p.B; ++b)
            bulk_g2s(dst + p.R * (uint32_t)p.stride * 4u + b * p.R * 4u, p.S + b * p.ld + k0, sbytes, bar);
}

// Partial sums of every consumer for BQ queries, met in shared memory (red,
// BQ x W words), then one u32 atomicAdd per (query, word) into out.  Called
// by every consumer thread (the issuing warp does not take part).
template <int BQ>
__device__ __forceinline__ void scan_flush(const ScanParams& p, uint32_t (&acc)[BQ][4], uint32_t* red, uint32_t* out,
                                           uint32_t cc, bool active) {
    const uint32_t tid = threadIdx.x;
    consumers_sync();  // red is free (a previous flush has finished reading it)
    for (uint32_t i = tid; i < BQ * p.W; i += kScanConsumers) red[i] = 0;
    consumers_sync();
    if (active) {
#pragma unroll
        for (int b = 0; b < BQ; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (acc[b][e]) atomicAdd(&red[b * p.W + 4u * cc + e], acc[b][e]);
                acc[b][e] = 0;
            }
    }
    consumers_sync();
    for (uint32_t i = tid; i < BQ * p.W; i += kScanConsumers)
        if (red[i]) atomicAdd(out + i, red[i]);
}

template <int BQ, bool DIAG>  // BQ: queries of this pass, exactly; DIAG: one bin's query per chunk (BQ = 1)
__global__ void __launch_bounds__(kScanThreads, 3) contract_scan_kernel(const ScanParams p) {
    static_assert(!DIAG || BQ == 1, "the diagonal form has one query per chunk");
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t full0 = smem_addr(scan_sm), empty0 = full0 + 32u;
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(scan_sm + 64);
    uint32_t* red = reinterpret_cast<uint32_t*>(scan_sm + kScanHeader + kScanStages * p.stage_bytes);
    if (tid == 0) {
        for (int s = 0; s < kScanStages; ++s) {
            mbar_init(full0 + 8u * s, 1);                     // the issuing thread's arrival + the copies' bytes
            mbar_init(empty0 + 8u * s, kScanConsumerWarps);   // one arrival per consumer warp
        }
        *abort_flag = 0u;
        fence_mbarrier_init();
    }
    __syncthreads();  // the only CTA-wide barrier
    // this CTA's chunks, c_first + j * c_step for c < c_end: dealt round-robin, or
    // (diagonal form) as one contiguous run, so that a bin's chunks stay together
    const uint64_t c_first = DIAG ? blockIdx.x * p.chunks_per_cta : blockIdx.x;
    const uint64_t c_step = DIAG ? 1 : gridDim.x;
    const uint64_t c_end = DIAG ? min(c_first + p.chunks_per_cta, p.nchunks) : p.nchunks;

    if (warp == kScanConsumerWarps) {
        // ---- the issuing warp: refill a stage once every consumer warp released it ----
        if (lane == 0) {
            uint64_t j = 0;
            for (uint64_t c = c_first; c < c_end; c += c_step, ++j) {
                const uint32_t s = (uint32_t)(j % kScanStages);
                if (j >= (uint64_t)kScanStages &&
                    !mbar_wait(empty0 + 8u * s, (uint32_t)((j / kScanStages - 1) & 1u))) {
                    atomicOr(&g_device_faults, PIR_FAULT_WAIT_TIMEOUT);
                    *abort_flag = 1u;
                    break;  // stop issuing; the consumers' bounded waits run out
                }
                fence_proxy_async_smem();  // consumers' reads before the refill
                scan_issue(p, s, c);
            }
            // the copies of the last stages issued are this thread's: see them land (bounded)
            // before it leaves
            const uint64_t first = j > (uint64_t)kScanStages ? j - kScanStages : 0;
            for (uint64_t jj = first; jj < j; ++jj)
                mbar_wait(full0 + 8u * (uint32_t)(jj % kScanStages), (uint32_t)((jj / kScanStages) & 1u));
        }
        return;
    }

    // ---- consumer (cc, rg): words 4cc..4cc+3 of rows 4rg..4rg+3 of every chunk (R <= 4 nrg) ----
    const uint32_t nc = p.W / 4, nrg = kScanConsumers / nc;
    const uint32_t cc = tid % nc, rg = tid / nc, i0 = 4u * rg;
    uint32_t acc[BQ][4];
#pragma unroll
    for (int b = 0; b < BQ; ++b)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[b][e] = 0;

    uint64_t j = 0, cur_bin = ~0ull;
    for (uint64_t c = c_first; c < c_end; c += c_step, ++j) {
        const uint32_t s = (uint32_t)(j % kScanStages), parity = (uint32_t)((j / kScanStages) & 1u);
        if (!mbar_wait(full0 + 8u * s, parity)) {
            if (lane == 0) atomicOr(&g_device_faults, PIR_FAULT_WAIT_TIMEOUT);
            *abort_flag = 1u;
        }
        const bool live = *abort_flag == 0u;  // after a failed wait the stages hold nothing trustworthy
        const uint64_t k0 = c * p.R;
        if constexpr (DIAG) {
            const uint64_t bin = k0 / p.bin_rows;  // chunks do not straddle bins
            if (bin != cur_bin) {
                if (cur_bin != ~0ull) scan_flush<BQ>(p, acc, red, p.out + cur_bin * p.W, cc, rg < nrg && live);
                cur_bin = bin;
            }
        }
        const uint32_t nr = (uint32_t)(p.K - k0 < p.R ? p.K - k0 : p.R), nr4 = nr & ~3u;
        const char* stage = scan_sm + kScanHeader + s * p.stage_bytes;
        const uint32_t* sS = reinterpret_cast<const uint32_t*>(stage + p.R * (uint32_t)p.stride * 4u);
        if (live && rg < nrg && i0 + 4u <= nr4) {
            // four whole rows: 128-bit loads of the table words and of each query's four shares
            uint4 t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                t[u] = *reinterpret_cast<const uint4*>(stage + ((uint64_t)(i0 + u) * p.stride + 4u * cc) * 4u);
#pragma unroll
            for (int b = 0; b < BQ; ++b) {
                const uint4 y = *reinterpret_cast<const uint4*>(sS + b * p.R + i0);
                acc[b][0] += y.x * t[0].x + y.y * t[1].x + y.z * t[2].x + y.w * t[3].x;
                acc[b][1] += y.x * t[0].y + y.y * t[1].y + y.z * t[2].y + y.w * t[3].y;
                acc[b][2] += y.x * t[0].z + y.y * t[1].z + y.z * t[2].z + y.w * t[3].z;
                acc[b][3] += y.x * t[0].w + y.y * t[1].w + y.z * t[2].w + y.w * t[3].w;
            }
        } else if (live && rg < nrg && i0 < nr) {
            // the ragged end of the last chunk: shares past nr & ~3 were not copied
            for (uint32_t i = i0; i < i0 + 4u && i < nr; ++i) {
                const uint4 t = *reinterpret_cast<const uint4*>(stage + ((uint64_t)i * p.stride + 4u * cc) * 4u);
#pragma unroll
                for (int b = 0; b < BQ; ++b) {
                    const uint32_t y = i < nr4 ? sS[b * p.R + i] : __ldg(p.S + b * p.ld + k0 + i);
                    acc[b][0] += y * t.x;
                    acc[b][1] += y * t.y;
                    acc[b][2] += y * t.z;
                    acc[b][3] += y * t.w;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8u * s);  // this warp is done with stage s
    }
    const bool live = *abort_flag == 0u;
    if (DIAG) {
        if (cur_bin != ~0ull) scan_flush<BQ>(p, acc, red, p.out + cur_bin * p.W, cc, rg < nrg && live);
    } else {
        scan_flush<BQ>(p, acc, red, p.out, cc, rg < nrg && live);
    }
}

// Diagnostic: one thread waits on an mbarrier that expects an arrival nobody
// makes; the bounded wait gives up after `polls` polls and records it, exactly
// as a scan consumer whose copy never lands would.
__global__ void wait_selftest_kernel(uint32_t polls, uint32_t* gave_up) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_addr(&bar);
    mbar_init(b, 1);
    fence_mbarrier_init();
    bool done = false;
    for (uint32_t i = 0; i < polls && !done; ++i) done = mbar_try_wait(b, 0);
    if (!done) atomicOr(&g_device_faults, PIR_FAULT_WAIT_TIMEOUT);
    *gave_up = done ? 0u : 1u;
}

// dst[i] = src[i] for i < words, either side in device memory or in pinned
// host memory mapped into the device's address space (the staged host call's
// keys in and shares out).  Reads bypass the caches (the host rewrites its
// side between launches).
__global__ void __launch_bounds__(256) words_copy_kernel(const uint32_t* __restrict__ src,
                                                         uint32_t* __restrict__ dst, uint64_t words) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = __ldcv(src + i);
}

}  // namespace dev

int launch_words_copy(const uint32_t* src, uint32_t* dst, uint64_t words, void* stream) {
    if (words == 0) return PIR_OK;
    const uint64_t blocks = std::min<uint64_t>((words + 255) / 256, 64);
    dev::words_copy_kernel<<<(uint32_t)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(src, dst, words);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "words copy launch");
}

int selftest_bounded_wait(uint32_t polls, void* stream) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail((int)e, "selftest alloc");
    dev::wait_selftest_kernel<<<1, 32, 0, s>>>(polls, d);
    uint32_t gave_up = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&gave_up, d, sizeof(gave_up), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail((int)e, "selftest");
    return gave_up ? PIR_ERR_TIMEOUT : PIR_OK;
}

bool scan_supported(const uint32_t* shares, uint64_t ld, const uint32_t* table, uint64_t stride, uint32_t width) {
    return (reinterpret_cast<uintptr_t>(shares) & 15u) == 0 && ld % 4 == 0 &&
           (reinterpret_cast<uintptr_t>(table) & 15u) == 0 && stride % 4 == 0 && width % 4 == 0 &&
           stride <= dev::kScanMaxWidth;
}

static uint32_t scan_rows_per_chunk(uint64_t stride, uint32_t width) {
    uint32_t R = (uint32_t)(dev::kScanTableStageBytes / (stride * 4u)) & ~3u;
    R = std::min(dev::kScanMaxRows, std::max(4u, R));
    return std::min(R, 4u * (uint32_t)(dev::kScanConsumers / (width / 4u)));  // four rows per consumer thread
}

static dev::ScanParams scan_params(uint64_t ld, const uint32_t* table, uint64_t stride, uint32_t width,
                                   uint64_t rows) {
    dev::ScanParams p{};
    p.ld = ld;
    p.T = table;
    p.stride = stride;
    p.K = rows;
    p.W = width;
    p.R = scan_rows_per_chunk(stride, width);
    p.nchunks = (rows + p.R - 1) / p.R;
    p.stage_bytes = p.R * (uint32_t)stride * 4u + 8u * p.R * 4u;
    return p;
}

// Sets the kernel's shared memory (stages + the reduction area for B queries)
// and launches it on as many CTAs as fit (at most one per chunk); `ctas` gets
// the grid size before the launch through `fix` (the diagonal form needs it).
template <typename Fix>
static int launch_scan_kernel(void (*kern)(dev::ScanParams), dev::ScanParams p, uint32_t B, cudaStream_t s, Fix fix) {
    using namespace dev;
    const size_t smem = kScanHeader + (size_t)kScanStages * p.stage_bytes + (((size_t)B * p.W * 4u + 15u) & ~15ull);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kScanThreads, smem);
    if (e != cudaSuccess) return cuda_fail((int)e, "scan setup");
    const int sms = std::max(1, device_sm_count());
    const uint64_t ctas = std::min<uint64_t>(p.nchunks, (uint64_t)sms * (uint64_t)std::max(1, per_sm));
    fix(p, ctas);
    kern<<<(uint32_t)ctas, kScanThreads, smem, s>>>(p);
    e = cudaGetLastError();
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "scan launch");
}

int launch_scan(const uint32_t* shares, uint64_t ld, uint32_t batch, const uint32_t* table, uint64_t stride,
                uint32_t width, uint64_t rows, uint32_t* out, void* stream) {
    using namespace dev;
    if (!scan_supported(shares, ld, table, stride, width)) return PIR_ERR_UNSUPPORTED;
    ScanParams p = scan_params(ld, table, stride, width, rows);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void (*const kerns[8])(ScanParams) = {contract_scan_kernel<1, false>, contract_scan_kernel<2, false>,
                                          contract_scan_kernel<3, false>, contract_scan_kernel<4, false>,
                                          contract_scan_kernel<5, false>, contract_scan_kernel<6, false>,
                                          contract_scan_kernel<7, false>, contract_scan_kernel<8, false>};
    // eight queries per pass; each pass streams the whole table once
    for (uint32_t b0 = 0; b0 < batch; b0 += 8) {
        p.B = std::min(8u, batch - b0);
        p.S = shares + (uint64_t)b0 * ld;
        p.out = out + (uint64_t)b0 * width;
        const int rc = launch_scan_kernel(kerns[p.B - 1], p, p.B, s, [](ScanParams&, uint64_t) {});
        if (rc != PIR_OK) return rc;
    }
    return PIR_OK;
}

bool scan_bins_supported(const uint32_t* table, uint64_t stride, uint32_t width, uint64_t bin_rows) {
    return (reinterpret_cast<uintptr_t>(table) & 15u) == 0 && stride % 4 == 0 && width % 4 == 0 &&
           stride <= dev::kScanMaxWidth && bin_rows % scan_rows_per_chunk(stride, width) == 0;
}

int launch_scan_bins(const uint32_t* shares, const uint32_t* table, uint64_t stride, uint32_t width, uint64_t rows,
                     uint64_t bin_rows, uint32_t* out, void* stream) {
    using namespace dev;
    if ((reinterpret_cast<uintptr_t>(shares) & 15u) != 0 || !scan_bins_supported(table, stride, width, bin_rows))
        return PIR_ERR_UNSUPPORTED;
    ScanParams p = scan_params(0, table, stride, width, rows);
    p.B = 1;
    p.S = shares;
    p.out = out;
    p.bin_rows = bin_rows;
    return launch_scan_kernel(contract_scan_kernel<1, true>, p, 1, reinterpret_cast<cudaStream_t>(stream),
                              [](ScanParams& q, uint64_t ctas) { q.chunks_per_cta = (q.nchunks + ctas - 1) / ctas; });
}

int device_faults(uint32_t* flags, bool clear) {
    uint32_t v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, dev::g_device_faults, sizeof(v));
    if (e != cudaSuccess) return cuda_fail((int)e, "read device faults");
    if (clear && v) {
        const uint32_t zero = 0;
        e = cudaMemcpyToSymbol(dev::g_device_faults, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail((int)e, "clear device faults");
    }
    *flags = v;
    return PIR_OK;
}

uint32_t* device_fault_word() {
    void* p = nullptr;
    return cudaGetSymbolAddress(&p, dev::g_device_faults) == cudaSuccess ? static_cast<uint32_t*>(p) : nullptr;
}

}  // namespace pir
