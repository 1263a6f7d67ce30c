// pir_server_eval_noalloc: the host-key / host-share server evaluation without
// any device allocation.
//
// pir_server_eval stages the caller's keys and the shares in device buffers
// it allocates per call.  Some callers cannot let a library allocate device
// memory: a serving runtime that owns the whole device-memory budget and
// hands none of it to plug-ins, or a request path that must not take the
// allocator's locks or risk the implicit device synchronisation an
// allocation can cause.  This entry point stages through one fixed region of
// device memory that is part of the library image instead.
//
// The region is a file-scope __device__ array (kScratchBytes, 256 KiB): every
// GPU that loads the library holds it until the process exits.  In host code
// the array's name is only a host-side stand-in, so its device address is
// looked up with cudaGetSymbolAddress once per device (with that device
// current) on the first call made on that device, and passed to the kernel.
// A device whose primary context is destroyed and created again
// (cudaDeviceReset) gets the array at a new address: the lookup is kept with
// the context's unique ID and repeated when the current context's ID differs.
// All calls share the region and it keeps the last call's contents: the
// share area is cleared at the start of every call, and calls whose work
// overlaps on the GPU (concurrent streams, or other host threads) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace pir {
namespace {

constexpr size_t kScratchBytes = 256u * 1024u;
constexpr size_t kKeyAreaBytes = 192u * 1024u;  // staged keys: [0, 192 KiB)
constexpr size_t kShareAreaBytes = kScratchBytes - kKeyAreaBytes;  // staged shares: [192 KiB, 256 KiB)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_scratch[kScratchBytes];

std::mutex g_setup_mutex;
uint8_t* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // unique ID of the context the address belongs to

// The driver's current context and its unique ID, through the runtime's
// driver entry points (the library does not link the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    return get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_scratch on the current device: looked up on the first
// call on the device, and again once its context has been replaced.
int scratch_for_current_device(uint8_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail((int)e, "noalloc: current device");
    if (dev < 0 || dev >= kMaxDevices) return PIR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long ctx = 0;
    const bool have_ctx = current_context_id(&ctx);
    if (!g_scratch_ptr[dev] || !have_ctx || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);  // makes the device's primary context current
        if (e != cudaSuccess) return cuda_fail((int)e, "noalloc: scratch address");
        g_scratch_ptr[dev] = static_cast<uint8_t*>(p);
        g_scratch_ctx[dev] = current_context_id(&ctx) ? ctx : 0;
    }
    *out = g_scratch_ptr[dev];
    return PIR_OK;
}

}  // namespace
}  // namespace pir

extern "C" int pir_server_eval_noalloc(const pir_table* t, const uint8_t* keys, size_t batch, uint32_t* out,
                                       void* stream) {
    using namespace pir;
    if (!t || !t->data || !keys || !out || batch == 0 || t->rows < 1 || t->width < 1 || t->stride < t->width ||
        (reinterpret_cast<uintptr_t>(t->data) & 3u) != 0)
        return PIR_ERR_ARG;
    {  // `out` is written by a device-to-host copy: it must be host memory
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, out) != cudaSuccess)
            cudaGetLastError();  // unregistered host memory on older runtimes
        else if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
            return PIR_ERR_ARG;
    }
    const uint32_t n = pir_domain_bits(t->rows);
    if (n == 0) return PIR_ERR_DOMAIN;
    const size_t kb = key_bytes(n);
    const size_t share_bytes = batch * (size_t)t->width * sizeof(uint32_t);
    if (batch > kKeyAreaBytes / kb || share_bytes > kShareAreaBytes) return PIR_ERR_UNSUPPORTED;
    for (size_t q = 0; q < batch; ++q) {
        uint32_t kn = 0, party = 0;
        const uint8_t* k = keys + q * kb;
        if (pir_key_check(k, key_bytes(k[5] <= PIR_MAX_DOMAIN_BITS ? k[5] : 0), &kn, &party) != PIR_OK)
            return PIR_ERR_KEY;
        if (kn != n) return PIR_ERR_DOMAIN;
    }
    uint8_t* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != PIR_OK) return rc;
    uint8_t* dkeys = scratch;
    uint32_t* dshares = reinterpret_cast<uint32_t*>(scratch + kKeyAreaBytes);

    const bool vec = (reinterpret_cast<uintptr_t>(t->data) & 15u) == 0 && t->stride % 4 == 0 && t->width % 4 == 0;
    pir_plan plan{};
    rc = plan_fused(t->rows, 0, n, t->width, (uint32_t)batch, vec, &plan);
    if (rc != PIR_OK) return rc;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dkeys, keys, batch * kb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail((int)e, "noalloc: copy keys");
    e = cudaMemsetAsync(dshares, 0, share_bytes, s);  // the kernel accumulates into the shares
    if (e != cudaSuccess) return cuda_fail((int)e, "noalloc: clear shares");
    EvalRequest req{};
    req.table = t->data;
    req.row_lo = 0;
    req.row_hi = t->rows;
    req.width = t->width;
    req.stride = t->stride;
    req.n = n;
    req.dkeys = dkeys;
    req.batch = (uint32_t)batch;
    req.dout = dshares;
    req.dstatus = nullptr;
    rc = launch_fused(req, plan, stream);
    if (rc != PIR_OK) return rc;
    e = cudaMemcpyAsync(out, dshares, share_bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail((int)e, "noalloc: copy shares");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail((int)e, "noalloc: synchronize");
    return PIR_OK;
}
